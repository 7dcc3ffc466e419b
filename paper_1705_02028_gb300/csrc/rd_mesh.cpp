// rd_mesh.cpp -- host side of the mesh store: validation, geometry, reordering, CSR.
//
// Geometry follows Sec. 3.2 of the paper: for a counter-clockwise triangle the
// inward normal n_i of the edge opposite corner i has |n_i| = edge length, the
// normals sum to zero, |T| is the signed area and l_max^T the longest edge; the
// nodal volume is V_i = sum_{T containing i} |T| / 3.  Periodic boundaries are
// "handled by the mesh" (Sec. 3.5): a corner reached across the boundary is
// placed at its periodic image xy + (dx Lx, dy Ly).
//
// Reordering restores data locality (Sec. 4.1.4 uses Morton order): vertices
// are sorted by the Morton code of their coordinates (or by reverse
// Cuthill-McKee), triangles by their smallest internal vertex id.  The
// vertex -> (triangle, corner) CSR lists the incident corners of every vertex
// in ascending triangle order; the update kernels gather through it instead of
// the atomic scatter of Sec. 4.2.1, so results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <queue>

#include "rd_internal.h"

namespace rd {

namespace {

uint32_t spread16(uint32_t x) {
  x &= 0xFFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

void morton_order(int32_t nv, const double* xy, std::vector<int32_t>& perm) {
  double x0 = xy[0], x1 = xy[0], y0 = xy[1], y1 = xy[1];
  for (int32_t i = 1; i < nv; ++i) {
    x0 = std::min(x0, xy[2 * i]); x1 = std::max(x1, xy[2 * i]);
    y0 = std::min(y0, xy[2 * i + 1]); y1 = std::max(y1, xy[2 * i + 1]);
  }
  double sx = x1 > x0 ? 65535.0 / (x1 - x0) : 0.0, sy = y1 > y0 ? 65535.0 / (y1 - y0) : 0.0;
  std::vector<uint64_t> key(nv);
  for (int32_t i = 0; i < nv; ++i) {
    uint32_t qx = (uint32_t)std::min(65535.0, std::max(0.0, std::floor((xy[2 * i] - x0) * sx)));
    uint32_t qy = (uint32_t)std::min(65535.0, std::max(0.0, std::floor((xy[2 * i + 1] - y0) * sy)));
    uint32_t code = spread16(qx) | (spread16(qy) << 1);
    key[i] = ((uint64_t)code << 32) | (uint32_t)i;
  }
  std::sort(key.begin(), key.end());
  perm.resize(nv);
  for (int32_t i = 0; i < nv; ++i) perm[i] = (int32_t)(key[i] & 0xFFFFFFFFu);
}

void rcm_order(int32_t nv, int32_t nt, const int32_t* tri, std::vector<int32_t>& perm) {
  // vertex graph from triangle edges
  std::vector<std::vector<int32_t>> adj(nv);
  for (int32_t t = 0; t < nt; ++t)
    for (int c = 0; c < 3; ++c) {
      int32_t a = tri[3 * t + c], b = tri[3 * t + (c + 1) % 3];
      adj[a].push_back(b);
      adj[b].push_back(a);
    }
  std::vector<int32_t> deg(nv);
  for (int32_t i = 0; i < nv; ++i) {
    auto& a = adj[i];
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
    deg[i] = (int32_t)a.size();
  }
  std::vector<int32_t> by_deg(nv);
  std::iota(by_deg.begin(), by_deg.end(), 0);
  std::stable_sort(by_deg.begin(), by_deg.end(), [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
  std::vector<char> seen(nv, 0);
  std::vector<int32_t> order;
  order.reserve(nv);
  for (int32_t s : by_deg) {
    if (seen[s]) continue;
    std::queue<int32_t> q;
    q.push(s);
    seen[s] = 1;
    while (!q.empty()) {
      int32_t v = q.front();
      q.pop();
      order.push_back(v);
      std::vector<int32_t> nb;
      for (int32_t w : adj[v])
        if (!seen[w]) { seen[w] = 1; nb.push_back(w); }
      std::stable_sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
      for (int32_t w : nb) q.push(w);
    }
  }
  std::reverse(order.begin(), order.end());
  perm = order;
}

}  // namespace

int build_host_mesh(int32_t nv, const double* xy, int32_t nt, const int32_t* tri,
                    const int8_t* shift, double Lx, double Ly, int32_t reorder, HostMesh& m) {
  if (nv < 3 || nt < 1 || !xy || !tri) return RD_EINVAL;
  if ((int64_t)nt * 3 >= (int64_t)INT32_MAX) return RD_EINVAL;
  if (reorder < RD_ORDER_NONE || reorder > RD_ORDER_RCM) return RD_EINVAL;
  for (int64_t e = 0; e < 3 * (int64_t)nt; ++e)
    if (tri[e] < 0 || tri[e] >= nv) return RD_EINVAL;
  if (shift) {
    for (int64_t e = 0; e < 6 * (int64_t)nt; ++e)
      if (shift[e] < -1 || shift[e] > 1) return RD_EINVAL;
    if (!(Lx > 0) || !(Ly > 0)) return RD_EINVAL;
  }
  for (int64_t e = 0; e < 2 * (int64_t)nv; ++e)
    if (!std::isfinite(xy[e])) return RD_EINVAL;

  m = HostMesh();
  m.nv = nv; m.nt = nt; m.Lx = Lx; m.Ly = Ly;

  // vertex order
  if (reorder == RD_ORDER_MORTON) {
    morton_order(nv, xy, m.vperm);
  } else if (reorder == RD_ORDER_RCM) {
    rcm_order(nv, nt, tri, m.vperm);
  } else {
    m.vperm.resize(nv);
    std::iota(m.vperm.begin(), m.vperm.end(), 0);
  }
  m.vinv.assign(nv, -1);
  for (int32_t i = 0; i < nv; ++i) m.vinv[m.vperm[i]] = i;

  // triangle order: by smallest internal vertex id, ties by caller id
  std::vector<uint64_t> tkey(nt);
  for (int32_t t = 0; t < nt; ++t) {
    int32_t a = m.vinv[tri[3 * t]], b = m.vinv[tri[3 * t + 1]], c = m.vinv[tri[3 * t + 2]];
    uint32_t k = (uint32_t)std::min(a, std::min(b, c));
    tkey[t] = ((uint64_t)k << 32) | (uint32_t)t;
  }
  if (reorder != RD_ORDER_NONE) std::sort(tkey.begin(), tkey.end());
  m.tperm.resize(nt);
  for (int32_t t = 0; t < nt; ++t) m.tperm[t] = (int32_t)(tkey[t] & 0xFFFFFFFFu);

  // connectivity and geometry in internal order
  m.tri.resize(3 * (size_t)nt);
  m.nx.resize(3 * (size_t)nt); m.ny.resize(3 * (size_t)nt); m.hl.resize(3 * (size_t)nt);
  m.area.resize(nt); m.lmax.resize(nt);
  m.V.assign(nv, 0.0);
  for (int32_t t = 0; t < nt; ++t) {
    int32_t to = m.tperm[t];
    double x[3], y[3];
    for (int c = 0; c < 3; ++c) {
      int32_t v = tri[3 * to + c];
      double dx = shift ? shift[6 * (size_t)to + 2 * c] : 0.0, dy = shift ? shift[6 * (size_t)to + 2 * c + 1] : 0.0;
      x[c] = xy[2 * v] + dx * Lx;
      y[c] = xy[2 * v + 1] + dy * Ly;
      m.tri[(size_t)c * nt + t] = m.vinv[v];
    }
    double A = 0.5 * ((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]));
    if (!(A > 0.0)) return RD_EINVAL;
    double lm = 0.0;
    for (int c = 0; c < 3; ++c) {
      int a = (c + 1) % 3, b = (c + 2) % 3;
      double nxx = y[a] - y[b], nyy = x[b] - x[a];
      double len = std::sqrt(nxx * nxx + nyy * nyy);
      if (!(len > 0.0)) return RD_EINVAL;
      m.nx[(size_t)c * nt + t] = nxx / len;
      m.ny[(size_t)c * nt + t] = nyy / len;
      m.hl[(size_t)c * nt + t] = len / 2.0;
      lm = std::max(lm, len);
    }
    m.area[t] = A;
    m.lmax[t] = lm;
    for (int c = 0; c < 3; ++c) m.V[m.tri[(size_t)c * nt + t]] += A / 3.0;
  }

  // CSR vertex -> (triangle, corner)
  m.csr_ptr.assign(nv + 1, 0);
  for (int64_t e = 0; e < 3 * (int64_t)nt; ++e) m.csr_ptr[m.tri[e] + 1]++;
  for (int32_t i = 0; i < nv; ++i) {
    if (m.csr_ptr[i + 1] == 0) return RD_EINVAL;  // vertex in no triangle
    m.csr_ptr[i + 1] += m.csr_ptr[i];
  }
  m.csr_ent.resize(3 * (size_t)nt);
  std::vector<int32_t> fill(m.csr_ptr.begin(), m.csr_ptr.end() - 1);
  for (int32_t t = 0; t < nt; ++t)
    for (int c = 0; c < 3; ++c) m.csr_ent[fill[m.tri[(size_t)c * nt + t]]++] = 3 * t + c;
  return RD_OK;
}

}  // namespace rd
