// rd_partition.cpp -- host plan of a vertex partition of the mesh store.
//
// The step of Sec. 3.4 reads, per triangle, the states of its three corners
// and writes shares that each corner gathers.  Part r of P owns the
// contiguous internal (Morton or RCM ordered) vertex range
// [r nv / P, (r + 1) nv / P) and computes every triangle that has a corner it
// owns -- a triangle whose corners belong to several parts is computed by each
// of them, with identical inputs and code, so no share crosses a part
// boundary.  The corners it does not own are its ghost vertices; their states
// are received from their owners before each stage (W^n before stage 1, W*
// before stage 2), and the dt of a step is the minimum of the parts' minima.
// Each owned vertex gathers its shares in the order of the global CSR (local
// triangles keep the global order), so a partitioned step is bitwise equal to
// the single-part step.
#include <algorithm>

#include "rd_internal.h"

namespace rd {

int build_part_plan(const HostMesh& h, int P, int r, PartPlanHost& out) {
  if (P < 1 || r < 0 || r >= P || P > h.nv) return RD_EINVAL;
  const int32_t nv = h.nv, nt = h.nt;
  auto lo = [&](int q) { return (int32_t)((int64_t)q * nv / P); };
  auto owner = [&](int32_t v) {
    int q = (int)((int64_t)v * P / nv);  // first guess, then correct by the exact bounds
    while (q > 0 && v < lo(q)) --q;
    while (q < P - 1 && v >= lo(q + 1)) ++q;
    return q;
  };
  PartPlanHost p;
  p.P = P;
  p.r = r;
  p.v0 = lo(r);
  p.v1 = lo(r + 1);
  // local triangles: every triangle with an owned corner, ascending
  std::vector<int32_t> tris;
  for (int32_t v = p.v0; v < p.v1; ++v)
    for (int32_t e = h.csr_ptr[v]; e < h.csr_ptr[v + 1]; ++e) tris.push_back(h.csr_ent[e] / 3);
  std::sort(tris.begin(), tris.end());
  tris.erase(std::unique(tris.begin(), tris.end()), tris.end());
  p.lt = tris;
  // ghost vertices: corners of local triangles outside the owned range, ascending
  std::vector<int32_t> ghosts;
  for (int32_t t : tris)
    for (int c = 0; c < 3; ++c) {
      const int32_t v = h.tri[(size_t)c * nt + t];
      if (v < p.v0 || v >= p.v1) ghosts.push_back(v);
    }
  std::sort(ghosts.begin(), ghosts.end());
  ghosts.erase(std::unique(ghosts.begin(), ghosts.end()), ghosts.end());
  const int32_t n_own = p.v1 - p.v0;
  p.lv.resize((size_t)n_own + ghosts.size());
  for (int32_t i = 0; i < n_own; ++i) p.lv[i] = p.v0 + i;
  for (size_t g = 0; g < ghosts.size(); ++g) p.lv[n_own + g] = ghosts[g];
  // receive slices: the ghosts owned by each part, in ascending order
  p.recv_ptr.assign(P + 1, 0);
  for (int32_t g : ghosts) p.recv_ptr[owner(g) + 1]++;
  for (int q = 0; q < P; ++q) p.recv_ptr[q + 1] += p.recv_ptr[q];
  // local corners and CSR of the owned vertices (entries 3 lt + c, ascending)
  const int32_t nlt = (int32_t)tris.size();
  p.ltri.resize(3 * (size_t)nlt);
  for (int32_t k = 0; k < nlt; ++k)
    for (int c = 0; c < 3; ++c) {
      const int32_t v = h.tri[(size_t)c * nt + tris[k]];
      int32_t l;
      if (v >= p.v0 && v < p.v1) {
        l = v - p.v0;
      } else {
        l = n_own + (int32_t)(std::lower_bound(ghosts.begin(), ghosts.end(), v) - ghosts.begin());
      }
      p.ltri[(size_t)c * nlt + k] = l;
    }
  p.csr_ptr.assign(n_own + 1, 0);
  p.csr_ent.clear();
  for (int32_t i = 0; i < n_own; ++i) {
    const int32_t v = p.v0 + i;
    for (int32_t e = h.csr_ptr[v]; e < h.csr_ptr[v + 1]; ++e) {
      const int32_t t = h.csr_ent[e] / 3, c = h.csr_ent[e] % 3;
      const int32_t k = (int32_t)(std::lower_bound(tris.begin(), tris.end(), t) - tris.begin());
      p.csr_ent.push_back(3 * k + c);
    }
    p.csr_ptr[i + 1] = (int32_t)p.csr_ent.size();
  }
  // send lists: owned vertices that part q holds as ghosts, i.e. owned vertices
  // sharing a triangle with a vertex q owns, ascending (q's ghost order)
  std::vector<std::vector<int32_t>> send(P);
  for (int32_t i = 0; i < n_own; ++i) {
    const int32_t v = p.v0 + i;
    int last = -1;
    std::vector<int> peers;
    for (int32_t e = h.csr_ptr[v]; e < h.csr_ptr[v + 1]; ++e) {
      const int32_t t = h.csr_ent[e] / 3;
      for (int c = 0; c < 3; ++c) {
        const int q = owner(h.tri[(size_t)c * nt + t]);
        if (q != r) peers.push_back(q);
      }
    }
    std::sort(peers.begin(), peers.end());
    for (int q : peers)
      if (q != last) {
        send[q].push_back(i);
        last = q;
      }
  }
  p.send_ptr.assign(P + 1, 0);
  p.send_idx.clear();
  for (int q = 0; q < P; ++q) {
    p.send_idx.insert(p.send_idx.end(), send[q].begin(), send[q].end());
    p.send_ptr[q + 1] = (int32_t)p.send_idx.size();
  }
  out = std::move(p);
  return RD_OK;
}

}  // namespace rd

// Host-only plan for callers without a GPU (and for tests of the exchange
// logic): builds the mesh store on the host and returns part `part` of
// `n_parts`.  Two-call pattern: sizes first (arrays NULL), then the arrays.
extern "C" int rd_partition_plan(int32_t n_vertex, const double* xy, int32_t n_tri, const int32_t* tri,
                                 const int8_t* image_shift, double Lx, double Ly, int32_t reorder, int32_t n_parts,
                                 int32_t part, int32_t sizes[4], int32_t* local_vertices, int32_t* local_triangles,
                                 int32_t* local_corners, int32_t* csr_ptr, int32_t* csr_ent, int32_t* send_ptr,
                                 int32_t* send_idx, int32_t* recv_ptr) {
  if (!sizes) return RD_EINVAL;
  rd::HostMesh h;
  int st = rd::build_host_mesh(n_vertex, xy, n_tri, tri, image_shift, Lx, Ly, reorder, h);
  if (st != RD_OK) return st;
  rd::PartPlanHost p;
  st = rd::build_part_plan(h, n_parts, part, p);
  if (st != RD_OK) return st;
  const int32_t n_own = p.v1 - p.v0, nlt = (int32_t)p.lt.size();
  sizes[0] = n_own;
  sizes[1] = (int32_t)p.lv.size() - n_own;
  sizes[2] = nlt;
  sizes[3] = (int32_t)p.send_idx.size();
  if (local_vertices)
    for (size_t i = 0; i < p.lv.size(); ++i) local_vertices[i] = h.vperm[p.lv[i]];
  if (local_triangles)
    for (int32_t k = 0; k < nlt; ++k) local_triangles[k] = h.tperm[p.lt[k]];
  if (local_corners) std::copy(p.ltri.begin(), p.ltri.end(), local_corners);
  if (csr_ptr) std::copy(p.csr_ptr.begin(), p.csr_ptr.end(), csr_ptr);
  if (csr_ent) std::copy(p.csr_ent.begin(), p.csr_ent.end(), csr_ent);
  if (send_ptr) std::copy(p.send_ptr.begin(), p.send_ptr.end(), send_ptr);
  if (send_idx) std::copy(p.send_idx.begin(), p.send_idx.end(), send_idx);
  if (recv_ptr) std::copy(p.recv_ptr.begin(), p.recv_ptr.end(), recv_ptr);
  return RD_OK;
}
