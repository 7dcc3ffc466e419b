// rd_boundary.cu -- boundary conditions of the mesh store (Sec. 3.5):
// ghost vertices held at their initial state (non-reflecting / inflow
// boundaries) and weakly imposed reflecting walls (correction flux split
// between the edge's two vertices with the parameter alpha).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rd_device.h"
#include "rd_kernels.cuh"

using namespace rd;

namespace {

// True if the edge opposite corner c of internal triangle t is shared with
// another triangle (the same geometric edge traversed the other way: equal
// endpoints and an exactly opposite unit normal).
bool interior_edge(const HostMesh& h, int32_t t, int c) {
  const size_t nt = h.nt;
  const int32_t a = h.tri[(size_t)((c + 1) % 3) * nt + t], b = h.tri[(size_t)((c + 2) % 3) * nt + t];
  const double nx = h.nx[(size_t)c * nt + t], ny = h.ny[(size_t)c * nt + t];
  for (int32_t e = h.csr_ptr[a]; e < h.csr_ptr[a + 1]; ++e) {
    const int32_t t2 = h.csr_ent[e] / 3;
    if (t2 == t) continue;
    for (int c2 = 0; c2 < 3; ++c2) {
      const int32_t a2 = h.tri[(size_t)((c2 + 1) % 3) * nt + t2], b2 = h.tri[(size_t)((c2 + 2) % 3) * nt + t2];
      if (a2 == b && b2 == a && h.nx[(size_t)c2 * nt + t2] == -nx && h.ny[(size_t)c2 * nt + t2] == -ny) return true;
    }
  }
  return false;
}

int upload_i32(DevBuf& b, const std::vector<int32_t>& v, cudaStream_t st) {
  dev_free(b);
  if (v.empty()) return RD_OK;
  CK(dev_alloc(b, v.size() * sizeof(int32_t), st));
  CU(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));
  return RD_OK;
}

}  // namespace

namespace rd {

// Wall geometry in precision T on the device (built on first use).
template <class T>
int mesh_wall_geometry(rd_mesh* m) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  if (m->n_wall == 0 || m->wgeo_ready[pi]) return RD_OK;
  std::vector<T> tmp(m->wgeo_host.size());
  for (size_t i = 0; i < tmp.size(); ++i) tmp[i] = (T)m->wgeo_host[i];
  dev_free(m->wgeo[pi]);
  CK(dev_alloc(m->wgeo[pi], tmp.size() * sizeof(T), m->stream));
  CU(cudaMemcpyAsync(m->wgeo[pi].p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, m->stream));
  CU(cudaStreamSynchronize(m->stream));
  m->wgeo_ready[pi] = true;
  return RD_OK;
}
template int mesh_wall_geometry<double>(rd_mesh*);
template int mesh_wall_geometry<float>(rd_mesh*);

void mesh_boundary_free(rd_mesh* m) {
  dev_free(m->ghost_of);
  dev_free(m->ghost_ids);
  dev_free(m->wptr);
  dev_free(m->wother);
  for (int p = 0; p < 2; ++p) {
    dev_free(m->wgeo[p]);
    m->wgeo_ready[p] = false;
  }
  m->wgeo_host.clear();
  m->n_ghost = m->n_wall = 0;
}

}  // namespace rd

extern "C" int rd_mesh_set_boundary(rd_mesh* m, const uint8_t* ghost, int32_t n_wall, const int32_t* wall,
                                    double alpha) {
  if (!m || n_wall < 0 || (n_wall > 0 && !wall)) return RD_EINVAL;
  if (!(alpha >= 0.0 && alpha <= 1.0)) return RD_EINVAL;
  const HostMesh& h = m->h;
  const int32_t nv = h.nv, nt = h.nt;
  // caller triangle -> internal triangle
  std::vector<int32_t> tinv(nt);
  for (int32_t t = 0; t < nt; ++t) tinv[h.tperm[t]] = t;
  // wall ends, validated
  std::vector<std::pair<int32_t, int32_t>> ends;  // (internal vertex, wall index * 2 + end)
  std::vector<int32_t> wt(n_wall), wc(n_wall);
  std::vector<uint64_t> seen;
  for (int32_t w = 0; w < n_wall; ++w) {
    const int32_t t = wall[2 * w], c = wall[2 * w + 1];
    if (t < 0 || t >= nt || c < 0 || c > 2) return RD_EINVAL;
    wt[w] = tinv[t];
    wc[w] = c;
    if (interior_edge(h, wt[w], c)) return RD_EINVAL;  // not on the boundary
    seen.push_back(((uint64_t)wt[w] << 2) | (uint64_t)c);
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return RD_EINVAL;  // listed twice

  // ghost vertices (caller order -> internal)
  std::vector<int32_t> ghost_of(nv, -1), ghost_ids;
  if (ghost)
    for (int32_t v = 0; v < nv; ++v)
      if (ghost[v]) {
        ghost_of[h.vinv[v]] = 0;
      }
  for (int32_t i = 0; i < nv; ++i)
    if (ghost_of[i] >= 0) {
      ghost_of[i] = (int32_t)ghost_ids.size();
      ghost_ids.push_back(i);
    }

  // wall CSR over internal vertices: each edge contributes one entry to each end
  std::vector<int32_t> wptr(nv + 1, 0), wother(2 * (size_t)n_wall);
  std::vector<double> wgeo(6 * (size_t)n_wall);
  for (int32_t w = 0; w < n_wall; ++w) {
    const int32_t t = wt[w], c = wc[w];
    wptr[h.tri[(size_t)((c + 1) % 3) * nt + t] + 1]++;
    wptr[h.tri[(size_t)((c + 2) % 3) * nt + t] + 1]++;
  }
  for (int32_t i = 0; i < nv; ++i) wptr[i + 1] += wptr[i];
  std::vector<int32_t> fill(wptr.begin(), wptr.end() - 1);
  for (int32_t w = 0; w < n_wall; ++w) {
    const int32_t t = wt[w], c = wc[w];
    const int32_t a = h.tri[(size_t)((c + 1) % 3) * nt + t], b = h.tri[(size_t)((c + 2) % 3) * nt + t];
    // outward normal of the wall = minus the inward normal of the edge in its triangle
    const double nx = -h.nx[(size_t)c * nt + t], ny = -h.ny[(size_t)c * nt + t], hl = h.hl[(size_t)c * nt + t];
    const int32_t ea = fill[a]++, eb = fill[b]++;
    wother[ea] = b;
    wother[eb] = a;
    for (int32_t e : {ea, eb}) {
      wgeo[3 * (size_t)e] = nx;
      wgeo[3 * (size_t)e + 1] = ny;
      wgeo[3 * (size_t)e + 2] = hl;
    }
  }

  cudaStream_t st = m->stream;
  CU(cudaStreamSynchronize(st));
  mesh_boundary_free(m);
  int rc = RD_OK;
  if (!ghost_ids.empty()) {
    rc = upload_i32(m->ghost_of, ghost_of, st);
    if (rc == RD_OK) rc = upload_i32(m->ghost_ids, ghost_ids, st);
  }
  if (rc == RD_OK && n_wall > 0) {
    rc = upload_i32(m->wptr, wptr, st);
    if (rc == RD_OK) rc = upload_i32(m->wother, wother, st);
  }
  if (rc != RD_OK) {
    mesh_boundary_free(m);
    m->bc_version++;
    return rc;
  }
  m->n_ghost = (int32_t)ghost_ids.size();
  m->n_wall = n_wall;
  m->wall_alpha = alpha;
  m->wgeo_host.swap(wgeo);
  m->bc_version++;
  return RD_OK;
}
