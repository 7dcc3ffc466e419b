// rd_meshgen.cu -- GPU Delaunay refinement of a periodic rectangle (Sec. 2.3,
// 2.4 and 4.1): starting from a coarse jittered grid, every round tests all
// triangles against the size and quality bounds, locates the circumcentres of
// the bad ones, selects an independent set of insertions by locking their
// cavities with random priorities (atomicMax), splits the containing triangles
// and restores the Delaunay property by rounds of parallel edge flips.  One
// thread per element; compactions are deterministic scans, so a run is
// reproducible.  All loops are bounded; a bound that is reached is reported
// as RD_ETIMEOUT rather than waited out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rd_device.h"
#include "rd_meshgen.cuh"

using namespace rd;
using namespace rd::mg;

struct rd_meshgen {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  rd_meshgen_params p{};
  int64_t Px = 0, Py = 0;
  double unit = 0.0;  // length of one grid unit
  int32_t cap_v = 0, cap_t = 0, nv = 0, nt = 0;
  int32_t rounds = 0, flips = 0, deferred = 0;
  DevBuf vx, vy, tv, ts, tn, tc, dirty;  // mesh
  DevBuf flag, offs, ctri, cedge, cpt, lock, win, part, total, nflips;
  double ms[5] = {0, 0, 0, 0, 0};        // quality+locate, cavities, insertion, flips, total
  Mesh dev() const {
    Mesh m;
    m.vx = (int32_t*)vx.p;
    m.vy = (int32_t*)vy.p;
    m.tv = (int32_t*)tv.p;
    m.ts = (int8_t*)ts.p;
    m.tn = (int32_t*)tn.p;
    m.tc = (int8_t*)tc.p;
    m.dirty = (uint8_t*)dirty.p;
    m.Px = Px;
    m.Py = Py;
    return m;
  }
};

namespace {

constexpr int BLK = 256;

// ---------------------------------------------------------------------------
// deterministic exclusive scan of n int32 flags (0/1) -> offsets, total
// ---------------------------------------------------------------------------
__global__ void k_scan_blocks(int n, const int* __restrict__ flag, int* __restrict__ offs, int* __restrict__ part) {
  __shared__ int s[BLK];
  const int i = blockIdx.x * BLK + threadIdx.x;
  const int v = i < n ? flag[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < BLK; o <<= 1) {
    const int add = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += add;
    __syncthreads();
  }
  if (i < n) offs[i] = s[threadIdx.x] - v;
  if (threadIdx.x == BLK - 1) part[blockIdx.x] = s[BLK - 1];
}
// single block: exclusive scan of the block sums (any count, in chunks of BLK)
__global__ void k_scan_parts(int nb, int* __restrict__ part, int* __restrict__ total) {
  __shared__ int s[BLK];
  int carry = 0;
  for (int base = 0; base < nb; base += BLK) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? part[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < BLK; o <<= 1) {
      const int add = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < nb) part[i] = carry + s[threadIdx.x] - v;
    const int blocksum = s[BLK - 1];
    __syncthreads();
    carry += blocksum;
  }
  if (threadIdx.x == 0) *total = carry;
}
__global__ void k_scan_add(int n, int* __restrict__ offs, const int* __restrict__ part) {
  const int i = blockIdx.x * BLK + threadIdx.x;
  if (i < n) offs[i] += part[blockIdx.x];
}

int scan(rd_meshgen* g, int n, int* total_host) {
  if (n <= 0) {
    *total_host = 0;
    return RD_OK;
  }
  const int nb = (n + BLK - 1) / BLK;
  cudaStream_t st = g->stream;
  k_scan_blocks<<<nb, BLK, 0, st>>>(n, (const int*)g->flag.p, (int*)g->offs.p, (int*)g->part.p);
  k_scan_parts<<<1, BLK, 0, st>>>(nb, (int*)g->part.p, (int*)g->total.p);
  k_scan_add<<<nb, BLK, 0, st>>>(n, (int*)g->offs.p, (const int*)g->part.p);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(total_host, g->total.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return RD_OK;
}

// ---------------------------------------------------------------------------
// refinement kernels
// ---------------------------------------------------------------------------
__global__ void k_quality(Mesh m, int nt, double R_units, double B, int* __restrict__ flag, P64* __restrict__ centre) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  P64 c;
  const bool bad = quality_test(m, t, R_units, B, c);
  flag[t] = bad ? 1 : 0;
  if (bad) centre[t] = c;
}

// compacted candidates: the circumcentre of the i-th bad triangle, located
// (containing triangle ctri[i], edge cedge[i] if on one, point cpt[i] in its frame)
__global__ void k_locate(Mesh m, int nt, const int* __restrict__ flag, const int* __restrict__ offs,
                         const P64* __restrict__ centre, int* __restrict__ ctri, int* __restrict__ cedge,
                         P64* __restrict__ cpt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt || !flag[t]) return;
  const int i = offs[t];
  P64 p = centre[t];
  int edge = -1;
  ctri[i] = locate(m, t, p, edge);
  cedge[i] = edge;
  cpt[i] = p;
}

__global__ void k_cavity_lock(Mesh m, int nc, const int* __restrict__ ctri, const int* __restrict__ cedge,
                              const P64* __restrict__ cpt, unsigned long long* __restrict__ lock, uint64_t seed,
                              uint32_t round) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc || ctri[i] < 0) return;
  int32_t list[MAX_CAVITY];
  const int n = cavity(m, ctri[i], cpt[i], cedge[i], list);
  if (n < 0) return;
  const unsigned long long pr = priority(seed, round, (uint32_t)i);
  for (int q = 0; q < n; ++q) atomicMax(lock + list[q], pr);
}

__global__ void k_cavity_win(Mesh m, int nc, const int* __restrict__ ctri, const int* __restrict__ cedge,
                             const P64* __restrict__ cpt, const unsigned long long* __restrict__ lock, uint64_t seed,
                             uint32_t round, int* __restrict__ win) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  int w = 0;
  if (ctri[i] >= 0) {
    int32_t list[MAX_CAVITY];
    const int n = cavity(m, ctri[i], cpt[i], cedge[i], list);
    if (n > 0) {
      const unsigned long long pr = priority(seed, round, (uint32_t)i);
      w = 1;
      for (int q = 0; q < n; ++q) w &= (lock[list[q]] == pr) ? 1 : 0;
    }
  }
  win[i] = w;
}

__global__ void k_insert(Mesh m, int nc, const int* __restrict__ win, const int* __restrict__ rank,
                         const int* __restrict__ ctri, const int* __restrict__ cedge, const P64* __restrict__ cpt,
                         int nv0, int nt0, int n_ins) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc || !win[i]) return;
  const int r = rank[i];
  if (r >= n_ins) return;  // beyond capacity this round
  if (cedge[i] >= 0)       // on an edge: split the two triangles that share it
    split4(m, ctri[i], cedge[i], nv0 + r, cpt[i], nt0 + 2 * r, nt0 + 2 * r + 1);
  else
    split3(m, ctri[i], nv0 + r, cpt[i], nt0 + 2 * r, nt0 + 2 * r + 1);
}

// ---------------------------------------------------------------------------
// Delaunay restoration by parallel flips (Sec. 2.4.6, Sec. 4.1.4)
// ---------------------------------------------------------------------------
// flag[t] = 1 + k for the first edge of a rewritten triangle t that is not
// locally Delaunay, 0 if none; t stays marked while it has such an edge
__global__ void k_edge_check(Mesh m, int nt, int* __restrict__ flag) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int f = 0;
  if (m.dirty[t]) {
    for (int k = 0; k < 3 && !f; ++k)
      if (edge_bad(m, t, k)) f = 1 + k;
    m.dirty[t] = f ? 1 : 0;
  }
  flag[t] = f;
}

// the six triangles a flip touches: t, n and the four outer neighbours
MG_HD int flip_set(const Mesh& m, int32_t t, int k, int32_t* s) {
  const int32_t n = m.tn[3 * (size_t)t + k];
  const int j = m.tc[3 * (size_t)t + k];
  s[0] = t;
  s[1] = n;
  s[2] = m.tn[3 * (size_t)t + (k + 1) % 3];
  s[3] = m.tn[3 * (size_t)t + (k + 2) % 3];
  s[4] = m.tn[3 * (size_t)n + (j + 1) % 3];
  s[5] = m.tn[3 * (size_t)n + (j + 2) % 3];
  return 6;
}

__global__ void k_flip_lock(Mesh m, int nt, const int* __restrict__ flag, unsigned long long* __restrict__ lock,
                            uint64_t seed, uint32_t round) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt || !flag[t]) return;
  int32_t s[6];
  flip_set(m, t, flag[t] - 1, s);
  const unsigned long long pr = priority(seed ^ 0x5bd1e995ull, round, (uint32_t)t);
  for (int q = 0; q < 6; ++q) atomicMax(lock + s[q], pr);
}

__global__ void k_flip_win(Mesh m, int nt, const int* __restrict__ flag, const unsigned long long* __restrict__ lock,
                           uint64_t seed, uint32_t round, int* __restrict__ win) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int w = 0;
  if (flag[t]) {
    int32_t s[6];
    flip_set(m, t, flag[t] - 1, s);
    const unsigned long long pr = priority(seed ^ 0x5bd1e995ull, round, (uint32_t)t);
    bool distinct = true;  // a flip needs six distinct triangles
    for (int a = 0; a < 6; ++a)
      for (int b = a + 1; b < 6; ++b) distinct = distinct && s[a] != s[b];
    w = distinct ? 1 : 0;
    for (int q = 0; q < 6; ++q) w &= (lock[s[q]] == pr) ? 1 : 0;
  }
  win[t] = w;
}

__global__ void k_flip(Mesh m, int nt, const int* __restrict__ flag, const int* __restrict__ win,
                       unsigned long long* __restrict__ nflips) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt || !win[t]) return;
  flip(m, t, flag[t] - 1);
  atomicAdd(nflips, 1ull);
}

inline unsigned nb(int n) { return (unsigned)((n + BLK - 1) / BLK); }

// Flip until every edge is locally Delaunay (at most max_rounds rounds).
int restore_delaunay(rd_meshgen* g, uint32_t& round_id, int max_rounds) {
  cudaStream_t st = g->stream;
  Mesh m = g->dev();
  for (int r = 0; r < max_rounds; ++r) {
    const int nt = g->nt;
    k_edge_check<<<nb(nt), BLK, 0, st>>>(m, nt, (int*)g->flag.p);
    int nbad = 0;  // sum of the flags: nonzero iff a rewritten triangle has a non-Delaunay edge
    CK(scan(g, nt, &nbad));
    if (nbad == 0) return RD_OK;
    CU(cudaMemsetAsync(g->lock.p, 0, (size_t)nt * sizeof(unsigned long long), st));
    k_flip_lock<<<nb(nt), BLK, 0, st>>>(m, nt, (const int*)g->flag.p, (unsigned long long*)g->lock.p, g->p.seed,
                                        round_id);
    k_flip_win<<<nb(nt), BLK, 0, st>>>(m, nt, (const int*)g->flag.p, (const unsigned long long*)g->lock.p, g->p.seed,
                                       round_id, (int*)g->win.p);
    k_flip<<<nb(nt), BLK, 0, st>>>(m, nt, (const int*)g->flag.p, (const int*)g->win.p,
                                   (unsigned long long*)g->nflips.p);
    CU(cudaGetLastError());
    ++round_id;
  }
  return RD_ETIMEOUT;
}

// Coarse periodic grid with jittered vertices, split along a-c (host).
void initial_mesh(const rd_meshgen_params& p, int64_t Px, int64_t Py, std::vector<int32_t>& vx,
                  std::vector<int32_t>& vy, std::vector<int32_t>& tv, std::vector<int8_t>& ts,
                  std::vector<int32_t>& tn, std::vector<int8_t>& tc) {
  const int Nx = p.nx0, Ny = p.ny0;
  const int nv = Nx * Ny, nt = 2 * nv;
  vx.resize(nv);
  vy.resize(nv);
  for (int j = 0; j < Ny; ++j)
    for (int i = 0; i < Nx; ++i) {
      const int v = j * Nx + i;
      uint64_t h = priority(p.seed, 0xFFFFFFFFu, (uint32_t)v);
      const double jx = ((double)(h >> 40) / 16777216.0 - 0.5) * 0.3, jy = ((double)((h >> 16) & 0xFFFFFF) / 16777216.0 - 0.5) * 0.3;
      int64_t x = (int64_t)std::llround((i + 0.5 + jx) * (double)Px / Nx);
      int64_t y = (int64_t)std::llround((j + 0.5 + jy) * (double)Py / Ny);
      vx[v] = (int32_t)(((x % Px) + Px) % Px);
      vy[v] = (int32_t)(((y % Py) + Py) % Py);
    }
  tv.resize(3 * (size_t)nt);
  ts.resize(6 * (size_t)nt);
  tn.resize(3 * (size_t)nt);
  tc.resize(3 * (size_t)nt);
  auto T1 = [&](int i, int j) { return 2 * (((j + Ny) % Ny) * Nx + ((i + Nx) % Nx)); };
  auto T2 = [&](int i, int j) { return T1(i, j) + 1; };
  for (int j = 0; j < Ny; ++j)
    for (int i = 0; i < Nx; ++i) {
      const int ip = (i + 1) % Nx, jp = (j + 1) % Ny;
      const int a = j * Nx + i, b = j * Nx + ip, c = jp * Nx + ip, d = jp * Nx + i;
      const int8_t sx = (int8_t)(i + 1 == Nx), sy = (int8_t)(j + 1 == Ny);
      const int t1 = T1(i, j), t2 = T2(i, j);
      const int32_t v1[3] = {a, b, c}, v2[3] = {a, c, d};
      const int8_t s1[6] = {0, 0, sx, 0, sx, sy}, s2[6] = {0, 0, sx, sy, 0, sy};
      // t1 = (a, b, c): opp a -> t2(i+1, j) corner 1; opp b -> t2(i, j) corner 2; opp c -> t2(i, j-1) corner 0
      const int32_t n1[3] = {T2(i + 1, j), t2, T2(i, j - 1)};
      const int8_t c1[3] = {1, 2, 0};
      // t2 = (a, c, d): opp a -> t1(i, j+1) corner 2; opp c -> t1(i-1, j) corner 0; opp d -> t1(i, j) corner 1
      const int32_t n2[3] = {T1(i, j + 1), T1(i - 1, j), t1};
      const int8_t c2[3] = {2, 0, 1};
      for (int k = 0; k < 3; ++k) {
        tv[3 * (size_t)t1 + k] = v1[k];
        tv[3 * (size_t)t2 + k] = v2[k];
        tn[3 * (size_t)t1 + k] = n1[k];
        tn[3 * (size_t)t2 + k] = n2[k];
        tc[3 * (size_t)t1 + k] = c1[k];
        tc[3 * (size_t)t2 + k] = c2[k];
      }
      for (int q = 0; q < 6; ++q) {
        ts[6 * (size_t)t1 + q] = s1[q];
        ts[6 * (size_t)t2 + q] = s2[q];
      }
    }
}

template <class V>
int upload(DevBuf& b, const std::vector<V>& v, size_t cap, cudaStream_t st) {
  CK(dev_alloc(b, cap * sizeof(V), st));
  CU(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, st));
  return RD_OK;
}

int run(rd_meshgen* g) {
  cudaStream_t st = g->stream;
  const rd_meshgen_params& p = g->p;
  std::vector<int32_t> vx, vy, tv, tn;
  std::vector<int8_t> ts, tc;
  initial_mesh(p, g->Px, g->Py, vx, vy, tv, ts, tn, tc);
  g->nv = (int32_t)vx.size();
  g->nt = (int32_t)(tv.size() / 3);
  const size_t cv = g->cap_v, ct = g->cap_t;
  CK(upload(g->vx, vx, cv, st));
  CK(upload(g->vy, vy, cv, st));
  CK(upload(g->tv, tv, 3 * ct, st));
  CK(upload(g->ts, ts, 6 * ct, st));
  CK(upload(g->tn, tn, 3 * ct, st));
  CK(upload(g->tc, tc, 3 * ct, st));
  CK(dev_alloc(g->dirty, ct, st));
  CU(cudaMemsetAsync(g->dirty.p, 1, ct, st));  // every initial triangle is checked
  CK(dev_alloc(g->nflips, sizeof(unsigned long long), st));
  CU(cudaMemsetAsync(g->nflips.p, 0, sizeof(unsigned long long), st));
  CK(dev_alloc(g->flag, ct * sizeof(int), st));
  CK(dev_alloc(g->offs, ct * sizeof(int), st));
  CK(dev_alloc(g->win, ct * sizeof(int), st));
  CK(dev_alloc(g->ctri, ct * sizeof(int), st));
  CK(dev_alloc(g->cedge, ct * sizeof(int), st));
  CK(dev_alloc(g->cpt, ct * sizeof(P64), st));
  CK(dev_alloc(g->lock, ct * sizeof(unsigned long long), st));
  CK(dev_alloc(g->part, ((ct + BLK - 1) / BLK + 1) * sizeof(int), st));
  CK(dev_alloc(g->total, sizeof(int), st));
  DevBuf centre;  // circumcentres of the bad triangles, in each triangle's frame
  CK(dev_alloc(centre, ct * sizeof(P64), st));

  cudaEvent_t e[6];
  for (auto& x : e) cudaEventCreate(&x);
  auto elapsed = [&](int a, int b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e[a], e[b]);
    return (double)ms;
  };
  cudaEventRecord(e[5], st);
  uint32_t flip_round = 1;
  int rc = restore_delaunay(g, flip_round, p.max_flip_rounds);
  const double R_units = p.max_circumradius / g->unit;
  for (int r = 0; rc == RD_OK; ++r) {
    Mesh m = g->dev();
    const int nt = g->nt;
    cudaEventRecord(e[0], st);
    k_quality<<<nb(nt), BLK, 0, st>>>(m, nt, R_units, p.quality, (int*)g->flag.p, (P64*)centre.p);
    int nc = 0;
    rc = scan(g, nt, &nc);
    if (rc != RD_OK || nc == 0) break;        // every triangle meets both bounds
    if (r == p.max_rounds) {
      rc = RD_ETIMEOUT;
      break;
    }
    k_locate<<<nb(nt), BLK, 0, st>>>(m, nt, (const int*)g->flag.p, (const int*)g->offs.p, (const P64*)centre.p,
                                     (int*)g->ctri.p, (int*)g->cedge.p, (P64*)g->cpt.p);
    cudaEventRecord(e[1], st);
    CU(cudaMemsetAsync(g->lock.p, 0, (size_t)nt * sizeof(unsigned long long), st));
    k_cavity_lock<<<nb(nc), BLK, 0, st>>>(m, nc, (const int*)g->ctri.p, (const int*)g->cedge.p,
                                          (const P64*)g->cpt.p, (unsigned long long*)g->lock.p, p.seed, (uint32_t)r);
    k_cavity_win<<<nb(nc), BLK, 0, st>>>(m, nc, (const int*)g->ctri.p, (const int*)g->cedge.p,
                                         (const P64*)g->cpt.p, (const unsigned long long*)g->lock.p, p.seed,
                                         (uint32_t)r, (int*)g->win.p);
    CU(cudaGetLastError());
    std::swap(g->flag, g->win);  // scan the winners: offs = rank of each winner
    int nwin = 0;
    rc = scan(g, nc, &nwin);
    std::swap(g->flag, g->win);
    if (rc != RD_OK) break;
    cudaEventRecord(e[2], st);
    // capacity: every insertion adds one vertex and two triangles
    int n_ins = nwin;
    n_ins = std::min(n_ins, g->cap_v - g->nv);
    n_ins = std::min(n_ins, (g->cap_t - g->nt) / 2);
    g->deferred += nc - n_ins;
    if (n_ins <= 0) {
      rc = nwin > 0 ? RD_ENOMEM : RD_ETIMEOUT;  // full, or no candidate could be inserted
      break;
    }
    k_insert<<<nb(nc), BLK, 0, st>>>(m, nc, (const int*)g->win.p, (const int*)g->offs.p, (const int*)g->ctri.p,
                                     (const int*)g->cedge.p, (const P64*)g->cpt.p, g->nv, g->nt, n_ins);
    CU(cudaGetLastError());
    g->nv += n_ins;
    g->nt += 2 * n_ins;
    cudaEventRecord(e[3], st);
    rc = restore_delaunay(g, flip_round, p.max_flip_rounds);
    cudaEventRecord(e[4], st);
    CU(cudaStreamSynchronize(st));
    g->ms[0] += elapsed(0, 1);
    g->ms[1] += elapsed(1, 2);
    g->ms[2] += elapsed(2, 3);
    g->ms[3] += elapsed(3, 4);
    g->rounds = r + 1;
  }
  cudaEventRecord(e[4], st);
  cudaEventSynchronize(e[4]);
  g->ms[4] = elapsed(5, 4);
  unsigned long long nfl = 0;
  if (cudaMemcpy(&nfl, g->nflips.p, sizeof(nfl), cudaMemcpyDeviceToHost) == cudaSuccess) g->flips = (int32_t)nfl;
  for (auto& x : e) cudaEventDestroy(x);
  dev_free(centre);
  return rc;
}

}  // namespace

extern "C" int rd_meshgen_run(const rd_meshgen_params* p, void* cuda_stream, rd_meshgen** out) {
  if (!p || !out) return RD_EINVAL;
  *out = nullptr;
  if (!(p->Lx > 0) || !(p->Ly > 0) || p->nx0 < 3 || p->ny0 < 3 || !(p->quality >= 1.0) ||
      !(p->max_circumradius > 0) || p->max_vertices < p->nx0 * p->ny0 || p->max_rounds < 1 ||
      p->max_flip_rounds < 1)
    return RD_EINVAL;
  if ((int64_t)p->max_vertices * 2 >= (int64_t)INT32_MAX / 3) return RD_EINVAL;
  rd_meshgen* g = new (std::nothrow) rd_meshgen();
  if (!g) return RD_ENOMEM;
  g->p = *p;
  g->Px = (int64_t)1 << UNIT_BITS;
  g->unit = p->Lx / (double)g->Px;
  g->Py = (int64_t)std::llround(p->Ly / g->unit);
  if (g->Py < 3 || g->Py > ((int64_t)1 << 31) - 1) {
    delete g;
    return RD_EINVAL;
  }
  g->cap_v = p->max_vertices;
  g->cap_t = 2 * p->max_vertices;
  if (cuda_stream) {
    g->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete g;
      return RD_ECUDA;
    }
    g->own_stream = true;
  }
  *out = g;
  return run(g);
}

extern "C" int rd_meshgen_sizes(const rd_meshgen* g, int32_t* n_vertex, int32_t* n_tri, int32_t* rounds,
                                int32_t* flips) {
  if (!g) return RD_EINVAL;
  if (n_vertex) *n_vertex = g->nv;
  if (n_tri) *n_tri = g->nt;
  if (rounds) *rounds = g->rounds;
  if (flips) *flips = g->flips;
  return RD_OK;
}

extern "C" int rd_meshgen_times(const rd_meshgen* g, double ms[5]) {
  if (!g || !ms) return RD_EINVAL;
  for (int k = 0; k < 5; ++k) ms[k] = g->ms[k];
  return RD_OK;
}

extern "C" int rd_meshgen_get(const rd_meshgen* g, double* xy, int32_t* tri, int8_t* shift, int64_t* xy_units) {
  if (!g) return RD_EINVAL;
  cudaStream_t st = g->stream;
  const size_t nv = g->nv, nt = g->nt;
  std::vector<int32_t> vx(nv), vy(nv), tv(3 * nt);
  std::vector<int8_t> ts(6 * nt);
  CU(cudaMemcpyAsync(vx.data(), g->vx.p, nv * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(vy.data(), g->vy.p, nv * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(tv.data(), g->tv.p, 3 * nt * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(ts.data(), g->ts.p, 6 * nt * sizeof(int8_t), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  for (size_t i = 0; i < nv; ++i) {
    if (xy) {
      xy[2 * i] = vx[i] * g->unit;
      xy[2 * i + 1] = vy[i] * g->unit;
    }
    if (xy_units) {
      xy_units[2 * i] = vx[i];
      xy_units[2 * i + 1] = vy[i];
    }
  }
  if (tri) std::memcpy(tri, tv.data(), tv.size() * sizeof(int32_t));
  if (shift) std::memcpy(shift, ts.data(), ts.size());
  return RD_OK;
}

extern "C" int rd_meshgen_domain(const rd_meshgen* g, double* Lx, double* Ly, int64_t* Px, int64_t* Py) {
  if (!g) return RD_EINVAL;
  if (Lx) *Lx = g->Px * g->unit;
  if (Ly) *Ly = g->Py * g->unit;
  if (Px) *Px = g->Px;
  if (Py) *Py = g->Py;
  return RD_OK;
}

extern "C" void rd_meshgen_destroy(rd_meshgen* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  DevBuf* bufs[] = {&g->vx, &g->vy, &g->tv, &g->ts, &g->tn, &g->tc, &g->dirty, &g->flag, &g->offs,
                    &g->ctri, &g->cedge, &g->cpt, &g->lock, &g->win, &g->part, &g->total, &g->nflips};
  for (DevBuf* b : bufs) dev_free(*b);
  if (g->own_stream) cudaStreamDestroy(g->stream);
  delete g;
}
