// rd_tiled.cu -- tiled form of the two-stage step: the corner shares stay on chip.
//
// The step of rd_kernels.cuh writes every triangle's twelve share words to
// global memory and gathers them back per vertex through the CSR.  Here the
// triangles, sorted by their smallest vertex id (the mesh store's order), are
// cut into tiles of tt consecutive triangles and one block processes a tile:
//
//   k_tile_stage1  stage 1 (Sec. 3.3) of the tile's triangles with the vertex
//                  states staged in shared memory; shares and CFL terms stay in
//                  shared memory; each interior vertex of the tile sums its
//                  corners in CSR order -> R1 and 2 V_i / sigma_i (block min)
//   k_tile_bnd1    boundary vertices: the same sums from the few corner shares
//                  that went to global memory; last block -> dt
//   k_tile_stage2  stages W* = W^n - dt/V R1 and Z(W*) for the tile's vertices
//                  (Eq. eqRK1), stage 2 (Sec. 3.4) of its triangles, and the
//                  final update W^{n+1} = W* - dt/V R2 (Eq. eqRK2) of its
//                  interior vertices
//   k_tile_bnd2    the same final update for the boundary vertices
//
// A vertex is interior to the tile owning it when all its triangles lie in
// that tile.  Every share, sum and update is computed by the same code and
// summed in the same CSR order as in the per-triangle form, so the two forms
// give bitwise identical states.  Walls, ghost vertices and the Bx sensor's
// range of |v| at W* keep the per-triangle stage 2.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "rd_device.h"
#include "rd_internal.h"
#include "rd_kernels.cuh"
#include "rd_tiled.h"

namespace rd {

namespace {

constexpr int TILE_MAX_THREADS = 256;
constexpr int TILE_BND_BLOCK = 256;

// Device view of a tile plan.
struct TileView {
  int nt, tt, n_tiles, n_bvert, slots;
  const int* vs;
  const int* hptr;
  const int* hlist;
  const uint16_t* lslot;
  const uint8_t* bmask;
  const int* bvert;
  const int* ptr;
  const int* ent;
};

// Shared-memory layout (bytes): shares [tt][12], CFL terms [tt] (stage 1),
// then per slot the staged vertex records.
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
template <class T>
__host__ __device__ inline size_t cfl_off(int tt) { return (size_t)12 * tt * sizeof(T); }
template <class T>
__host__ __device__ inline size_t slot_off(int tt) { return cfl_off<T>(tt) + (((size_t)tt * sizeof(T) + 15) & ~(size_t)15); }
template <class T>
size_t smem_stage1(int tt, int slots) { return slot_off<T>(tt) + align16((size_t)4 * slots * sizeof(T)) + align16((size_t)slots * sizeof(T)); }
template <class T>
size_t smem_stage2(int tt, int slots) { return cfl_off<T>(tt) + 3 * align16((size_t)4 * slots * sizeof(T)); }
template <class T>
__host__ __device__ inline size_t smem_stage1_base(int tt, int slots) {
  return slot_off<T>(tt) + align16((size_t)4 * slots * sizeof(T)) + align16((size_t)slots * sizeof(T));
}
template <class T>
__host__ __device__ inline size_t smem_stage2_base(int tt, int slots) {
  return cfl_off<T>(tt) + 3 * align16((size_t)4 * slots * sizeof(T));
}
// Geometry block of a tile staged in shared memory (plans with RD_TILE_STAGE_GEOMETRY):
// nx, ny, hl [3][tt], area [tt], l_max [tt] in T, corner slots [3][tt] uint16,
// boundary masks [tt] uint8.
template <class T>
__host__ __device__ inline size_t geo_bytes(int tt) {
  return (((size_t)11 * tt * sizeof(T) + 15) & ~(size_t)15) + (((size_t)6 * tt + 15) & ~(size_t)15) +
         (((size_t)tt + 15) & ~(size_t)15);
}

// Shared-memory view of a tile's staged geometry.
template <class T>
struct TileGeo {
  T* g;          // [11][tt]: nx0..2, ny0..2, hl0..2, area, l_max
  uint16_t* sl;  // [3][tt]
  uint8_t* bm;   // [tt]
  __device__ static TileGeo at(unsigned char* base, int tt) {
    TileGeo q;
    q.g = reinterpret_cast<T*>(base);
    q.sl = reinterpret_cast<uint16_t*>(base + (((size_t)11 * tt * sizeof(T) + 15) & ~(size_t)15));
    q.bm = reinterpret_cast<uint8_t*>(reinterpret_cast<unsigned char*>(q.sl) + (((size_t)6 * tt + 15) & ~(size_t)15));
    return q;
  }
};

// Copy the geometry of triangles [t0, t0 + n) of a tile into shared memory
// (every thread of the block; coalesced loads, many in flight per thread).
template <class T>
__device__ __forceinline__ void stage_geometry(const TileView& P, const DevGeo<T>& g, int t0, int n, int tt,
                                               TileGeo<T> q) {
  const int nt = P.nt;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int t = t0 + j;
    T v[11];
    uint16_t sl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[c] = __ldg(g.nx + (size_t)c * nt + t);
      v[3 + c] = __ldg(g.ny + (size_t)c * nt + t);
      v[6 + c] = __ldg(g.hl + (size_t)c * nt + t);
      sl[c] = __ldg(P.lslot + (size_t)c * nt + t);
    }
    v[9] = __ldg(g.area + t);
    v[10] = __ldg(g.lmax + t);
    const uint8_t bm = __ldg(P.bmask + t);
#pragma unroll
    for (int k = 0; k < 11; ++k) q.g[k * tt + j] = v[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) q.sl[c * tt + j] = sl[c];
    q.bm[j] = bm;
  }
}

__device__ __forceinline__ void sld4(const float* p, float o[4]) {
  float4 a = *reinterpret_cast<const float4*>(p);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void sld4(const double* p, double o[4]) {
  double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// One flag per block: the control block's stop word read once by thread 0, so
// that every thread of the block takes the same branch around the barriers.
__device__ __forceinline__ bool block_stopped(const DevCtl* ctl) {
  __shared__ int stop;
  if (threadIdx.x == 0) stop = ctl->stop;
  __syncthreads();
  return stop != 0;
}

template <class T>
__device__ __forceinline__ void tile_geo_of(const TileGeo<T>& q, int lt, int tt, int sl[3], T nx[3], T ny[3],
                                            T hl[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    sl[c] = q.sl[c * tt + lt];
    nx[c] = q.g[c * tt + lt];
    ny[c] = q.g[(3 + c) * tt + lt];
    hl[c] = q.g[(6 + c) * tt + lt];
  }
}

template <class T>
__device__ __forceinline__ void load_geo(int t, int nt, const DevGeo<T>& g, const uint16_t* __restrict__ lslot,
                                         int sl[3], T nx[3], T ny[3], T hl[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    sl[c] = __ldg(lslot + (size_t)c * nt + t);
    nx[c] = __ldg(g.nx + (size_t)c * nt + t);
    ny[c] = __ldg(g.ny + (size_t)c * nt + t);
    hl[c] = __ldg(g.hl + (size_t)c * nt + t);
  }
}

template <class T, int SCHEME, bool GS>
__global__ void __launch_bounds__(TILE_MAX_THREADS, (TriOcc<T, 1>::value))
    k_tile_stage1(TileView P, DevGeo<T> g, const T* __restrict__ Z, const T* __restrict__ spd, Gas<T> gas, T eps,
                  T* __restrict__ share, T* __restrict__ rec, T* __restrict__ cfl, const T* __restrict__ V,
                  T* __restrict__ R1, T* __restrict__ partial, DevCtl* ctl, BlendArgs<T> ba) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (block_stopped(ctl)) return;
  const int p = blockIdx.x, nt = P.nt, t0 = p * P.tt, n = min(P.tt, nt - t0);
  const int v0 = __ldg(P.vs + p), nown = __ldg(P.vs + p + 1) - v0;
  const int h0 = __ldg(P.hptr + p), nsl = nown + __ldg(P.hptr + p + 1) - h0;
  T* sh = reinterpret_cast<T*>(smem);
  T* scf = reinterpret_cast<T*>(smem + cfl_off<T>(P.tt));
  T* sZ = reinterpret_cast<T*>(smem + slot_off<T>(P.tt));
  T* sS = sZ + 4 * (size_t)P.slots;
  const TileGeo<T> sg = TileGeo<T>::at(smem + smem_stage1_base<T>(P.tt, P.slots), P.tt);
  if (GS) stage_geometry(P, g, t0, n, P.tt, sg);
  for (int s = threadIdx.x; s < nsl; s += blockDim.x) {
    const int v = s < nown ? v0 + s : __ldg(P.hlist + h0 + s - nown);
    T z[4];
    load_vec4(Z, v, z);
    st4(sZ + 4 * s, z);
    sS[s] = __ldg(spd + v);
  }
  __syncthreads();
  const int mode = SCHEME == RD_BMAX2 ? ba.mode : BLEND_B;
  for (int lt = threadIdx.x; lt < n; lt += blockDim.x) {
    const int t = t0 + lt;
    int sl[3];
    T nx[3], ny[3], hl[3], Zc[3][4];
    if (GS)
      tile_geo_of(sg, lt, P.tt, sl, nx, ny, hl);
    else
      load_geo(t, nt, g, P.lslot, sl, nx, ny, hl);
#pragma unroll
    for (int c = 0; c < 3; ++c) sld4(sZ + 4 * sl[c], Zc[c]);
    T lam;
    {
      const T s0 = sS[sl[0]], s1 = sS[sl[1]], s2 = sS[sl[2]];
      lam = mag_less(s1, s0) ? s0 : s1;  // speeds are >= 0
      lam = mag_less(s2, lam) ? lam : s2;
    }
    const T cf = (GS ? sg.g[10 * P.tt + lt] : __ldg(g.lmax + t)) * lam;
    T out[3][4], r[16];
    T thx = T(0);
    if (SCHEME == RD_BMAX2 && mode == BLEND_X)
      thx = bx_theta(Zc, nx, ny, hl, GS ? sg.g[9 * P.tt + lt] : __ldg(g.area + t), ba.L, vrange_of<T>(ba.vr));
    const int st = stage1_body<T, SCHEME>(Zc, nx, ny, hl, gas, eps, out, r, mode, thx);
    if (st) {
      atomicOr(&ctl->status, st);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) out[i][k] = T(0);
    } else if (SCHEME != RD_N1) {
      T* rp = rec + (size_t)t * 16;
#pragma unroll
      for (int k = 0; k < 4; ++k) st4(rp + 4 * k, r + 4 * k);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) st4(sh + 12 * lt + 4 * i, out[i]);
    scf[lt] = cf;
    const unsigned bm = GS ? (unsigned)sg.bm[lt] : (unsigned)__ldg(P.bmask + t);
    if (bm) {
      cfl[t] = cf;
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if ((bm >> i) & 1u) st4(share + (size_t)t * 12 + 4 * i, out[i]);
    }
  }
  __syncthreads();
  // interior vertices: corner sums in CSR order from shared memory
  T ratio = T(INFINITY);
  const int base = 3 * t0;
  for (int li = threadIdx.x; li < nown; li += blockDim.x) {
    const int i = v0 + li;
    const int e0 = __ldg(P.ptr + i), e1 = __ldg(P.ptr + i + 1);
    if (__ldg(P.ent + e0) < base) continue;  // boundary vertex
    T r[4] = {T(0), T(0), T(0), T(0)};
    T sig = T(0);
    for (int e = e0; e < e1; ++e) {
      const int le = __ldg(P.ent + e) - base;
      T q[4];
      sld4(sh + 4 * le, q);
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] += q[k];
      sig += scf[le / 3];
    }
    st4(R1 + 4 * (size_t)i, r);
    const T x = T(2) * __ldg(V + i) / sig;
    ratio = x < ratio ? x : ratio;
  }
  const T m = block_min(ratio);
  if (threadIdx.x == 0) partial[p] = m;
}

template <class T>
__global__ void __launch_bounds__(TILE_BND_BLOCK) k_tile_bnd1(TileView P, const T* __restrict__ share,
                                                             const T* __restrict__ cfl, const T* __restrict__ V,
                                                             T* __restrict__ R1, T* __restrict__ partial, T cflnum,
                                                             DevCtl* ctl) {
  if (block_stopped(ctl)) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  T ratio = T(INFINITY);
  if (j < P.n_bvert) {
    const int i = __ldg(P.bvert + j);
    T r[4] = {T(0), T(0), T(0), T(0)};
    T sig = T(0);
    gather_corners<T, true>(__ldg(P.ptr + i), __ldg(P.ptr + i + 1), P.ent, share, cfl, r, sig);
    st4(R1 + 4 * (size_t)i, r);
    ratio = T(2) * __ldg(V + i) / sig;
  }
  dt_finish(ratio, partial, P.n_tiles + blockIdx.x, P.n_tiles + gridDim.x, cflnum, ctl);
}

template <class T, int SCHEME, bool GS>
__global__ void __launch_bounds__(TILE_MAX_THREADS, (TriOcc<T, 2>::value))
    k_tile_stage2(TileView P, DevGeo<T> g, const T* __restrict__ Wn, const T* __restrict__ R1,
                  const T* __restrict__ V, const T* __restrict__ rec, Gas<T> gas, T gamma, T eps,
                  T* __restrict__ share, T* __restrict__ Wout, T* __restrict__ Zout, T* __restrict__ spdout,
                  DevCtl* ctl, BlendArgs<T> ba) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (block_stopped(ctl)) return;
  const int p = blockIdx.x, nt = P.nt, t0 = p * P.tt, n = min(P.tt, nt - t0);
  const int v0 = __ldg(P.vs + p), nown = __ldg(P.vs + p + 1) - v0;
  const int h0 = __ldg(P.hptr + p), nsl = nown + __ldg(P.hptr + p + 1) - h0;
  const T dt = (T)ctl->dt;
  T* sh = reinterpret_cast<T*>(smem);
  T* sWn = reinterpret_cast<T*>(smem + cfl_off<T>(P.tt));
  T* sWs = sWn + 4 * (size_t)P.slots;
  T* sZs = sWs + 4 * (size_t)P.slots;
  const TileGeo<T> sg = TileGeo<T>::at(smem + smem_stage2_base<T>(P.tt, P.slots), P.tt);
  if (GS) stage_geometry(P, g, t0, n, P.tt, sg);
  // W* = W^n - dt/V R1 and Z(W*) of the tile's owned and halo vertices
  for (int s = threadIdx.x; s < nsl; s += blockDim.x) {
    const int v = s < nown ? v0 + s : __ldg(P.hlist + h0 + s - nown);
    T w[4], r[4], ws[4], z[4], sp;
    load_vec4(Wn, v, w);
    load_vec4(R1, v, r);
    const T f = dt / __ldg(V + v);
#pragma unroll
    for (int k = 0; k < 4; ++k) ws[k] = w[k] - f * r[k];
    if (!vertex_Z(ws, gamma, z, sp)) {
      atomicOr(&ctl->status, ST_NONPHYS_VERTEX);
      ctl->stop = 1;
    }
    st4(sWn + 4 * s, w);
    st4(sWs + 4 * s, ws);
    st4(sZs + 4 * s, z);
  }
  __syncthreads();
  const int mode = SCHEME == RD_BMAX2 ? ba.mode : BLEND_B;
  const int slump = (SCHEME == RD_BMAX2 || SCHEME == RD_LDA2) ? ba.sl : 0;
  for (int lt = threadIdx.x; lt < n; lt += blockDim.x) {
    const int t = t0 + lt;
    int sl[3];
    T nx[3], ny[3], hl[3], Zc[3][4], wn[3][4], ws[3][4], r[16];
    if (GS)
      tile_geo_of(sg, lt, P.tt, sl, nx, ny, hl);
    else
      load_geo(t, nt, g, P.lslot, sl, nx, ny, hl);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sld4(sZs + 4 * sl[c], Zc[c]);
      sld4(sWn + 4 * sl[c], wn[c]);
      sld4(sWs + 4 * sl[c], ws[c]);
    }
    const T* rp = rec + (size_t)t * 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) ld4(rp + 4 * k, r + 4 * k);
    T out[3][4];
    const T area = GS ? sg.g[9 * P.tt + lt] : __ldg(g.area + t);
    const int st = stage2_body<T, SCHEME>(Zc, wn, ws, r, nx, ny, hl, area, dt, gas, eps, out, mode, T(0), slump);
    if (st) {
      atomicOr(&ctl->status, st);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) out[i][k] = T(0);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) st4(sh + 12 * lt + 4 * i, out[i]);
    const unsigned bm = GS ? (unsigned)sg.bm[lt] : (unsigned)__ldg(P.bmask + t);
    if (bm) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if ((bm >> i) & 1u) st4(share + (size_t)t * 12 + 4 * i, out[i]);
    }
  }
  __syncthreads();
  // interior vertices: W^{n+1} = W* - dt/V R2, Z and |v|+c for the next step
  const int base = 3 * t0;
  for (int li = threadIdx.x; li < nown; li += blockDim.x) {
    const int i = v0 + li;
    const int e0 = __ldg(P.ptr + i), e1 = __ldg(P.ptr + i + 1);
    if (__ldg(P.ent + e0) < base) continue;  // boundary vertex
    T r[4] = {T(0), T(0), T(0), T(0)};
    for (int e = e0; e < e1; ++e) {
      T q[4];
      sld4(sh + 4 * (__ldg(P.ent + e) - base), q);
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] += q[k];
    }
    const T f = dt / __ldg(V + i);
    T W[4], Zn[4], sp;
    sld4(sWs + 4 * li, W);
#pragma unroll
    for (int k = 0; k < 4; ++k) W[k] = W[k] - f * r[k];
    const bool ok = vertex_Z(W, gamma, Zn, sp);
    st4(Wout + 4 * (size_t)i, W);
    st4(Zout + 4 * (size_t)i, Zn);
    spdout[i] = sp;
    if (!ok) {
      atomicOr(&ctl->status, ST_NONPHYS_VERTEX);
      ctl->stop = 1;
    }
  }
}

template <class T>
__global__ void __launch_bounds__(TILE_BND_BLOCK) k_tile_bnd2(TileView P, const T* __restrict__ share,
                                                             const T* __restrict__ Wn, const T* __restrict__ R1,
                                                             const T* __restrict__ V, T gamma, T* __restrict__ Wout,
                                                             T* __restrict__ Zout, T* __restrict__ spdout,
                                                             DevCtl* ctl) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.n_bvert || ctl->stop) return;
  const int i = __ldg(P.bvert + j);
  const T dt = (T)ctl->dt;
  const T f = dt / __ldg(V + i);
  T W[4], r[4], Zn[4], sp;
  load_vec4(Wn, i, W);
  load_vec4(R1, i, r);
#pragma unroll
  for (int k = 0; k < 4; ++k) W[k] = W[k] - f * r[k];  // W*, as staged by k_tile_stage2
  r[0] = r[1] = r[2] = r[3] = T(0);
  T unused = T(0);
  gather_corners<T, false>(__ldg(P.ptr + i), __ldg(P.ptr + i + 1), P.ent, share, nullptr, r, unused);
#pragma unroll
  for (int k = 0; k < 4; ++k) W[k] = W[k] - f * r[k];
  const bool ok = vertex_Z(W, gamma, Zn, sp);
  st4(Wout + 4 * (size_t)i, W);
  st4(Zout + 4 * (size_t)i, Zn);
  spdout[i] = sp;
  if (!ok) {
    atomicOr(&ctl->status, ST_NONPHYS_VERTEX);
    ctl->stop = 1;
  }
}

TileView view_of(const rd_state* s) {
  const TilePlan* tp = s->tiles;
  const rd_mesh* m = s->m;
  TileView P;
  P.nt = m->h.nt;
  P.tt = tp->tt;
  P.n_tiles = tp->n_tiles;
  P.n_bvert = tp->n_bvert;
  P.slots = tp->slots;
  P.vs = (const int*)tp->vs.p;
  P.hptr = (const int*)tp->hptr.p;
  P.hlist = (const int*)tp->hlist.p;
  P.lslot = (const uint16_t*)tp->lslot.p;
  P.bmask = (const uint8_t*)tp->bmask.p;
  P.bvert = (const int*)tp->bvert.p;
  P.ptr = (const int*)m->ptr.p;
  P.ent = (const int*)m->ent.p;
  return P;
}

template <class T>
DevGeo<T> geo_view(const rd_mesh* m) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  DevGeo<T> g;
  g.nx = (const T*)m->geo[pi][0].p;
  g.ny = (const T*)m->geo[pi][1].p;
  g.hl = (const T*)m->geo[pi][2].p;
  g.area = (const T*)m->geo[pi][3].p;
  g.lmax = (const T*)m->geo[pi][4].p;
  return g;
}

template <class T, bool GS>
int smem_attrs_gs(size_t b1, size_t b2) {
  CU(cudaFuncSetAttribute(k_tile_stage1<T, RD_N1, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b1));
  CU(cudaFuncSetAttribute(k_tile_stage1<T, RD_LDA2, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b1));
  CU(cudaFuncSetAttribute(k_tile_stage1<T, RD_B2, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b1));
  CU(cudaFuncSetAttribute(k_tile_stage1<T, RD_BMAX2, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b1));
  CU(cudaFuncSetAttribute(k_tile_stage2<T, RD_LDA2, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b2));
  CU(cudaFuncSetAttribute(k_tile_stage2<T, RD_B2, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b2));
  CU(cudaFuncSetAttribute(k_tile_stage2<T, RD_BMAX2, GS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b2));
  return RD_OK;
}

// Opt every instantiation of a precision into the dynamic shared memory it
// needs (above the 48 KB default).  The limits only grow, so that the plans of
// other states stay launchable.
template <class T>
int tile_smem_attrs(size_t b1, size_t b2) {
  static size_t lim1 = 0, lim2 = 0;
  b1 = std::max(b1, lim1);
  b2 = std::max(b2, lim2);
  CK((smem_attrs_gs<T, false>(b1, b2)));
  CK((smem_attrs_gs<T, true>(b1, b2)));
  lim1 = b1;
  lim2 = b2;
  return RD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host: the tile plan of a mesh.
// ---------------------------------------------------------------------------
int build_tile_plan(const HostMesh& h, int tt, TilePlanHost& out) {
  const int32_t nt = h.nt, nv = h.nv;
  if (tt < 32 || tt > MAX_TILE_TRIANGLES || tt % 32) return RD_EINVAL;
  std::vector<int32_t> minv(nt);
  for (int32_t t = 0; t < nt; ++t) {
    int32_t a = h.tri[t], b = h.tri[(size_t)nt + t], c = h.tri[2 * (size_t)nt + t];
    minv[t] = std::min(a, std::min(b, c));
    if (t > 0 && minv[t] < minv[t - 1]) return RD_ENOTSUP;  // triangles not sorted by smallest vertex
  }
  if (minv[0] != 0) return RD_ENOTSUP;
  const int32_t n_tiles = (int32_t)((nt + (int64_t)tt - 1) / tt);
  out = TilePlanHost();
  out.tt = tt;
  out.n_tiles = n_tiles;
  out.vs.resize((size_t)n_tiles + 1);
  for (int32_t p = 0; p < n_tiles; ++p) out.vs[p] = minv[(size_t)p * tt];
  out.vs[n_tiles] = nv;
  // boundary vertices: a triangle before the owning tile's first one
  std::vector<uint8_t> isb(nv, 0);
  for (int32_t p = 0; p < n_tiles; ++p) {
    const int64_t base = 3 * (int64_t)p * tt;
    for (int32_t i = out.vs[p]; i < out.vs[p + 1]; ++i)
      if (h.csr_ent[h.csr_ptr[i]] < base) {
        isb[i] = 1;
        out.bvert.push_back(i);
      }
  }
  out.bmask.resize(nt);
  for (int32_t t = 0; t < nt; ++t)
    out.bmask[t] = (uint8_t)(isb[h.tri[t]] | (isb[h.tri[(size_t)nt + t]] << 1) | (isb[h.tri[2 * (size_t)nt + t]] << 2));
  // halo vertices (corners beyond the tile's vertex range) and corner slots
  out.hptr.assign((size_t)n_tiles + 1, 0);
  out.lslot.resize(3 * (size_t)nt);
  std::vector<int32_t> halo;
  int slots = 0;
  for (int32_t p = 0; p < n_tiles; ++p) {
    const int32_t t0 = p * tt, t1 = std::min(nt, t0 + tt);
    const int32_t v0 = out.vs[p], v1 = out.vs[p + 1];
    halo.clear();
    for (int c = 0; c < 3; ++c)
      for (int32_t t = t0; t < t1; ++t) {
        int32_t v = h.tri[(size_t)c * nt + t];
        if (v >= v1) halo.push_back(v);
      }
    std::sort(halo.begin(), halo.end());
    halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
    const int nown = v1 - v0, nsl = nown + (int)halo.size();
    if (nsl > 65535) return RD_ENOTSUP;
    slots = std::max(slots, nsl);
    for (int c = 0; c < 3; ++c)
      for (int32_t t = t0; t < t1; ++t) {
        int32_t v = h.tri[(size_t)c * nt + t];
        int sl = v < v1 ? v - v0 : nown + (int)(std::lower_bound(halo.begin(), halo.end(), v) - halo.begin());
        out.lslot[(size_t)c * nt + t] = (uint16_t)sl;
      }
    out.hlist.insert(out.hlist.end(), halo.begin(), halo.end());
    out.hptr[p + 1] = (int32_t)out.hlist.size();
  }
  out.slots = slots;
  out.n_bvert = (int32_t)out.bvert.size();
  return RD_OK;
}

void tile_plan_free(TilePlan* tp) {
  if (!tp) return;
  DevBuf* bufs[] = {&tp->vs, &tp->hptr, &tp->hlist, &tp->lslot, &tp->bmask, &tp->bvert, &tp->partial};
  for (DevBuf* b : bufs) dev_free(*b);
  delete tp;
}

size_t tile_smem_bytes(int precision, int stage, int tt, int slots, bool gs) {
  if (precision == RD_FP64)
    return (stage == 1 ? smem_stage1<double>(tt, slots) : smem_stage2<double>(tt, slots)) +
           (gs ? geo_bytes<double>(tt) : 0);
  return (stage == 1 ? smem_stage1<float>(tt, slots) : smem_stage2<float>(tt, slots)) + (gs ? geo_bytes<float>(tt) : 0);
}

bool tiled_stage2_applies(const rd_state* s) {
  return s->p.scheme != RD_N1 && s->p.scheme != RD_BX2 && s->m->n_wall == 0 && s->m->n_ghost == 0;
}

template <class T, bool GS>
void launch_tile_stage1(const rd_params& pr, unsigned grid, int bt, size_t b1, cudaStream_t st, const TileView& P,
                        const DevGeo<T>& g, const T* Za, const T* Sa, const Gas<T>& gas, T eps, T* share, T* rec, T* cf,
                        const T* V, T* R1, T* partial, DevCtl* ctl, const BlendArgs<T>& ba) {
  switch (pr.scheme) {
    case RD_N1:
      k_tile_stage1<T, RD_N1, GS><<<grid, bt, b1, st>>>(P, g, Za, Sa, gas, eps, share, rec, cf, V, R1, partial, ctl,
                                                        ba);
      break;
    case RD_LDA2:
      k_tile_stage1<T, RD_LDA2, GS><<<grid, bt, b1, st>>>(P, g, Za, Sa, gas, eps, share, rec, cf, V, R1, partial, ctl,
                                                          ba);
      break;
    default:
      if (pr.scheme == RD_B2 && pr.lumping == RD_LUMP_GLOBAL)
        k_tile_stage1<T, RD_B2, GS><<<grid, bt, b1, st>>>(P, g, Za, Sa, gas, eps, share, rec, cf, V, R1, partial, ctl,
                                                          ba);
      else
        k_tile_stage1<T, RD_BMAX2, GS><<<grid, bt, b1, st>>>(P, g, Za, Sa, gas, eps, share, rec, cf, V, R1, partial,
                                                             ctl, ba);
      break;
  }
}

template <class T, bool GS>
void launch_tile_stage2(const rd_params& pr, unsigned grid, int bt, size_t b2, cudaStream_t st, const TileView& P,
                        const DevGeo<T>& g, const T* Wa, const T* R1, const T* V, const T* rec, const Gas<T>& gas,
                        T gamma, T eps, T* share, T* Wb, T* Zb, T* Sb, DevCtl* ctl, const BlendArgs<T>& ba) {
  if (pr.scheme == RD_LDA2)
    k_tile_stage2<T, RD_LDA2, GS><<<grid, bt, b2, st>>>(P, g, Wa, R1, V, rec, gas, gamma, eps, share, Wb, Zb, Sb, ctl,
                                                        ba);
  else if (pr.scheme == RD_B2 && pr.lumping == RD_LUMP_GLOBAL)
    k_tile_stage2<T, RD_B2, GS><<<grid, bt, b2, st>>>(P, g, Wa, R1, V, rec, gas, gamma, eps, share, Wb, Zb, Sb, ctl,
                                                      ba);
  else
    k_tile_stage2<T, RD_BMAX2, GS><<<grid, bt, b2, st>>>(P, g, Wa, R1, V, rec, gas, gamma, eps, share, Wb, Zb, Sb, ctl,
                                                         ba);
}

template <class T>
int tiled_stage1(rd_state* s, int a, cudaEvent_t* ev) {
  rd_mesh* m = s->m;
  const TilePlan* tp = s->tiles;
  cudaStream_t st = m->stream;
  const TileView P = view_of(s);
  const DevGeo<T> g = geo_view<T>(m);
  const T* V = (const T*)m->geo[s->pi][5].p;
  const T* Za = (const T*)s->Z[a].p;
  const T* Sa = (const T*)s->spd[a].p;
  T* share = (T*)s->share.p;
  T* rec = (T*)s->rec.p;
  T* cf = (T*)s->cfl.p;
  T* R1 = (T*)s->R1.p;
  T* partial = (T*)tp->partial.p;
  DevCtl* ctl = (DevCtl*)s->ctl.p;
  const Gas<T> gas = Gas<T>::of((T)s->p.gamma);
  const T eps = (T)s->p.eps_fix;
  BlendArgs<T> ba = tile_blend_args<T>(s);
  ba.vr = (unsigned long long*)s->vr.p;  // |v| range of W^n
  const size_t b1 = smem_stage1<T>(tp->tt, tp->slots) + (tp->gs ? geo_bytes<T>(tp->tt) : 0);
  const unsigned grid = (unsigned)tp->n_tiles;
  const int bt = tp->bt;
  if (tp->gs)
    launch_tile_stage1<T, true>(s->p, grid, bt, b1, st, P, g, Za, Sa, gas, eps, share, rec, cf, V, R1, partial, ctl, ba);
  else
    launch_tile_stage1<T, false>(s->p, grid, bt, b1, st, P, g, Za, Sa, gas, eps, share, rec, cf, V, R1, partial, ctl,
                                 ba);
  if (ev) cudaEventRecord(ev[1], st);
  const unsigned gb = tp->n_bvert > 0 ? nblk(tp->n_bvert, TILE_BND_BLOCK) : 1u;
  k_tile_bnd1<T><<<gb, TILE_BND_BLOCK, 0, st>>>(P, share, cf, V, R1, partial, (T)s->p.cfl, ctl);
  CU(cudaGetLastError());
  return RD_OK;
}

template <class T>
int tiled_stage2(rd_state* s, int a, cudaEvent_t* ev) {
  rd_mesh* m = s->m;
  const TilePlan* tp = s->tiles;
  cudaStream_t st = m->stream;
  const int b = 1 - a;
  const TileView P = view_of(s);
  const DevGeo<T> g = geo_view<T>(m);
  const T* V = (const T*)m->geo[s->pi][5].p;
  const T* Wa = (const T*)s->W[a].p;
  const T* R1 = (const T*)s->R1.p;
  T* share = (T*)s->share.p;
  DevCtl* ctl = (DevCtl*)s->ctl.p;
  const T gamma = (T)s->p.gamma, eps = (T)s->p.eps_fix;
  const Gas<T> gas = Gas<T>::of(gamma);
  const BlendArgs<T> ba = tile_blend_args<T>(s);
  const size_t b2 = smem_stage2<T>(tp->tt, tp->slots) + (tp->gs ? geo_bytes<T>(tp->tt) : 0);
  const unsigned grid = (unsigned)tp->n_tiles;
  const int bt = tp->bt;
  T* Wb = (T*)s->W[b].p;
  T* Zb = (T*)s->Z[b].p;
  T* Sb = (T*)s->spd[b].p;
  const T* rec = (const T*)s->rec.p;
  if (tp->gs)
    launch_tile_stage2<T, true>(s->p, grid, bt, b2, st, P, g, Wa, R1, V, rec, gas, gamma, eps, share, Wb, Zb, Sb, ctl,
                                ba);
  else
    launch_tile_stage2<T, false>(s->p, grid, bt, b2, st, P, g, Wa, R1, V, rec, gas, gamma, eps, share, Wb, Zb, Sb, ctl,
                                 ba);
  if (ev) cudaEventRecord(ev[4], st);
  if (tp->n_bvert > 0)
    k_tile_bnd2<T><<<nblk(tp->n_bvert, TILE_BND_BLOCK), TILE_BND_BLOCK, 0, st>>>(P, share, Wa, R1, V, gamma, Wb, Zb,
                                                                                Sb, ctl);
  CU(cudaGetLastError());
  return RD_OK;
}

template int tiled_stage1<double>(rd_state*, int, cudaEvent_t*);
template int tiled_stage1<float>(rd_state*, int, cudaEvent_t*);
template int tiled_stage2<double>(rd_state*, int, cudaEvent_t*);
template int tiled_stage2<float>(rd_state*, int, cudaEvent_t*);

// Upload a host plan into a fresh device plan of state s (bt threads per block).
int tile_plan_upload(rd_state* s, const TilePlanHost& hp, int bt, bool gs, TilePlan** out) {
  cudaStream_t st = s->m->stream;
  TilePlan* tp = new (std::nothrow) TilePlan();
  if (!tp) return RD_ENOMEM;
  tp->tt = hp.tt;
  tp->bt = bt;
  tp->gs = gs;
  tp->n_tiles = hp.n_tiles;
  tp->n_bvert = hp.n_bvert;
  tp->slots = hp.slots;
  auto up = [&](DevBuf& d, const void* src, size_t bytes) -> int {
    CK(dev_alloc(d, bytes, st));
    if (bytes) CU(cudaMemcpyAsync(d.p, src, bytes, cudaMemcpyHostToDevice, st));
    return RD_OK;
  };
  int rc = RD_OK;
  if (rc == RD_OK) rc = up(tp->vs, hp.vs.data(), hp.vs.size() * sizeof(int32_t));
  if (rc == RD_OK) rc = up(tp->hptr, hp.hptr.data(), hp.hptr.size() * sizeof(int32_t));
  if (rc == RD_OK) rc = up(tp->hlist, hp.hlist.data(), hp.hlist.size() * sizeof(int32_t));
  if (rc == RD_OK) rc = up(tp->lslot, hp.lslot.data(), hp.lslot.size() * sizeof(uint16_t));
  if (rc == RD_OK) rc = up(tp->bmask, hp.bmask.data(), hp.bmask.size());
  if (rc == RD_OK) rc = up(tp->bvert, hp.bvert.data(), hp.bvert.size() * sizeof(int32_t));
  const size_t nbb = hp.n_bvert > 0 ? nblk(hp.n_bvert, TILE_BND_BLOCK) : 1u;
  if (rc == RD_OK) rc = dev_alloc(tp->partial, ((size_t)hp.n_tiles + nbb) * sizeof(double), st);
  if (rc == RD_OK) {
    const size_t b1 = tile_smem_bytes(s->p.precision, 1, hp.tt, hp.slots, gs);
    const size_t b2 = tile_smem_bytes(s->p.precision, 2, hp.tt, hp.slots, gs);
    rc = s->pi == 0 ? tile_smem_attrs<double>(b1, b2) : tile_smem_attrs<float>(b1, b2);
  }
  if (rc == RD_OK && cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    rc = RD_ECUDA;
  }
  if (rc != RD_OK) {
    tile_plan_free(tp);
    return rc;
  }
  *out = tp;
  return RD_OK;
}

}  // namespace rd

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace rd;

extern "C" int rd_state_set_tiling(rd_state* s, int32_t tile_triangles, int32_t threads) {
  return rd_state_set_tiling_ex(s, tile_triangles, threads, 0);
}

extern "C" int rd_state_set_tiling_ex(rd_state* s, int32_t tile_triangles, int32_t threads, int32_t flags) {
  if (!s) return RD_EINVAL;
  if (flags & ~RD_TILE_STAGE_GEOMETRY) return RD_EINVAL;
  const bool gs = (flags & RD_TILE_STAGE_GEOMETRY) != 0;
  if (tile_triangles == 0) {
    if (s->tiles) {
      cudaStreamSynchronize(s->m->stream);
      tile_plan_free(s->tiles);
      s->tiles = nullptr;
    }
  } else {
    if (s->p.precision == RD_DF64) return RD_ENOTSUP;  // the double-float kernels are untiled
    if (threads < 32 || threads > TILE_MAX_THREADS || threads % 32) return RD_EINVAL;
    if (tile_triangles < 32 || tile_triangles > MAX_TILE_TRIANGLES || tile_triangles % 32) return RD_EINVAL;
    TilePlanHost hp;
    CK(build_tile_plan(s->m->h, tile_triangles, hp));
    int dev = 0, optin = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t need = std::max(tile_smem_bytes(s->p.precision, 1, hp.tt, hp.slots, gs),
                                 tile_smem_bytes(s->p.precision, 2, hp.tt, hp.slots, gs)) + 1024;
    if (need > (size_t)optin) return RD_ENOTSUP;
    TilePlan* tp = nullptr;
    CK(tile_plan_upload(s, hp, threads, gs, &tp));
    if (s->tiles) {
      cudaStreamSynchronize(s->m->stream);
      tile_plan_free(s->tiles);
    }
    s->tiles = tp;
  }
  if (s->g2) {  // the captured graph holds the old kernels
    cudaGraphExecDestroy(s->g2);
    s->g2 = nullptr;
  }
  s->graph_failed = false;
  return RD_OK;
}

extern "C" int rd_state_get_tiling(const rd_state* s, int32_t* tile_triangles, int32_t* threads,
                                   int32_t* n_boundary_vertices) {
  if (!s) return RD_EINVAL;
  if (tile_triangles) *tile_triangles = s->tiles ? s->tiles->tt : 0;
  if (threads) *threads = s->tiles ? s->tiles->bt : 0;
  if (n_boundary_vertices) *n_boundary_vertices = s->tiles ? s->tiles->n_bvert : 0;
  return RD_OK;
}

extern "C" int rd_state_get_tiling_flags(const rd_state* s, int32_t* flags) {
  if (!s || !flags) return RD_EINVAL;
  *flags = (s->tiles && s->tiles->gs) ? RD_TILE_STAGE_GEOMETRY : 0;
  return RD_OK;
}
