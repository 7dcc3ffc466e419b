// rd_adjoint.cu -- discrete adjoint of a rollout of the RD step, with checkpoints.
//
// rd_adjoint_forward advances a state n steps (ordinary CFL steps), records
// each step's dt and keeps the state every `ckpt_every` steps.
// rd_adjoint_backward then returns dL/dW0 for a given dL/dW_final of the SAME
// discrete map with the recorded dt sequence held fixed: for each segment,
// newest first, it re-runs the segment's steps from its checkpoint (keeping
// W^n of every step and the branch masks of both stages), then walks the
// steps backwards:
//   stage-2 triangle reverse -> gather -> lambda* (adjoint of W*)
//   stage-1 triangle reverse -> gather -> lambda^n
// Gathers go through the same vertex -> corner CSR as the forward pass, so
// the adjoint is deterministic too.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "rd_adjoint.cuh"
#include "rd_device.h"
#include "rd_internal.h"

using namespace rd;

namespace {

constexpr int ADJ_TRI_BLOCK = 128;
constexpr int ADJ_VTX_BLOCK = 256;

template <class T>
__device__ __forceinline__ void load_tri3(int t, int nt, const int* __restrict__ tri, const DevGeo<T>& g, int v[3],
                                          T nx[3], T ny[3], T hl[3]) {
  for (int c = 0; c < 3; ++c) {
    v[c] = __ldg(tri + (size_t)c * nt + t);
    nx[c] = __ldg(g.nx + (size_t)c * nt + t);
    ny[c] = __ldg(g.ny + (size_t)c * nt + t);
    hl[c] = __ldg(g.hl + (size_t)c * nt + t);
  }
}

__global__ void k_set_dt(DevCtl* ctl, double dt) { ctl->dt = dt; }
__global__ void k_record_dt(const DevCtl* ctl, double* out) { *out = ctl->dt; }

template <class T, int SCHEME>
__global__ void __launch_bounds__(ADJ_TRI_BLOCK) k_mask1(int nt, const int* __restrict__ tri, DevGeo<T> g,
                                                         const T* __restrict__ Z, T gamma, T eps,
                                                         Mask* __restrict__ mask) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int v[3];
  T nx[3], ny[3], hl[3], Zc[3][4];
  load_tri3(t, nt, tri, g, v, nx, ny, hl);
  for (int c = 0; c < 3; ++c) load_vec4(Z, v[c], Zc[c]);
  mask[t] = stage1_mask<T, SCHEME>(Zc, nx, ny, hl, gamma, eps);
}

template <class T, int SCHEME>
__global__ void __launch_bounds__(ADJ_TRI_BLOCK) k_mask2(int nt, const int* __restrict__ tri, DevGeo<T> g,
                                                         const T* __restrict__ Zs, const T* __restrict__ Wn,
                                                         const T* __restrict__ Ws, const T* __restrict__ rec, T dt,
                                                         T gamma, T eps, Mask* __restrict__ mask) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int v[3];
  T nx[3], ny[3], hl[3], Zc[3][4], wn[3][4], ws[3][4], r[16];
  load_tri3(t, nt, tri, g, v, nx, ny, hl);
  for (int c = 0; c < 3; ++c) {
    load_vec4(Zs, v[c], Zc[c]);
    load_vec4(Wn, v[c], wn[c]);
    load_vec4(Ws, v[c], ws[c]);
  }
  for (int k = 0; k < 4; ++k) ld4(rec + (size_t)t * 16 + 4 * k, r + 4 * k);
  mask[t] = stage2_mask<T, SCHEME>(Zc, wn, ws, r, nx, ny, hl, __ldg(g.area + t), dt, gamma, eps);
}

// Forward re-run kernels that also record the branch masks, so each triangle is
// linearised once per stage: the same steps as k_tri_stage1 / k_tri_stage2
// (linearise, LDA, blend, total residuals), with the masks read off the same
// intermediate values stage1_mask / stage2_mask compute.
template <class T, int SCHEME>
__global__ void __launch_bounds__(ADJ_TRI_BLOCK) k_stage1_masked(int nt, const int* __restrict__ tri, DevGeo<T> g,
                                                                 const T* __restrict__ Z, const T* __restrict__ spd,
                                                                 Gas<T> gas, T eps, T* __restrict__ share,
                                                                 T* __restrict__ rec, T* __restrict__ cfl,
                                                                 DevCtl* ctl, Mask* __restrict__ mask,
                                                                 T* __restrict__ lin = nullptr) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int v[3];
  T nx[3], ny[3], hl[3], Zc[3][4];
  load_tri3(t, nt, tri, g, v, nx, ny, hl);
  for (int c = 0; c < 3; ++c) load_vec4(Z, v[c], Zc[c]);
  {
    T s0 = __ldg(spd + v[0]), s1 = __ldg(spd + v[1]), s2 = __ldg(spd + v[2]);
    T lam = mag_less(s1, s0) ? s0 : s1;
    lam = mag_less(s2, lam) ? lam : s2;
    cfl[t] = __ldg(g.lmax + t) * lam;
  }
  TriLin<T> L;
  int st = linearise(Zc, nx, ny, hl, gas, eps, L);
  if (st) {
    mask[t] = 0;
    atomicOr(&ctl->status, st);
    return;
  }
  Mask mk = node_mask(L, hl, eps);
  if (lin) store_lin(L, lin, t, nt);
  T out[3][4];
  if (SCHEME == RD_N1) {
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 4; ++k) out[i][k] = L.phiN[i][k];
  } else {
    T lda[3][4];
    lda_apply(L, L.phiT, lda);
    if (SCHEME == RD_LDA2) {
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) out[i][k] = lda[i][k];
    } else {
      mk |= blend_mask(L.phiT, L.phiN);
      blend(L.phiT, L.phiN, lda, out);
    }
    T* rp = rec + (size_t)t * 16;
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 4; ++k) rp[4 * i + k] = L.phiN[i][k];
    for (int k = 0; k < 4; ++k) rp[12 + k] = L.phiT[k];
  }
  mask[t] = mk;
  T* sp = share + (size_t)t * 12;
  for (int i = 0; i < 3; ++i) st4(sp + 4 * i, out[i]);
}

template <class T, int SCHEME>
__global__ void __launch_bounds__(ADJ_TRI_BLOCK) k_stage2_masked(int nt, const int* __restrict__ tri, DevGeo<T> g,
                                                                 const T* __restrict__ Zs, const T* __restrict__ Wn,
                                                                 const T* __restrict__ Ws, const T* __restrict__ rec,
                                                                 Gas<T> gas, T eps, T* __restrict__ share,
                                                                 DevCtl* ctl, Mask* __restrict__ mask,
                                                                 T* __restrict__ lin = nullptr) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int v[3];
  T nx[3], ny[3], hl[3], Zc[3][4], wn[3][4], ws[3][4], r[16];
  load_tri3(t, nt, tri, g, v, nx, ny, hl);
  for (int c = 0; c < 3; ++c) {
    load_vec4(Zs, v[c], Zc[c]);
    load_vec4(Wn, v[c], wn[c]);
    load_vec4(Ws, v[c], ws[c]);
  }
  for (int k = 0; k < 4; ++k) ld4(rec + (size_t)t * 16 + 4 * k, r + 4 * k);
  const T dt = (T)ctl->dt;
  TriLin<T> L;
  int st = linearise(Zc, nx, ny, hl, gas, eps, L);
  if (st) {
    mask[t] = 0;
    atomicOr(&ctl->status, st);
    return;
  }
  Mask mk = node_mask(L, hl, eps);
  if (lin) store_lin(L, lin, t, nt);
  const T idt = rcp(dt);
  T PhiN[3][4], PhiT[4];
  stage2_totals(L, wn, ws, r, __ldg(g.area + t), idt, PhiN, PhiT);
  T lda[3][4], out[3][4];
  lda_apply(L, PhiT, lda);
  if (SCHEME == RD_LDA2) {
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 4; ++k) out[i][k] = lda[i][k];
  } else {
    mk |= blend_mask(PhiT, PhiN);
    blend(PhiT, PhiN, lda, out);
  }
  mask[t] = mk;
  T* sp = share + (size_t)t * 12;
  for (int i = 0; i < 3; ++i) st4(sp + 4 * i, out[i]);
}

// adjoint of the stage-2 triangle pass: per corner (Z*, W*, W^n) bars, per triangle the record bar
template <class T, int SCHEME, bool LIN>
__global__ void __launch_bounds__(ADJ_TRI_BLOCK) k_adj_stage2(int nt, const int* __restrict__ tri, DevGeo<T> g,
                                                              const T* __restrict__ V, const T* __restrict__ Zs,
                                                              const T* __restrict__ Wn, const T* __restrict__ Ws,
                                                              const T* __restrict__ rec,
                                                              const Mask* __restrict__ mask,
                                                              const T* __restrict__ lam_next, T dt, T gamma, T eps,
                                                              T* __restrict__ cb2, T* __restrict__ recb,
                                                              DevCtl* ctl, const T* __restrict__ lin = nullptr) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int v[3];
  T nx[3], ny[3], hl[3], Zc[3][4], wn[3][4], ws[3][4], r[16], ob[3][4];
  load_tri3(t, nt, tri, g, v, nx, ny, hl);
  for (int c = 0; c < 3; ++c) {
    load_vec4(Zs, v[c], Zc[c]);
    load_vec4(Wn, v[c], wn[c]);
    load_vec4(Ws, v[c], ws[c]);
    T lam[4];
    load_vec4(lam_next, v[c], lam);
    T f = dt / __ldg(V + v[c]);
    for (int k = 0; k < 4; ++k) ob[c][k] = -f * lam[k];
  }
  for (int k = 0; k < 4; ++k) ld4(rec + (size_t)t * 16 + 4 * k, r + 4 * k);
  T Zsb[3][4], Wnb[3][4], Wsb[3][4], rb[16];
  int st;
  if (LIN) {  // the forward re-run's linearisation of this triangle
    TriLin<T> L;
    load_lin(L, lin, t, nt);
    st = stage2_rev_lin<T, SCHEME>(L, Zc, wn, ws, r, nx, ny, hl, __ldg(g.area + t), dt, gamma, eps, __ldg(mask + t),
                                   ob, Zsb, Wnb, Wsb, rb);
  } else {
    st = stage2_rev<T, SCHEME>(Zc, wn, ws, r, nx, ny, hl, __ldg(g.area + t), dt, gamma, eps, __ldg(mask + t), ob,
                               Zsb, Wnb, Wsb, rb);
  }
  if (st) {
    atomicOr(&ctl->status, st);
    return;
  }
  T* o = cb2 + (size_t)t * 36;
  for (int c = 0; c < 3; ++c) {
    st4(o + 12 * c, Zsb[c]);
    st4(o + 12 * c + 4, Wsb[c]);
    st4(o + 12 * c + 8, Wnb[c]);
  }
  for (int k = 0; k < 4; ++k) st4(recb + (size_t)t * 16 + 4 * k, rb + 4 * k);
}

// lambda*_i = lambda^{n+1}_i + sum_corners (W* bar + (dZ/dW*)^T Z* bar)
template <class T>
__global__ void __launch_bounds__(ADJ_VTX_BLOCK) k_adj_gather2(int nv, const int* __restrict__ ptr,
                                                               const int* __restrict__ ent, const T* __restrict__ cb2,
                                                               const T* __restrict__ lam_next,
                                                               const T* __restrict__ Ws, T gamma,
                                                               T* __restrict__ lams) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  T zb[4] = {T(0), T(0), T(0), T(0)}, wb[4];
  load_vec4(lam_next, i, wb);
  int e0 = __ldg(ptr + i), e1 = __ldg(ptr + i + 1);
  for (int e = e0; e < e1; ++e) {
    int te = __ldg(ent + e);
    const T* o = cb2 + (size_t)(te / 3) * 36 + 12 * (te % 3);
    T a[4], b[4];
    ld4(o, a);
    ld4(o + 4, b);
    for (int k = 0; k < 4; ++k) {
      zb[k] += a[k];
      wb[k] += b[k];
    }
  }
  T w[4];
  load_vec4(Ws, i, w);
  vertex_Z_rev(w, gamma, zb, wb);
  st4(lams + 4 * (size_t)i, wb);
}

// adjoint of the stage-1 (or forward-Euler) triangle pass: per corner Z^n bar
template <class T, int SCHEME, bool LIN>
__global__ void __launch_bounds__(ADJ_TRI_BLOCK) k_adj_stage1(int nt, const int* __restrict__ tri, DevGeo<T> g,
                                                              const T* __restrict__ V, const T* __restrict__ Z,
                                                              const Mask* __restrict__ mask,
                                                              const T* __restrict__ lams,
                                                              const T* __restrict__ recb, T dt, T gamma, T eps,
                                                              T* __restrict__ cb1, DevCtl* ctl,
                                                              const T* __restrict__ lin = nullptr) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int v[3];
  T nx[3], ny[3], hl[3], Zc[3][4], ob[3][4], rb[16];
  load_tri3(t, nt, tri, g, v, nx, ny, hl);
  for (int c = 0; c < 3; ++c) {
    load_vec4(Z, v[c], Zc[c]);
    T lam[4];
    load_vec4(lams, v[c], lam);
    T f = dt / __ldg(V + v[c]);
    for (int k = 0; k < 4; ++k) ob[c][k] = -f * lam[k];
  }
  if (recb) {
    for (int k = 0; k < 4; ++k) ld4(recb + (size_t)t * 16 + 4 * k, rb + 4 * k);
  } else {
    for (int k = 0; k < 16; ++k) rb[k] = T(0);
  }
  T Zb[3][4];
  int st;
  if (LIN) {  // the forward re-run's linearisation of this triangle
    TriLin<T> L;
    load_lin(L, lin, t, nt);
    st = stage1_rev_lin<T, SCHEME>(L, Zc, nx, ny, hl, gamma, eps, __ldg(mask + t), ob, rb, Zb);
  } else {
    st = stage1_rev<T, SCHEME>(Zc, nx, ny, hl, gamma, eps, __ldg(mask + t), ob, rb, Zb);
  }
  if (st) {
    atomicOr(&ctl->status, st);
    return;
  }
  T* o = cb1 + (size_t)t * 12;
  for (int c = 0; c < 3; ++c) st4(o + 4 * c, Zb[c]);
}

// lambda^n_i = lambda*_i + sum_corners (W^n bar of stage 2) + (dZ/dW^n)^T sum_corners (Z^n bar of stage 1)
template <class T>
__global__ void __launch_bounds__(ADJ_VTX_BLOCK) k_adj_gather1(int nv, const int* __restrict__ ptr,
                                                               const int* __restrict__ ent, const T* __restrict__ cb1,
                                                               const T* __restrict__ cb2, const T* __restrict__ lams,
                                                               const T* __restrict__ Wn, T gamma,
                                                               T* __restrict__ lam_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  T zb[4] = {T(0), T(0), T(0), T(0)}, wb[4];
  load_vec4(lams, i, wb);
  int e0 = __ldg(ptr + i), e1 = __ldg(ptr + i + 1);
  for (int e = e0; e < e1; ++e) {
    int te = __ldg(ent + e);
    T a[4];
    ld4(cb1 + (size_t)te * 4, a);
    for (int k = 0; k < 4; ++k) zb[k] += a[k];
    if (cb2) {
      T b[4];
      ld4(cb2 + (size_t)(te / 3) * 36 + 12 * (te % 3) + 8, b);
      for (int k = 0; k < 4; ++k) wb[k] += b[k];
    }
  }
  T w[4];
  load_vec4(Wn, i, w);
  vertex_Z_rev(w, gamma, zb, wb);
  st4(lam_out + 4 * (size_t)i, wb);
}

}  // namespace

// ---------------------------------------------------------------------------
// state-side bookkeeping (buffers live in a separate struct owned by rd_state)
// ---------------------------------------------------------------------------
struct rd_adjoint_store {
  int32_t n_steps = 0, ckpt_every = 0, n_ckpt = 0;
  std::vector<double> dts;                 // host copy of the recorded dt sequence
  DevBuf dts_dev, ckpt, segW, Zn, spd, Ws, Zs, R1, share, rec, cfl, partial, ctl, mask1, mask2, lam, lams, cb1,
      cb2, recb, stage;
  // two-stage schemes, when a segment's worth fits in a quarter of the free device
  // memory: Z^n, W*, Z* and the stage-2 record of every step of the segment, kept
  // from the forward re-run so that the reverse sweep does not recompute stage 1
  DevBuf segZn, segWs, segZs, segRec;
  bool stored = false;
  // and, when that leaves room, both stages' linearisations of every triangle
  // and step (LIN_WORDS words each, field-major), so that the reverse kernels
  // do not linearise again
  DevBuf segL1, segL2;
  bool storedL = false;
  ~rd_adjoint_store() {
    DevBuf* b[] = {&dts_dev, &ckpt, &segW, &Zn, &spd, &Ws, &Zs, &R1, &share, &rec, &cfl, &partial, &ctl,
                   &mask1, &mask2, &lam, &lams, &cb1, &cb2, &recb, &stage, &segZn, &segWs, &segZs, &segRec,
                   &segL1, &segL2};
    for (DevBuf* d : b) dev_free(*d);
  }
};

void rd::adjoint_free(rd_adjoint_store* a) { delete a; }

namespace {

template <class T>
DevGeo<T> geo(const rd_mesh* m, int pi) {
  return DevGeo<T>{(const T*)m->geo[pi][0].p, (const T*)m->geo[pi][1].p, (const T*)m->geo[pi][2].p,
                   (const T*)m->geo[pi][3].p, (const T*)m->geo[pi][4].p};
}

int ensure(rd_adjoint_store* A, rd_state* s, cudaStream_t st) {
  const size_t nv = s->m->h.nv, nt = s->m->h.nt, ts = s->ts, k = (size_t)A->ckpt_every;
  if (A->segW.p) return RD_OK;
  CK(dev_alloc(A->segW, (k + 1) * 4 * nv * ts, st));
  CK(dev_alloc(A->Zn, 4 * nv * ts, st));
  CK(dev_alloc(A->spd, nv * ts, st));
  CK(dev_alloc(A->Ws, 4 * nv * ts, st));
  CK(dev_alloc(A->Zs, 4 * nv * ts, st));
  CK(dev_alloc(A->R1, 4 * nv * ts, st));
  CK(dev_alloc(A->share, 12 * nt * ts, st));
  CK(dev_alloc(A->rec, 16 * nt * ts, st));
  CK(dev_alloc(A->cfl, nt * ts, st));
  CK(dev_alloc(A->partial, (size_t)nblk(nv, VTX_BLOCK_MIN) * ts, st));
  CK(dev_alloc(A->ctl, sizeof(DevCtl), st));
  CK(dev_alloc(A->mask1, k * nt * sizeof(Mask), st));
  CK(dev_alloc(A->mask2, k * nt * sizeof(Mask), st));
  CK(dev_alloc(A->lam, 4 * nv * ts, st));
  CK(dev_alloc(A->lams, 4 * nv * ts, st));
  CK(dev_alloc(A->cb1, 12 * nt * ts, st));
  CK(dev_alloc(A->cb2, 36 * nt * ts, st));
  CK(dev_alloc(A->recb, 16 * nt * ts, st));
  CK(dev_alloc(A->stage, 4 * nv * sizeof(double), st));
  A->stored = false;
  if (s->p.scheme != RD_N1) {
    size_t free_b = 0, total_b = 0;
    const size_t need = k * (12 * nv + 16 * nt) * ts;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && need <= free_b / 4) {
      if (dev_alloc(A->segZn, k * 4 * nv * ts, st) == RD_OK && dev_alloc(A->segWs, k * 4 * nv * ts, st) == RD_OK &&
          dev_alloc(A->segZs, k * 4 * nv * ts, st) == RD_OK && dev_alloc(A->segRec, k * 16 * nt * ts, st) == RD_OK)
        A->stored = true;
    }
    cudaGetLastError();
    if (!A->stored) {  // recompute instead
      dev_free(A->segZn);
      dev_free(A->segWs);
      dev_free(A->segZs);
      dev_free(A->segRec);
    }
  }
  A->storedL = false;
  if (A->stored || s->p.scheme == RD_N1) {
    size_t free_b = 0, total_b = 0;
    const size_t lin = k * LIN_WORDS * nt * ts;
    const int nl = s->p.scheme == RD_N1 ? 1 : 2;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && nl * lin <= free_b / 4) {
      if (dev_alloc(A->segL1, lin, st) == RD_OK && (nl == 1 || dev_alloc(A->segL2, lin, st) == RD_OK))
        A->storedL = true;
    }
    cudaGetLastError();
    if (!A->storedL) {
      dev_free(A->segL1);
      dev_free(A->segL2);
    }
  }
  return RD_OK;
}

template <class T, int S>
int backward(rd_state* s, rd_adjoint_store* A, const double* dLdWf, double* dLdW0) {
  rd_mesh* m = s->m;
  cudaStream_t st = m->stream;
  const int nv = m->h.nv, nt = m->h.nt, pi = s->pi, k = A->ckpt_every;
  const bool two = (S != RD_N1);
  DevGeo<T> g = geo<T>(m, pi);
  const T* V = (const T*)m->geo[pi][5].p;
  const int* tri = (const int*)m->tri.p;
  const int* ptr = (const int*)m->ptr.p;
  const int* ent = (const int*)m->ent.p;
  DevCtl* ctl = (DevCtl*)A->ctl.p;
  const T gamma = (T)s->p.gamma, eps = (T)s->p.eps_fix, cflnum = (T)s->p.cfl;
  const unsigned gt = nblk(nt, ADJ_TRI_BLOCK), gv = nblk(nv, ADJ_VTX_BLOCK);
  const size_t wsz = 4 * (size_t)nv;
  T* segW = (T*)A->segW.p;
  T* Zn = (T*)A->Zn.p;
  T* spd = (T*)A->spd.p;
  T* Ws = (T*)A->Ws.p;
  T* Zs = (T*)A->Zs.p;
  T* lam = (T*)A->lam.p;
  T* lams = (T*)A->lams.p;
  T* share = (T*)A->share.p;
  T* rec = (T*)A->rec.p;
  T* cf = (T*)A->cfl.p;
  Mask* mask1 = (Mask*)A->mask1.p;
  Mask* mask2 = (Mask*)A->mask2.p;
  CU(cudaMemsetAsync(ctl, 0, sizeof(DevCtl), st));
  // dL/dW_final (caller order, double) -> lam (internal order, T)
  CU(cudaMemcpyAsync(A->stage.p, dLdWf, wsz * sizeof(double), cudaMemcpyHostToDevice, st));
  k_permute_in<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, (const int*)m->vperm.p, (const double*)A->stage.p, lam, ctl);

  // stage-1 pass at W^n (shares, record, CFL terms), then W*, Z* with the recorded dt
  auto stage1_and_wstar = [&](const T* Wn, double dt, T* Wout, T* Zout) {
    k_prepare<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, Wn, gamma, Zn, spd, ctl);
    k_tri_stage1<T, S><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, nv, tri, g, Zn, spd, Gas<T>::of(gamma), eps, share, two ? rec : nullptr,
                                                      cf, ctl);
    launch_gather_cfl<T>(VTX_BLOCK, st, nv, ptr, ent, share, cf, V, (T*)A->R1.p, (T*)A->partial.p, cflnum, ctl);
    k_set_dt<<<1, 1, 0, st>>>(ctl, dt);
    k_update<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, Wn, (const T*)A->R1.p, ptr, ent, nullptr, V, gamma, Wout, Zout,
                                              nullptr, ctl);
  };

  for (int seg = A->n_ckpt - 1; seg >= 0; --seg) {
    const int n0 = seg * k, n1 = std::min(n0 + k, A->n_steps);
    CU(cudaMemcpyAsync(segW, (const T*)A->ckpt.p + (size_t)seg * wsz, wsz * sizeof(T), cudaMemcpyDeviceToDevice, st));
    // forward re-run of the segment: keep W^n of every step and both stages' masks
    // (each triangle linearised once per stage: the masks come with the shares)
    for (int j = 0; j < n1 - n0; ++j) {
      const double dt = A->dts[n0 + j];
      T* Wn = segW + (size_t)j * wsz;
      T* Wn1 = segW + (size_t)(j + 1) * wsz;
      T* Znj = A->stored ? (T*)A->segZn.p + (size_t)j * wsz : Zn;
      T* Wsj = A->stored ? (T*)A->segWs.p + (size_t)j * wsz : Ws;
      T* Zsj = A->stored ? (T*)A->segZs.p + (size_t)j * wsz : Zs;
      T* recj = A->stored ? (T*)A->segRec.p + (size_t)j * 16 * nt : rec;
      T* lin1 = A->storedL ? (T*)A->segL1.p + (size_t)j * LIN_WORDS * nt : nullptr;
      T* lin2 = A->storedL && two ? (T*)A->segL2.p + (size_t)j * LIN_WORDS * nt : nullptr;
      k_prepare<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, Wn, gamma, Znj, spd, ctl);
      k_stage1_masked<T, S><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, tri, g, Znj, spd, Gas<T>::of(gamma), eps, share,
                                                          recj, cf, ctl, mask1 + (size_t)j * nt, lin1);
      launch_gather_cfl<T>(VTX_BLOCK, st, nv, ptr, ent, share, cf, V, (T*)A->R1.p, (T*)A->partial.p, cflnum, ctl);
      k_set_dt<<<1, 1, 0, st>>>(ctl, dt);
      if (two) {
        k_update<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, Wn, (const T*)A->R1.p, ptr, ent, nullptr, V, gamma, Wsj, Zsj,
                                                  nullptr, ctl);
        k_stage2_masked<T, S><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, tri, g, Zsj, Wn, Wsj, recj, Gas<T>::of(gamma), eps,
                                                            share, ctl, mask2 + (size_t)j * nt, lin2);
        // Z of W^{n+1} is not needed (the next step's k_prepare recomputes it): scratch
        k_update<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, Wsj, nullptr, ptr, ent, share, V, gamma, Wn1, Zs, nullptr, ctl);
      } else {
        k_update<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, Wn, (const T*)A->R1.p, ptr, ent, nullptr, V, gamma, Wn1, Zs,
                                                  nullptr, ctl);
      }
    }
    // reverse sweep over the segment
    for (int j = n1 - n0 - 1; j >= 0; --j) {
      const double dt = A->dts[n0 + j];
      T* Wn = segW + (size_t)j * wsz;
      const T* lin1 = A->storedL ? (const T*)A->segL1.p + (size_t)j * LIN_WORDS * nt : nullptr;
      const T* lin2 = A->storedL && two ? (const T*)A->segL2.p + (size_t)j * LIN_WORDS * nt : nullptr;
      if (two) {
        T *Znj = Zn, *Wsj = Ws, *Zsj = Zs, *recj = rec;
        if (A->stored) {  // kept by the forward re-run
          Znj = (T*)A->segZn.p + (size_t)j * wsz;
          Wsj = (T*)A->segWs.p + (size_t)j * wsz;
          Zsj = (T*)A->segZs.p + (size_t)j * wsz;
          recj = (T*)A->segRec.p + (size_t)j * 16 * nt;
        } else {
          stage1_and_wstar(Wn, dt, Ws, Zs);
        }
        if (lin2)
          k_adj_stage2<T, S, true><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, tri, g, V, Zsj, Wn, Wsj, recj,
                                                                 mask2 + (size_t)j * nt, lam, (T)dt, gamma, eps,
                                                                 (T*)A->cb2.p, (T*)A->recb.p, ctl, lin2);
        else
          k_adj_stage2<T, S, false><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, tri, g, V, Zsj, Wn, Wsj, recj,
                                                                  mask2 + (size_t)j * nt, lam, (T)dt, gamma, eps,
                                                                  (T*)A->cb2.p, (T*)A->recb.p, ctl, nullptr);
        k_adj_gather2<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, ptr, ent, (const T*)A->cb2.p, lam, Wsj, gamma, lams);
        if (lin1)
          k_adj_stage1<T, S, true><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, tri, g, V, Znj, mask1 + (size_t)j * nt, lams,
                                                                 (const T*)A->recb.p, (T)dt, gamma, eps,
                                                                 (T*)A->cb1.p, ctl, lin1);
        else
          k_adj_stage1<T, S, false><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, tri, g, V, Znj, mask1 + (size_t)j * nt, lams,
                                                                  (const T*)A->recb.p, (T)dt, gamma, eps,
                                                                  (T*)A->cb1.p, ctl, nullptr);
        k_adj_gather1<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, ptr, ent, (const T*)A->cb1.p, (const T*)A->cb2.p, lams,
                                                       Wn, gamma, lam);
      } else {
        k_prepare<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, Wn, gamma, Zn, spd, ctl);
        if (lin1)
          k_adj_stage1<T, S, true><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, tri, g, V, Zn, mask1 + (size_t)j * nt, lam,
                                                                 nullptr, (T)dt, gamma, eps, (T*)A->cb1.p, ctl, lin1);
        else
          k_adj_stage1<T, S, false><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, tri, g, V, Zn, mask1 + (size_t)j * nt, lam,
                                                                  nullptr, (T)dt, gamma, eps, (T*)A->cb1.p, ctl,
                                                                  nullptr);
        k_adj_gather1<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, ptr, ent, (const T*)A->cb1.p, nullptr, lam, Wn, gamma,
                                                       lam);
      }
    }
    CU(cudaGetLastError());
  }
  k_permute_out<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, (const int*)m->vperm.p, lam, (double*)A->stage.p);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(dLdW0, A->stage.p, wsz * sizeof(double), cudaMemcpyDeviceToHost, st));
  DevCtl c;
  CU(cudaMemcpyAsync(&c, ctl, sizeof(c), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return c.status ? RD_ENONPHYSICAL : RD_OK;
}

}  // namespace

extern "C" int rd_adjoint_forward(rd_state* s, int32_t n_steps, int32_t ckpt_every, double* dts_out) {
  if (s && (s->p.scheme > RD_LDA2 || s->p.lumping != RD_LUMP_GLOBAL || s->m->n_ghost || s->m->n_wall ||
            s->p.precision == RD_DF64))
    return RD_ENOTSUP;
  if (!s || n_steps < 1 || ckpt_every < 1) return RD_EINVAL;
  rd_mesh* m = s->m;
  cudaStream_t st = m->stream;
  DevCtl c0;
  CK(state_read_ctl(s, c0));
  if (c0.status) return RD_ENONPHYSICAL;
  if (!s->adj || s->adj->n_steps != n_steps || s->adj->ckpt_every != ckpt_every) {
    delete s->adj;
    s->adj = new (std::nothrow) rd_adjoint_store();
    if (!s->adj) return RD_ENOMEM;
  }
  rd_adjoint_store* A = s->adj;
  A->n_steps = n_steps;
  A->ckpt_every = ckpt_every;
  A->n_ckpt = (n_steps + ckpt_every - 1) / ckpt_every;
  const size_t wsz = 4 * (size_t)m->h.nv * s->ts;
  if (!A->ckpt.p) CK(dev_alloc(A->ckpt, (size_t)A->n_ckpt * wsz, st));
  if (!A->dts_dev.p) CK(dev_alloc(A->dts_dev, (size_t)n_steps * sizeof(double), st));
  CK(ensure(A, s, st));
  int a = (int)(c0.steps & 1);
  for (int32_t n = 0; n < n_steps; ++n) {
    if (n % ckpt_every == 0)
      CU(cudaMemcpyAsync((char*)A->ckpt.p + (size_t)(n / ckpt_every) * wsz, s->W[a].p, wsz, cudaMemcpyDeviceToDevice,
                         st));
    CK(state_step(s, a, 0.0));
    k_record_dt<<<1, 1, 0, st>>>((const DevCtl*)s->ctl.p, (double*)A->dts_dev.p + n);
    a ^= 1;
  }
  CU(cudaGetLastError());
  A->dts.assign(n_steps, 0.0);
  CU(cudaMemcpyAsync(A->dts.data(), A->dts_dev.p, n_steps * sizeof(double), cudaMemcpyDeviceToHost, st));
  DevCtl c;
  CK(state_read_ctl(s, c));
  s->launched = c.steps;
  if (c.status || c.steps != c0.steps + n_steps) {
    A->n_steps = 0;
    return RD_ENONPHYSICAL;
  }
  if (dts_out) std::memcpy(dts_out, A->dts.data(), n_steps * sizeof(double));
  return RD_OK;
}

extern "C" int rd_adjoint_backward(rd_state* s, const double* dL_dW_final, double* dL_dW0) {
  if (s && (s->p.scheme > RD_LDA2 || s->p.lumping != RD_LUMP_GLOBAL || s->m->n_ghost || s->m->n_wall ||
            s->p.precision == RD_DF64))
    return RD_ENOTSUP;
  if (!s || !dL_dW_final || !dL_dW0 || !s->adj || s->adj->n_steps < 1) return RD_EINVAL;
  rd_adjoint_store* A = s->adj;
  if (s->pi == 0) {
    switch (s->p.scheme) {
      case RD_N1: return backward<double, RD_N1>(s, A, dL_dW_final, dL_dW0);
      case RD_B2: return backward<double, RD_B2>(s, A, dL_dW_final, dL_dW0);
      default: return backward<double, RD_LDA2>(s, A, dL_dW_final, dL_dW0);
    }
  }
  switch (s->p.scheme) {
    case RD_N1: return backward<float, RD_N1>(s, A, dL_dW_final, dL_dW0);
    case RD_B2: return backward<float, RD_B2>(s, A, dL_dW_final, dL_dW0);
    default: return backward<float, RD_LDA2>(s, A, dL_dW_final, dL_dW0);
  }
}

namespace {

template <class T, int S>
int branch_masks(rd_state* s, uint64_t* mask1, uint64_t* mask2) {
  rd_mesh* m = s->m;
  cudaStream_t st = m->stream;
  rd_adjoint_store* A = s->adj;
  const int nv = m->h.nv, nt = m->h.nt, pi = s->pi;
  DevGeo<T> g = geo<T>(m, pi);
  const T* V = (const T*)m->geo[pi][5].p;
  const int* tri = (const int*)m->tri.p;
  const int* ptr = (const int*)m->ptr.p;
  const int* ent = (const int*)m->ent.p;
  DevCtl* ctl = (DevCtl*)A->ctl.p;
  const T gamma = (T)s->p.gamma, eps = (T)s->p.eps_fix, cflnum = (T)s->p.cfl;
  const unsigned gt = nblk(nt, ADJ_TRI_BLOCK), gv = nblk(nv, ADJ_VTX_BLOCK);
  DevCtl c;
  CK(state_read_ctl(s, c));
  const T* Wn = (const T*)s->W[(int)(c.steps & 1)].p;
  CU(cudaMemsetAsync(ctl, 0, sizeof(DevCtl), st));
  k_prepare<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, Wn, gamma, (T*)A->Zn.p, (T*)A->spd.p, ctl);
  k_tri_stage1<T, S><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, nv, tri, g, (const T*)A->Zn.p, (const T*)A->spd.p, Gas<T>::of(gamma), eps,
                                                    (T*)A->share.p, (T*)A->rec.p, (T*)A->cfl.p, ctl);
  launch_gather_cfl<T>(VTX_BLOCK, st, nv, ptr, ent, (const T*)A->share.p, (const T*)A->cfl.p, V, (T*)A->R1.p,
                       (T*)A->partial.p, cflnum, ctl);
  k_update<T><<<gv, ADJ_VTX_BLOCK, 0, st>>>(nv, Wn, (const T*)A->R1.p, ptr, ent, nullptr, V, gamma, (T*)A->Ws.p,
                                            (T*)A->Zs.p, nullptr, ctl);
  k_mask1<T, S><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, tri, g, (const T*)A->Zn.p, gamma, eps, (Mask*)A->mask1.p);
  DevCtl cc;
  CU(cudaMemcpyAsync(&cc, ctl, sizeof(cc), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (cc.status) return RD_ENONPHYSICAL;
  if (S != RD_N1)
    k_mask2<T, S><<<gt, ADJ_TRI_BLOCK, 0, st>>>(nt, tri, g, (const T*)A->Zs.p, Wn, (const T*)A->Ws.p,
                                                (const T*)A->rec.p, (T)cc.dt, gamma, eps, (Mask*)A->mask2.p);
  CU(cudaGetLastError());
  std::vector<Mask> h1(nt), h2(nt, 0);
  CU(cudaMemcpyAsync(h1.data(), A->mask1.p, nt * sizeof(Mask), cudaMemcpyDeviceToHost, st));
  if (S != RD_N1) CU(cudaMemcpyAsync(h2.data(), A->mask2.p, nt * sizeof(Mask), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  for (int t = 0; t < nt; ++t) {
    if (mask1) mask1[m->h.tperm[t]] = h1[t];
    if (mask2) mask2[m->h.tperm[t]] = h2[t];
  }
  return RD_OK;
}

}  // namespace

extern "C" int rd_state_branch_masks(rd_state* s, uint64_t* mask1, uint64_t* mask2) {
  if (s && (s->p.scheme > RD_LDA2 || s->p.lumping != RD_LUMP_GLOBAL || s->m->n_ghost || s->m->n_wall ||
            s->p.precision == RD_DF64))
    return RD_ENOTSUP;
  if (!s) return RD_EINVAL;
  cudaStream_t st = s->m->stream;
  if (!s->adj) {
    s->adj = new (std::nothrow) rd_adjoint_store();
    if (!s->adj) return RD_ENOMEM;
    s->adj->ckpt_every = 1;
  }
  CK(ensure(s->adj, s, st));
  if (s->pi == 0) {
    switch (s->p.scheme) {
      case RD_N1: return branch_masks<double, RD_N1>(s, mask1, mask2);
      case RD_B2: return branch_masks<double, RD_B2>(s, mask1, mask2);
      default: return branch_masks<double, RD_LDA2>(s, mask1, mask2);
    }
  }
  switch (s->p.scheme) {
    case RD_N1: return branch_masks<float, RD_N1>(s, mask1, mask2);
    case RD_B2: return branch_masks<float, RD_B2>(s, mask1, mask2);
    default: return branch_masks<float, RD_LDA2>(s, mask1, mask2);
  }
}
