// rd_df64_kernels.cuh -- triangle kernels of the RD_DF64 precision: FP64
// state, FP64 vertex kernels, per-triangle algebra (Sec. 3.2-3.4) in
// double-float.  The launchers df_stage1 / df_stage2 (declared in rd_df64.h)
// take a register budget and a barrier setting; each rd_df64_s*_r*.cu
// translation unit instantiates one stage at one or two budgets, so that the
// large straight-line kernels compile in parallel.
//
// GB300 runs FP64 at 1/64 of its FP32 rate and the FP64 triangle kernels keep
// the FP64 pipe ~90 % busy.  These kernels form, in double precision, only
// the quantities whose cancellation carries the residual -- the nodal mean
// Zbar and the differences Z_i - Zbar of each triangle, and in stage 2 the
// state change W*_i - W^n_i -- and run everything else (Roe state, eigen-split,
// phi^T, the 4x4 LU, N / LDA / blend, stage-2 totals) in double-float
// arithmetic (rd_dfloat.cuh) on the FP32 pipe.  Inputs and outputs keep the
// FP64 layout of the plain step, so the gathers, updates and the dt reduction
// are the FP64 ones; the stage-2 record phi^N(W^n), phi^T(W^n) stays in
// double-float (two floats per value: the bytes of one double).
#pragma once

#include <cuda_runtime.h>

#include "rd_device.h"
#include "rd_df64.h"
#include "rd_dfloat.cuh"
#include "rd_internal.h"
#include "rd_kernels.cuh"
#include "rd_tiled.h"

namespace rd {

namespace {

using dw::from_df;
using dw::to_df;

// Zbar (double, then split) and dZ_i = Z_i - Zbar of one triangle; the double
// operations are non-contractible so that every kernel variant forms the same bits.
__device__ __forceinline__ void split_nodal(const double Z[3][4], dfloat Zb[4], dfloat dZ[3][4]) {
  const double third = 1.0 / 3.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double zb = __dmul_rn(__dadd_rn(__dadd_rn(Z[0][k], Z[1][k]), Z[2][k]), third);
    Zb[k] = to_df(zb);
#pragma unroll
    for (int c = 0; c < 3; ++c) dZ[c][k] = to_df(__dsub_rn(Z[c][k], zb));
  }
}

__device__ __forceinline__ dfloat ld_df(const float2* p) {
  const float2 a = __ldg(p);
  return dfloat(a.x, a.y);
}

// Per-triangle geometry of the double-float kernels: unit normals and half
// edge lengths [3][nt] and areas [nt] already split into double-float pairs
// (float2), so no conversion runs per triangle; l_max in double for the CFL term.
__device__ __forceinline__ void load_tri_df(int t, int nt, const int* __restrict__ tri, const DevGeoDF& g, int v[3],
                                            dfloat nx[3], dfloat ny[3], dfloat hl[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v[c] = __ldg(tri + (size_t)c * nt + t);
    nx[c] = ld_df(g.nx + (size_t)c * nt + t);
    ny[c] = ld_df(g.ny + (size_t)c * nt + t);
    hl[c] = ld_df(g.hl + (size_t)c * nt + t);
  }
}

// W*_i - W^n_i of a triangle's corners, split into double-float by the stage-1
// vertex update.  Loaded after the linearisation at W*, where it is first
// needed, so that its 24 registers are not live across it.
__device__ __forceinline__ void ld_dw(const float2* __restrict__ dw, const int v[3], dfloat dW[3][4]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float4* q = reinterpret_cast<const float4*>(dw + 4 * (size_t)v[c]);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    dW[c][0] = dfloat(a.x, a.y);
    dW[c][1] = dfloat(a.z, a.w);
    dW[c][2] = dfloat(b.x, b.y);
    dW[c][3] = dfloat(b.z, b.w);
  }
}

// 16-value stage-2 record in double-float: 32 floats, eight 16-byte vectors.
__device__ __forceinline__ void st_rec(dfloat* p, const dfloat r[16]) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int k = 0; k < 8; ++k) q[k] = make_float4(r[2 * k].hi, r[2 * k].lo, r[2 * k + 1].hi, r[2 * k + 1].lo);
}
__device__ __forceinline__ void ld_rec(const dfloat* p, dfloat r[16]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 a = __ldg(q + k);
    r[2 * k] = dfloat(a.x, a.y);
    r[2 * k + 1] = dfloat(a.z, a.w);
  }
}

// REGS: register budget per thread (128, 96 or 80: four, five or six warps per
// SM sub-partition).  The kernel is latency-bound on its double-float
// dependency chains, so resident warps matter more than spills: 128 registers
// (a few hundred bytes of spills) measured 1.4-1.7x faster than the spill-free
// 255-register build, and 168 (three warps, almost no spills) 1.2x slower
// than 128.  Below 128 the spills grow (at the N-scheme solve the 4x4 LU, the
// three node systems, the Roe state and the linearised states are live
// together), and only the barrier variant gains.  SYNC: a block barrier between the
// phases of the per-triangle algebra.  The body is ~10^4 instructions of
// straight-line code, far more than the instruction caches hold, and warps
// that drift apart miss in them (ncu: "no instruction" is the leading stall);
// the barriers keep a block's warps on the same stretch of code.  Every
// thread reaches every barrier: threads past the last triangle repeat the
// last one without storing, and a failed phase only skips the later phases'
// arithmetic.  The autotuner picks the variant.
__device__ __forceinline__ void phase_sync(bool on) {
  if (on) __syncthreads();
}

// One flag per block: the control block's stop word read once, so that every
// thread of the block takes the same branch around the barriers.
__device__ __forceinline__ bool block_stop(const DevCtl* ctl) {
  __shared__ int stop;
  if (threadIdx.x == 0) stop = ctl->stop;
  __syncthreads();
  return stop != 0;
}

template <int SCHEME, int REGS, bool SYNC>
__global__ void __maxnreg__(REGS)
    k_tri_stage1_df(int nt, const int* __restrict__ tri, DevGeoDF g, const double* __restrict__ Z,
                    const double* __restrict__ spd, Gas<dfloat> gas, dfloat eps, double* __restrict__ share,
                    dfloat* __restrict__ rec, double* __restrict__ cfl, DevCtl* ctl, BlendArgs<double> ba) {
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (SYNC) {
    if (block_stop(ctl)) return;
  } else if (t0 >= nt || ctl->stop) {
    return;
  }
  const bool act = t0 < nt;
  const int t = act ? t0 : nt - 1;
  int v[3];
  double Zc[3][4];
  dfloat nxd[3], nyd[3], hld[3];
  load_tri_df(t, nt, tri, g, v, nxd, nyd, hld);
#pragma unroll
  for (int c = 0; c < 3; ++c) load_vec4(Z, v[c], Zc[c]);
  {
    double s0 = __ldg(spd + v[0]), s1 = __ldg(spd + v[1]), s2 = __ldg(spd + v[2]);
    double lam = mag_less(s1, s0) ? s0 : s1;  // speeds are >= 0
    lam = mag_less(s2, lam) ? lam : s2;
    if (act) cfl[t] = __dmul_rn(__ldg(g.lmax + t), lam);
  }
  const int mode = SCHEME == RD_BMAX2 ? ba.mode : BLEND_B;
  double thx = 0.0;
  if (SCHEME == RD_BMAX2 && mode == BLEND_X) {
    double nx[3], ny[3], hl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      nx[c] = from_df(nxd[c]);
      ny[c] = from_df(nyd[c]);
      hl[c] = from_df(hld[c]);
    }
    thx = bx_theta(Zc, nx, ny, hl, from_df(ld_df(g.area + t)), ba.L, vrange_of<double>(ba.vr));
  }
  dfloat Zb[4], dZ[3][4];
  split_nodal(Zc, Zb, dZ);
  dfloat out[3][4], r[16];
  int st;
  if (SYNC) {
    TriLin<dfloat> L;
    dfloat S[4], lda[3][4];
    phase_sync(true);
    st = lin_roe(Zb, dZ, nxd, nyd, hld, gas, L);
    phase_sync(true);
    if (!st) lin_split(nxd, nyd, hld, eps, L);
    phase_sync(true);
    if (!st) st = lin_assemble(L);
    phase_sync(true);
    if (!st) lin_wh_sum(dZ, gas, L, S);
    phase_sync(true);
    if (!st) lin_nsolve(L, S);
    phase_sync(true);
    if (!st && SCHEME != RD_N1) lda_apply(L, L.phiT, lda);
    phase_sync(true);
    if (!st) stage1_finish<dfloat, SCHEME>(L, lda, out, r, mode, to_df(thx));
  } else {
    st = stage1_body_d<dfloat, SCHEME>(Zb, dZ, nxd, nyd, hld, gas, eps, out, r, mode, to_df(thx));
  }
  if (!act) return;
  if (st) {
    atomicOr(&ctl->status, st);
    return;
  }
  if (SCHEME != RD_N1) st_rec(rec + (size_t)t * 16, r);
  double* sp = share + (size_t)t * 12;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double o[4] = {from_df(out[i][0]), from_df(out[i][1]), from_df(out[i][2]), from_df(out[i][3])};
    st4(sp + 4 * i, o);
  }
}

template <int SCHEME, int REGS, bool SYNC>
__global__ void __maxnreg__(REGS)
    k_tri_stage2_df(int nt, const int* __restrict__ tri, DevGeoDF g, const double* __restrict__ Zs,
                    const float2* __restrict__ dw, const dfloat* __restrict__ rec, Gas<dfloat> gas, dfloat eps,
                    double* __restrict__ share, DevCtl* ctl, BlendArgs<double> ba,
                    const double* __restrict__ dtm, const uint16_t* __restrict__ tmesh) {
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (SYNC) {
    if (block_stop(ctl)) return;
  } else if (t0 >= nt || ctl->stop) {
    return;
  }
  const bool act = t0 < nt;
  const int t = act ? t0 : nt - 1;
  int v[3];
  double Zc[3][4];
  dfloat nxd[3], nyd[3], hld[3];
  load_tri_df(t, nt, tri, g, v, nxd, nyd, hld);
#pragma unroll
  for (int c = 0; c < 3; ++c) load_vec4(Zs, v[c], Zc[c]);
  const dfloat aread = ld_df(g.area + t);
  const int mode = SCHEME == RD_BMAX2 ? ba.mode : BLEND_B;
  const int sl = (SCHEME == RD_BMAX2 || SCHEME == RD_LDA2) ? ba.sl : 0;
  double thx = 0.0;
  if (SCHEME == RD_BMAX2 && mode == BLEND_X) {
    double nx[3], ny[3], hl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      nx[c] = from_df(nxd[c]);
      ny[c] = from_df(nyd[c]);
      hl[c] = from_df(hld[c]);
    }
    thx = bx_theta(Zc, nx, ny, hl, from_df(aread), ba.L, vrange_of<double>(ba.vr));
  }
  dfloat Zb[4], dZ[3][4];
  split_nodal(Zc, Zb, dZ);
  dfloat out[3][4];
  const dfloat dt = to_df(dtm ? __ldg(dtm + __ldg(tmesh + t)) : ctl->dt);  // batched form: each mesh's dt
  int st;
  if (SYNC) {
    TriLin<dfloat> L;
    dfloat S[4], lda[3][4], PhiN[3][4], PhiT[4];
    const dfloat idt = rcp(dt);
    phase_sync(true);
    st = lin_roe(Zb, dZ, nxd, nyd, hld, gas, L);
    phase_sync(true);
    if (!st) lin_split(nxd, nyd, hld, eps, L);
    phase_sync(true);
    if (!st) st = lin_assemble(L);
    phase_sync(true);
    if (!st) lin_wh_sum(dZ, gas, L, S);
    phase_sync(true);
    if (!st) lin_nsolve(L, S);
    phase_sync(true);
    dfloat dW[3][4];
    if (!st) {
      dfloat r[16];
      ld_dw(dw, v, dW);
      ld_rec(rec + (size_t)t * 16, r);
      stage2_totals_dw(L, dW, r, aread, idt, PhiN, PhiT);
      lda_apply(L, PhiT, lda);
    }
    phase_sync(true);
    if (!st) stage2_finish<dfloat, SCHEME>(PhiN, PhiT, lda, dW, aread, idt, out, mode, to_df(thx), sl);
  } else {
    TriLin<dfloat> L;
    st = linearise_core(Zb, dZ, nxd, nyd, hld, gas, eps, L);
    if (!st) {
      dfloat dW[3][4], r[16], PhiN[3][4], PhiT[4];
      ld_dw(dw, v, dW);
      ld_rec(rec + (size_t)t * 16, r);
      const dfloat idt = rcp(dt);
      stage2_totals_dw(L, dW, r, aread, idt, PhiN, PhiT);
      stage2_shares<dfloat, SCHEME>(L, PhiN, PhiT, dW, aread, idt, out, mode, to_df(thx), sl);
    }
  }
  if (!act) return;
  if (st) {
    atomicOr(&ctl->status, st);
    return;
  }
  double* sp = share + (size_t)t * 12;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double o[4] = {from_df(out[i][0]), from_df(out[i][1]), from_df(out[i][2]), from_df(out[i][3])};
    st4(sp + 4 * i, o);
  }
}

Gas<dfloat> gas_df(double gamma) {
  Gas<dfloat> q;
  q.gamma = dfloat(gamma);
  q.g1 = dfloat(gamma - 1.0);
  q.g = dfloat((gamma - 1.0) / gamma);
  q.ig = dfloat(1.0 / gamma);
  return q;
}

}  // namespace

template <int REGS, bool SYNC>
int df_stage1(const rd_params& p, const TriArraysDF& a, BlendArgs<double> ba, unsigned grid, int block,
                  cudaStream_t st) {
  const Gas<dfloat> gas = gas_df(p.gamma);
  const dfloat eps(p.eps_fix);
  dfloat* rec = (dfloat*)a.rec;
  switch (p.scheme) {
    case RD_N1:
      k_tri_stage1_df<RD_N1, REGS, SYNC><<<grid, block, 0, st>>>(a.nt, a.tri, a.g, a.Z, a.spd, gas, eps, a.share, nullptr,
                                                          a.cfl, a.ctl, ba);
      break;
    case RD_LDA2:
      k_tri_stage1_df<RD_LDA2, REGS, SYNC><<<grid, block, 0, st>>>(a.nt, a.tri, a.g, a.Z, a.spd, gas, eps, a.share, rec,
                                                            a.cfl, a.ctl, ba);
      break;
    default:
      if (p.scheme == RD_B2 && p.lumping == RD_LUMP_GLOBAL)
        k_tri_stage1_df<RD_B2, REGS, SYNC><<<grid, block, 0, st>>>(a.nt, a.tri, a.g, a.Z, a.spd, gas, eps, a.share, rec,
                                                            a.cfl, a.ctl, ba);
      else
        k_tri_stage1_df<RD_BMAX2, REGS, SYNC><<<grid, block, 0, st>>>(a.nt, a.tri, a.g, a.Z, a.spd, gas, eps, a.share, rec,
                                                               a.cfl, a.ctl, ba);
      break;
  }
  CU(cudaGetLastError());
  return RD_OK;
}

template <int REGS, bool SYNC>
int df_stage2(const rd_params& p, const TriArraysDF& a, BlendArgs<double> ba, unsigned grid, int block,
                  cudaStream_t st) {
  const Gas<dfloat> gas = gas_df(p.gamma);
  const dfloat eps(p.eps_fix);
  const dfloat* rec = (const dfloat*)a.rec;
  if (p.scheme == RD_LDA2)
    k_tri_stage2_df<RD_LDA2, REGS, SYNC><<<grid, block, 0, st>>>(a.nt, a.tri, a.g, a.Z, a.dw, rec, gas, eps, a.share,
                                                                a.ctl, ba, a.dtm, a.tmesh);
  else if (p.scheme == RD_B2 && p.lumping == RD_LUMP_GLOBAL)
    k_tri_stage2_df<RD_B2, REGS, SYNC><<<grid, block, 0, st>>>(a.nt, a.tri, a.g, a.Z, a.dw, rec, gas, eps, a.share,
                                                              a.ctl, ba, a.dtm, a.tmesh);
  else
    k_tri_stage2_df<RD_BMAX2, REGS, SYNC><<<grid, block, 0, st>>>(a.nt, a.tri, a.g, a.Z, a.dw, rec, gas, eps,
                                                                 a.share, a.ctl, ba, a.dtm, a.tmesh);
  CU(cudaGetLastError());
  return RD_OK;
}

}  // namespace rd

// Explicit instantiation of one stage's launcher at one register budget and
// barrier setting.
#define RD_DF64_INSTANTIATE(STAGE, REGS, SYNC)                                                     \
  template int rd::df_stage##STAGE<REGS, SYNC>(const rd_params&, const rd::TriArraysDF&,              \
                                               rd::BlendArgs<double>, unsigned, int, cudaStream_t);
