// rd_kernels.cuh -- CUDA kernels of the residual-distribution step (sm_103a).
//
// One B2 step (Sec. 3.4, Eqs. eqRK1/eqRK2) is five kernels plus a one-thread
// commit; N1 (forward Euler, Eq. eqUpdate) is three plus the commit:
//
//   k_tri_stage1    per triangle: Roe linearisation at W^n, phi^T, N / LDA / B
//                   shares (Sec. 3.3), CFL term l_max^T lambda_max^T (Sec. 3.2)
//   k_gather_cfl    per vertex: R1 = sum of shares through the CSR, sigma_i,
//                   block min of 2 V_i / sigma_i, last block -> dt
//   k_update1       per vertex: W* = W^n - dt/V R1 (N1: W^{n+1}); Z(W*), checks
//   k_tri_stage2    per triangle: linearisation at W*, total residuals
//                   Phi^N, Phi^LDA (m^LDA = |T|/3 beta_i), blend
//   k_update2       per vertex: W^{n+1} = W* - dt/V R2, Z and |v|+c for the next step
//   k_commit        one thread: t += dt, steps++, stop test
//
// Arithmetic notes (all algebraically identical to the paper's definitions):
//   * K_i^{+-} v is applied in factored form R_i Lambda_i^{+-} (L_i v) with the
//     closed-form left eigenvectors L = R^{-1} of App. A's right eigenvectors.
//   * N^ = (sum_j K_j^-)^{-1} is never formed: sum_j K_j^- is LU-factorised with
//     partial pivoting and solved for the two right-hand sides the N and LDA
//     schemes need (N^ sum_j K_j^- W^_j and N^ phi^T).
//   * phi^T = sum_i K_i Z_i uses the flux Jacobians dF/dZ, dG/dZ at Zbar
//     applied to sum_i (n_i/2) Z_i (Sec. 3.2, eqRes..eqLinearA).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rd_internal.h"

#define RD_HD __host__ __device__ __forceinline__
#include "rd_dfloat.cuh"

namespace rd {

// Minimum resident 256-thread blocks per SM asked of the triangle kernels.  The
// FP32 kernels are latency bound: stage 1 runs fastest at 24 warps per SM (85
// registers), stage 2, which holds three vertex states per corner, at 16 warps
// (128 registers; 24 warps spill).  The FP64 kernels are bound by the FP64
// pipe and keep their registers.
template <class T, int STAGE>
struct TriOcc {
  static constexpr int value = 1;
};
template <>
struct TriOcc<float, 1> {
  static constexpr int value = 3;
};
template <>
struct TriOcc<float, 2> {
  static constexpr int value = 2;
};

// Constants of the ideal-gas closure, formed once per launch on the host so that
// no thread divides by gamma: gamma, g1 = gamma - 1, g = (gamma - 1) / gamma,
// ig = 1 / gamma.  Host and device divisions are both correctly rounded, so
// the values equal those a thread would compute.
template <class T>
struct Gas {
  T gamma, g1, g, ig;
  static RD_HD Gas of(T gamma) {
    Gas q;
    q.gamma = gamma;
    q.g1 = gamma - T(1);
    q.g = q.g1 / gamma;
    q.ig = T(1) / gamma;
    return q;
  }
};

// Reciprocal used by the triangle kernels.  In double precision on the device:
// the hardware's approximate reciprocal (rcp.approx.ftz.f64) refined by two
// Newton-Raphson steps r <- r + r (1 - x r), each of which squares the
// relative error, which leaves r within an ulp of 1/x at about half the FP64
// pipe cost of the IEEE division.  Arguments outside [2^-1000, 2^1000) in
// magnitude (zero, subnormal, huge, inf, NaN) take the IEEE division.
#ifndef RD_FAST_RCP
#define RD_FAST_RCP 1
#endif
template <class T>
RD_HD T rcp(T x) {
  return T(1) / x;
}
#if defined(__CUDACC__)
// The IEEE division of the rare out-of-range arguments, out of line: inlined,
// the compiler may evaluate it beside the fast path and select.
static __device__ __noinline__ double rcp_ieee(double x) { return 1.0 / x; }
#endif
RD_HD double rcp(double x) {
#if defined(__CUDA_ARCH__) && RD_FAST_RCP
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  if (e > 23 && e < 2023) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double t = fma(-x, r, 1.0);
    r = fma(r, t, r);
    t = fma(-x, r, 1.0);
    return fma(r, t, r);
  }
  return rcp_ieee(x);
#else
  return 1.0 / x;
#endif
}

// Blends of N and LDA (Sec. 3.3.3): diagonal Theta (B), every diagonal entry
// max_k / min_k Theta_kk (Bmax / Bmin), or the scalar shock-sensor theta (Bx).
enum : int { BLEND_B = 0, BLEND_MAX = 1, BLEND_MIN = 2, BLEND_X = 3 };

// Magnitude comparisons through the IEEE-754 bit patterns.  For numbers that
// are not NaN the integer order of |x|'s bit pattern is the numeric order of
// |x|, so in double precision these run on the integer pipe instead of the
// FP64 pipe that the triangle kernels saturate.  Results equal the
// floating-point comparisons for every non-NaN input; other scalar types
// (float, the operation-counting type) use the plain comparisons.
RD_HD long long mag_bits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
#else
  long long b;
  __builtin_memcpy(&b, &x, sizeof b);
  return b & 0x7fffffffffffffffLL;
#endif
}
template <class T>
RD_HD bool mag_less(T a, T b) {  // |a| < |b|
  return fabs(a) < fabs(b);
}
RD_HD bool mag_less(double a, double b) { return mag_bits(a) < mag_bits(b); }
template <class T>
RD_HD bool mag_positive(T a) {  // |a| > 0 (false for NaN)
  return fabs(a) > T(0);
}
RD_HD bool mag_positive(double a) {
  return (unsigned long long)(mag_bits(a) - 1) < 0x7ff0000000000000ULL;
}
template <class T>
RD_HD bool positive(T a) {  // a > 0 (false for NaN)
  return a > T(0);
}
RD_HD bool positive(double a) {
#ifdef __CUDA_ARCH__
  long long b = __double_as_longlong(a);
#else
  long long b;
  __builtin_memcpy(&b, &a, sizeof b);
#endif
  return (unsigned long long)(b - 1) < 0x7ff0000000000000ULL;
}

template <class T>
struct DevGeo {
  const T* nx;    // [3][nt] unit inward normals
  const T* ny;
  const T* hl;    // [3][nt] half edge lengths
  const T* area;  // [nt]
  const T* lmax;  // [nt]
};

template <class T>
struct RoeState {
  T u, v, h, c, q2h, ic2, ic2h, i2c, g1, alpha, g1u, g1v;
};

// Per node i: unit normal, w = u.n, and for K_i^+ ([0]) and K_i^- ([1]) the
// four numbers of the rank-two form below.
template <class T>
struct NodeSys {
  T nx, ny, w;
  T l3[2], s1[2], s2[2], hp[2];
};

// Regularised |lambda|: (lambda^2 + delta^2) / (2 delta) below delta (C^1), i2d = 1 / (2 delta).
template <class T>
RD_HD T abs_reg(T lam, T delta, T i2d) {
  return mag_less(lam, delta) ? (lam * lam + delta * delta) * i2d : fabs(lam);
}
// The three regularised |lambda| of a node that has one below delta (rare).
template <class T>
RD_HD void abs_reg3(const T la[3], T delta, T ab[3]) {
  const T i2d = T(0.5) / delta;
#pragma unroll
  for (int k = 0; k < 3; ++k) ab[k] = abs_reg(la[k], delta, i2d);
}
#if defined(__CUDACC__)
// Out of line on the device, so that the common path carries none of its work;
// scalar arguments and result, so that no array of the caller needs an address.
template <class T>
struct Abs3 {
  T a0, a1, a2;
};
template <class T>
RD_HD Abs3<T> abs_reg3_val(T la0, T la1, T la2, T delta) {
  const T i2d = T(0.5) / delta;
  return Abs3<T>{abs_reg(la0, delta, i2d), abs_reg(la1, delta, i2d), abs_reg(la2, delta, i2d)};
}
template <class T>
__device__ __noinline__ Abs3<T> abs_reg3_dev(T la0, T la1, T la2, T delta) {
  return abs_reg3_val(la0, la1, la2, delta);
}
#endif

// K^{+-} in closed form (App. A).  With the right eigenvectors of App. A,
// e = (1, u, v, h), d = (0, nx, ny, w), the pressure row a = (alpha, -g1 u,
// -g1 v, g1) and the normal-velocity row b = (-w, nx, ny, 0), the two acoustic
// projectors are (e +- c d)(a +- c b)^T / (2 c^2) and the entropy and shear
// projectors sum to I minus them, so for eigenvalues (l1, l2, l3, l3)
//   K = l3 I + e (s1 a + s2 b)^T + d (s2 a + hp b)^T,
//   mu1 = l1 - l3, mu2 = l2 - l3, s1 = (mu1 + mu2) / (2 c^2),
//   s2 = (mu1 - mu2) / (2 c), hp = (mu1 + mu2) / 2.
// PLUS selects Lambda^+ or Lambda^-; o = K^{+-} v.
// Pressure-row product a . v, the node-independent part of K^{+-} v.
template <class T>
RD_HD T pressure_row(const RoeState<T>& r, const T v[4]) {
  return r.alpha * v[0] - r.g1u * v[1] - r.g1v * v[2] + r.g1 * v[3];
}
// o = K^{+-} v given A = a . v (shared when one v meets all three nodes).
template <class T, bool PLUS>
RD_HD void Kpm_apply_a(const RoeState<T>& r, const NodeSys<T>& n, const T v[4], T A, T o[4]) {
  const int j = PLUS ? 0 : 1;
  T B = n.nx * v[1] + n.ny * v[2] - n.w * v[0];
  T P = n.s1[j] * A + n.s2[j] * B;
  T Q = n.s2[j] * A + n.hp[j] * B;
  T l3 = n.l3[j];
  o[0] = l3 * v[0] + P;
  o[1] = l3 * v[1] + r.u * P + n.nx * Q;
  o[2] = l3 * v[2] + r.v * P + n.ny * Q;
  o[3] = l3 * v[3] + r.h * P + n.w * Q;
}
template <class T, bool PLUS>
RD_HD void Kpm_apply(const RoeState<T>& r, const NodeSys<T>& n, const T v[4], T o[4]) {
  Kpm_apply_a<T, PLUS>(r, n, v, pressure_row(r, v), o);
}

// LU factorisation with partial pivoting of a 4x4 matrix held in registers.
template <class T>
struct LU4 {
  T a[4][4];
  T rdiag[4];  // reciprocal pivots
  int piv[3];
  RD_HD bool factor() {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int p = k;
      T best = a[k][k];
#pragma unroll
      for (int r = k + 1; r < 4; ++r) {
        if (mag_less(best, a[r][k])) {
          best = a[r][k];
          p = r;
        }
      }
      if (k < 3) piv[k] = p;
#pragma unroll
      for (int r = k + 1; r < 4; ++r) {
        bool sw = (p == r);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          T x = a[k][c], y = a[r][c];
          a[k][c] = sw ? y : x;
          a[r][c] = sw ? x : y;
        }
      }
      ok = ok && mag_positive(best);
      T inv = rcp(a[k][k]);
      rdiag[k] = inv;
#pragma unroll
      for (int r = k + 1; r < 4; ++r) {
        T f = a[r][k] * inv;
        a[r][k] = f;
#pragma unroll
        for (int c = k + 1; c < 4; ++c) a[r][c] -= f * a[k][c];
      }
    }
    return ok;
  }
  RD_HD void solve(const T b[4], T x[4]) const {
    T y[4] = {b[0], b[1], b[2], b[3]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int r = k + 1; r < 4; ++r) {
        bool sw = (piv[k] == r);
        T s = y[k], t = y[r];
        y[k] = sw ? t : s;
        y[r] = sw ? s : t;
      }
    }
#pragma unroll
    for (int r = 1; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < r; ++c) y[r] -= a[r][c] * y[c];
#pragma unroll
    for (int r = 3; r >= 0; --r) {
#pragma unroll
      for (int c = r + 1; c < 4; ++c) y[r] -= a[r][c] * y[c];
      y[r] = y[r] * rdiag[r];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = y[k];
  }
  // z = A^{-T} b (A = P^T L U): U^T y = b, L^T w = y, z = P^T w.
  RD_HD void solve_t(const T b[4], T z[4]) const {
    T y[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      T s = b[r];
#pragma unroll
      for (int c = 0; c < r; ++c) s -= a[c][r] * y[c];
      y[r] = s * rdiag[r];
    }
#pragma unroll
    for (int r = 3; r >= 0; --r) {
      T s = y[r];
#pragma unroll
      for (int c = r + 1; c < 4; ++c) s -= a[c][r] * z[c];
      z[r] = s;
    }
#pragma unroll
    for (int k = 2; k >= 0; --k) {
#pragma unroll
      for (int r = k + 1; r < 4; ++r) {
        bool sw = (piv[k] == r);
        T p = z[k], q = z[r];
        z[k] = sw ? q : p;
        z[r] = sw ? p : q;
      }
    }
  }
};

// Linearisation of one triangle and its N-scheme shares (Sec. 3.2, 3.3.1).
template <class T>
struct TriLin {
  RoeState<T> r;
  NodeSys<T> nd[3];
  LU4<T> lu;
  T phiT[4];
  T phiN[3][4];
  // intermediates kept for the reverse sweep (dead in the forward kernels)
  T Zb[4], gx[4], gy[4], Wh[3][4], win[4];
};

// Core of the linearisation.  Zb is the nodal mean Zbar; Z are the nodal
// values entering phi^T = dF/dZ(Zbar) sum_i (n_i/2) Z_i + ... and the
// linearised states W^_i = dW/dZ(Zbar) Z_i.  Because sum_i n_i = 0 and the N
// scheme only sees differences W^_i - W^_j, the nodal values may be given
// relative to any common reference: linearise() passes Z_i itself; the
// double-float kernels pass Z_i - Zbar, formed in double precision, so that
// their 48-bit arithmetic acts on the differences (which carry the residual)
// rather than on the full states (App. A algebra unchanged).
template <class T>
RD_HD int lin_roe(const T Zbar[4], const T Z[3][4], const T nx[3], const T ny[3], const T hl[3], const Gas<T>& gas,
                  TriLin<T>& L) {
  T* Zb = L.Zb;
#pragma unroll
  for (int k = 0; k < 4; ++k) Zb[k] = Zbar[k];
  RoeState<T>& r = L.r;
  r.g1 = gas.g1;
  T iz = rcp(Zb[0]);
  r.u = Zb[1] * iz;
  r.v = Zb[2] * iz;
  r.h = Zb[3] * iz;
  r.q2h = (r.u * r.u + r.v * r.v) * T(0.5);
  T c2 = r.g1 * (r.h - r.q2h);
  if (!positive(c2)) return ST_ROE;
  r.c = sqrt(c2);
  r.ic2 = rcp(c2);
  r.ic2h = r.ic2 * T(0.5);
  r.i2c = r.c * r.ic2h;
  r.alpha = r.g1 * r.q2h;
  r.g1u = r.g1 * r.u;
  r.g1v = r.g1 * r.v;

  // phi^T = dF/dZ(Zbar) gx + dG/dZ(Zbar) gy, g = sum_i (n_i / 2) Z_i
  T* gx = L.gx;
  T* gy = L.gy;
#pragma unroll
  for (int k = 0; k < 4; ++k) gx[k] = gy[k] = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T ax = nx[i] * hl[i], ay = ny[i] * hl[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      gx[k] += ax * Z[i][k];
      gy[k] += ay * Z[i][k];
    }
  }
  {
    const T g = gas.g;
    L.phiT[0] = Zb[1] * gx[0] + Zb[0] * gx[1] + Zb[2] * gy[0] + Zb[0] * gy[2];
    L.phiT[1] = g * Zb[3] * gx[0] + (T(2) - g) * Zb[1] * gx[1] - g * Zb[2] * gx[2] + g * Zb[0] * gx[3] +
                Zb[2] * gy[1] + Zb[1] * gy[2];
    L.phiT[2] = Zb[2] * gx[1] + Zb[1] * gx[2] + g * Zb[3] * gy[0] - g * Zb[1] * gy[1] +
                (T(2) - g) * Zb[2] * gy[2] + g * Zb[0] * gy[3];
    L.phiT[3] = Zb[3] * gx[1] + Zb[1] * gx[3] + Zb[3] * gy[2] + Zb[2] * gy[3];
  }

  return 0;
}

// Eigen-split of the three nodes (after lin_roe).
template <class T>
RD_HD void lin_split(const T nx[3], const T ny[3], const T hl[3], T eps, TriLin<T>& L) {
  const RoeState<T>& r = L.r;
  // eigen-split per node (App. A), regularised |lambda| below delta
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    NodeSys<T>& n = L.nd[i];
    n.nx = nx[i];
    n.ny = ny[i];
    n.w = r.u * n.nx + r.v * n.ny;
    T delta = eps * r.c * hl[i];
    T la[3] = {(n.w + r.c) * hl[i], (n.w - r.c) * hl[i], n.w * hl[i]};
    T ab[3];
    if (mag_less(la[0], delta) || mag_less(la[1], delta) || mag_less(la[2], delta)) {
#ifdef __CUDA_ARCH__
      const Abs3<T> a = abs_reg3_dev(la[0], la[1], la[2], delta);
      ab[0] = a.a0;
      ab[1] = a.a1;
      ab[2] = a.a2;
#else
      abs_reg3(la, delta, ab);
#endif
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) ab[k] = fabs(la[k]);
    }
    // Lambda^{+-} = (la +- |la|) / 2, mu_k = l_k - l_3.  Since la_1 + la_2 = 2 la_3
    // and la_1 - la_2 = 2 c hl:  mu_1 + mu_2 = +-X,  mu_1 - mu_2 = c hl +- Y with
    // X = (|la_1| + |la_2|) / 2 - |la_3|, Y = (|la_1| - |la_2|) / 2, and
    // (c hl) i2c = hl / 2 (i2c = 1 / 2c).
    const T X = T(0.5) * (ab[0] + ab[1]) - ab[2];
    const T Yi = (T(0.5) * (ab[0] - ab[1])) * r.i2c;
    const T s1 = X * r.ic2h, hp = X * T(0.5), q2 = T(0.5) * hl[i];
    const T l3m = T(0.5) * la[2], l3a = T(0.5) * ab[2];
    n.l3[0] = l3m + l3a;
    n.l3[1] = l3m - l3a;
    n.s1[0] = s1;
    n.s1[1] = -s1;
    n.hp[0] = hp;
    n.hp[1] = -hp;
    n.s2[0] = q2 + Yi;
    n.s2[1] = q2 - Yi;
  }

}

template <class T>
RD_HD int lin_roe_split(const T Zbar[4], const T Z[3][4], const T nx[3], const T ny[3], const T hl[3],
                        const Gas<T>& gas, T eps, TriLin<T>& L) {
  const int st = lin_roe(Zbar, Z, nx, ny, hl, gas, L);
  if (st) return st;
  lin_split(nx, ny, hl, eps, L);
  return 0;
}

// Phase 2 of the linearisation: sum_j K_j^- assembled and LU-factorised.
template <class T>
RD_HD int lin_assemble(TriLin<T>& L) {
  const RoeState<T>& r = L.r;
  // sum_j K_j^- = (sum l3) I + e P^T + sum_j d_j q_j^T,
  //   P = (sum s1) a + sum_j s2_j b_j,  q_j = s2_j a + hp_j b_j.
  // With d_j = (0, nx, ny, w)_j and b_j = (-w, nx, ny, 0)_j the rows
  // M_x = sum_j nx_j q_j (and M_y, M_w) need only the moments
  // P_x = sum s2 nx, ..., S_xy = sum hp nx ny, ...:
  //   M_x = P_x a + (-S_xw, S_xx, S_xy, 0), M_y = P_y a + (-S_yw, S_xy, S_yy, 0),
  //   M_w = P_w a + (-S_ww, S_xw, S_yw, 0).
  {
    T L3 = T(0), S1 = T(0), Pw = T(0), Px = T(0), Py = T(0);
    T Sxx = T(0), Sxy = T(0), Syy = T(0), Sxw = T(0), Syw = T(0), Sww = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const NodeSys<T>& n = L.nd[j];
      L3 += n.l3[1];
      S1 += n.s1[1];
      Pw += n.s2[1] * n.w;
      Px += n.s2[1] * n.nx;
      Py += n.s2[1] * n.ny;
      const T hx = n.hp[1] * n.nx, hy = n.hp[1] * n.ny, hw = n.hp[1] * n.w;
      Sxx += hx * n.nx;
      Sxy += hx * n.ny;
      Syy += hy * n.ny;
      Sxw += hx * n.w;
      Syw += hy * n.w;
      Sww += hw * n.w;
    }
    const T M1[4] = {Px * r.alpha - Sxw, Sxx - Px * r.g1u, Sxy - Px * r.g1v, Px * r.g1};
    const T M2[4] = {Py * r.alpha - Syw, Sxy - Py * r.g1u, Syy - Py * r.g1v, Py * r.g1};
    const T M3[4] = {Pw * r.alpha - Sww, Sxw - Pw * r.g1u, Syw - Pw * r.g1v, Pw * r.g1};
    T P[4] = {S1 * r.alpha - Pw, Px - S1 * r.g1u, Py - S1 * r.g1v, S1 * r.g1};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      L.lu.a[0][c] = P[c];
      L.lu.a[1][c] = r.u * P[c] + M1[c];
      L.lu.a[2][c] = r.v * P[c] + M2[c];
      L.lu.a[3][c] = r.h * P[c] + M3[c];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) L.lu.a[k][k] += L3;
  }
  return L.lu.factor() ? 0 : ST_SINGULAR;
}

// Phase 3: linearised states, N^ sum_j K_j^- W^_j and the N-scheme shares.
template <class T>
RD_HD void lin_wh_sum(const T Z[3][4], const Gas<T>& gas, TriLin<T>& L, T S[4]) {
  const RoeState<T>& r = L.r;
  const T* Zb = L.Zb;

  // conservative linearised states W^_i = dW/dZ(Zbar) Z_i and
  // S = sum_j K_j^- W^_j = sum_j l3_j W^_j + e sum_j P_j + sum_j d_j Q_j
  // (P_j = s1 A + s2 B, Q_j = s2 A + hp B, A = a . W^_j, B = b_j . W^_j)
  T (*Wh)[4] = L.Wh;
#pragma unroll
  for (int k = 0; k < 4; ++k) S[k] = T(0);
  {
    const T g = gas.g, ig = gas.ig;
    T SP = T(0), SQx = T(0), SQy = T(0), SQw = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Wh[i][0] = T(2) * Zb[0] * Z[i][0];
      Wh[i][1] = Zb[1] * Z[i][0] + Zb[0] * Z[i][1];
      Wh[i][2] = Zb[2] * Z[i][0] + Zb[0] * Z[i][2];
      Wh[i][3] = (Zb[3] * Z[i][0] + Zb[0] * Z[i][3]) * ig + g * (Zb[1] * Z[i][1] + Zb[2] * Z[i][2]);
      const NodeSys<T>& n = L.nd[i];
      const T A = pressure_row(r, Wh[i]);
      const T B = n.nx * Wh[i][1] + n.ny * Wh[i][2] - n.w * Wh[i][0];
      const T Pj = n.s1[1] * A + n.s2[1] * B;
      const T Qj = n.s2[1] * A + n.hp[1] * B;
#pragma unroll
      for (int k = 0; k < 4; ++k) S[k] += n.l3[1] * Wh[i][k];
      SP += Pj;
      SQx += n.nx * Qj;
      SQy += n.ny * Qj;
      SQw += n.w * Qj;
    }
    S[0] += SP;
    S[1] += r.u * SP + SQx;
    S[2] += r.v * SP + SQy;
    S[3] += r.h * SP + SQw;
  }
}

// N-scheme shares from S = sum_j K_j^- W^_j (after lin_wh_sum).
template <class T>
RD_HD void lin_nsolve(TriLin<T>& L, const T S[4]) {
  const RoeState<T>& r = L.r;
  T (*Wh)[4] = L.Wh;
  // N scheme: phi_i^N = K_i^+ (W^_i - N^ sum_j K_j^- W^_j)
  T* win = L.win;
  L.lu.solve(S, win);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T d[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = Wh[i][k] - win[k];
    Kpm_apply<T, true>(r, L.nd[i], d, L.phiN[i]);
  }
}

template <class T>
RD_HD void lin_nshares(const T Z[3][4], const Gas<T>& gas, TriLin<T>& L) {
  T S[4];
  lin_wh_sum(Z, gas, L, S);
  lin_nsolve(L, S);
}

// The linearisation in its three phases (the double-float kernels may place a
// block barrier between them so that the warps of a block fetch the long
// straight-line code together).
template <class T>
RD_HD int linearise_core(const T Zbar[4], const T Z[3][4], const T nx[3], const T ny[3], const T hl[3],
                         const Gas<T>& gas, T eps, TriLin<T>& L) {
  int st = lin_roe_split(Zbar, Z, nx, ny, hl, gas, eps, L);
  if (st) return st;
  st = lin_assemble(L);
  if (st) return st;
  lin_nshares(Z, gas, L);
  return 0;
}

template <class T>
RD_HD int linearise(const T Z[3][4], const T nx[3], const T ny[3], const T hl[3],
                    const Gas<T>& gas, T eps, TriLin<T>& L) {
  const T third = T(1) / T(3);
  T Zb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) Zb[k] = (Z[0][k] + Z[1][k] + Z[2][k]) * third;
  return linearise_core(Zb, Z, nx, ny, hl, gas, eps, L);
}

template <class T>
RD_HD int linearise(const T Z[3][4], const T nx[3], const T ny[3], const T hl[3], T gamma, T eps, TriLin<T>& L) {
  return linearise(Z, nx, ny, hl, Gas<T>::of(gamma), eps, L);
}

// beta_i x = -K_i^+ N^ x for the three nodes (Sec. 3.3.2).
template <class T>
RD_HD void lda_apply(const TriLin<T>& L, const T x[4], T out[3][4]) {
  T y[4];
  L.lu.solve(x, y);
  const T A = pressure_row(L.r, y);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T o[4];
    Kpm_apply_a<T, true>(L.r, L.nd[i], y, A, o);
#pragma unroll
    for (int k = 0; k < 4; ++k) out[i][k] = -o[k];
  }
}

// Theta_kk = |tot_k| / max(sum_i |N_ik|, |tot_k|) (0/0 -> 0); out = Theta N + (1-Theta) LDA,
// evaluated as LDA + Theta (N - LDA).
template <class T>
RD_HD void blend(const T tot[4], const T N[3][4], const T lda[3][4], T out[3][4], int mode = BLEND_B,
                 T theta_x = T(0)) {
  T th[4];
  if (mode == BLEND_X) {
#pragma unroll
    for (int k = 0; k < 4; ++k) th[k] = theta_x;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T num = fabs(tot[k]);
      T den = fabs(N[0][k]) + fabs(N[1][k]) + fabs(N[2][k]);
      den = mag_less(num, den) ? den : num;
      th[k] = mag_positive(den) ? num * rcp(den) : T(0);
    }
    if (mode == BLEND_MAX || mode == BLEND_MIN) {
      // Bmax / Bmin: one weight, the largest or smallest Theta_kk (all >= 0)
      T e = th[0];
#pragma unroll
      for (int k = 1; k < 4; ++k) {
        bool take = mode == BLEND_MAX ? mag_less(e, th[k]) : mag_less(th[k], e);
        e = take ? th[k] : e;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) th[k] = e;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) out[i][k] = lda[i][k] + th[k] * (N[i][k] - lda[i][k]);
}

// Shock sensor of the Bx blend (Sec. 3.3.3): theta = min(1, s^2 h_T / L),
// s = max(0, -L div v / vrange), div v of the linear interpolant of the vertex
// velocities u_c = Z_c1 / Z_c0, v_c = Z_c2 / Z_c0 (grad phi_c = n_c |e_c| / (2 |T|)
// with unit inward normals n_c and |e_c| = 2 hl_c), h_T = sqrt(2 |T|).
template <class T>
RD_HD T bx_theta(const T Z[3][4], const T nx[3], const T ny[3], const T hl[3], T area, T L, T vrange) {
  if (!positive(vrange)) return T(0);
  T div = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T iz = T(1) / Z[c][0];
    div += (Z[c][1] * iz * nx[c] + Z[c][2] * iz * ny[c]) * hl[c];
  }
  T s = -L * (div / area) / vrange;
  if (!positive(s)) return T(0);
  T th = s * s * sqrt(T(2) * area) / L;
  return mag_less(th, T(1)) ? th : T(1);
}

// Run-time blend configuration of the two-stage triangle kernels.
template <class T>
struct BlendArgs {
  int mode = BLEND_B;                      // BLEND_B | BLEND_MAX | BLEND_MIN | BLEND_X
  int sl = 0;                              // stage 2: selective lumping
  T L = T(1);                              // domain size max(Lx, Ly) (Bx)
  const unsigned long long* vr = nullptr;  // Bx: bits of |v|_max, |v|_min of the distributed state
};
template <class T>
__device__ __forceinline__ T vrange_of(const unsigned long long* vr) {
  return (T)(__longlong_as_double((long long)vr[0]) - __longlong_as_double((long long)vr[1]));
}

template <class T>
__device__ __forceinline__ void load_tri(int t, int nt, const int* __restrict__ tri, const DevGeo<T>& g,
                                         int v[3], T nx[3], T ny[3], T hl[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v[c] = __ldg(tri + (size_t)c * nt + t);
    nx[c] = __ldg(g.nx + (size_t)c * nt + t);
    ny[c] = __ldg(g.ny + (size_t)c * nt + t);
    hl[c] = __ldg(g.hl + (size_t)c * nt + t);
  }
}

// Vertex arrays are records of four components ([nv][4]): one 16-byte load
// (float) or two (double) per vertex.
__device__ __forceinline__ void ld4(const float* __restrict__ p, float out[4]) {
  float4 a = __ldg(reinterpret_cast<const float4*>(p));
  out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
}
__device__ __forceinline__ void ld4(const double* __restrict__ p, double out[4]) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
template <class T>
__device__ __forceinline__ void load_vec4(const T* __restrict__ A, int i, T out[4]) {
  ld4(A + 4 * (size_t)i, out);
}

// ---------------------------------------------------------------------------
// Per-triangle bodies (host+device: the same code is instantiated on a
// counting scalar type to count the kernels' floating-point operations).
// ---------------------------------------------------------------------------

// Stage 1 (and forward Euler) shares at W^n.  SCHEME: RD_N1 -> phi^N,
// RD_LDA2 -> phi^LDA, RD_B2 -> phi^B (Sec. 3.3).  rec (two-stage schemes):
// phi^N_0..2 and phi^T at W^n, reused by stage 2.  Returns an ST_* status.
template <class T, int SCHEME>
RD_HD void stage1_shares(const TriLin<T>& L, T out[3][4], T rec[16], int bmode, T theta_x);

template <class T, int SCHEME>
RD_HD int stage1_body(const T Z[3][4], const T nx[3], const T ny[3], const T hl[3], const Gas<T>& gas, T eps,
                      T out[3][4], T rec[16], int bmode = BLEND_B, T theta_x = T(0)) {
  TriLin<T> L;
  int st = linearise(Z, nx, ny, hl, gas, eps, L);
  if (st) return st;
  stage1_shares<T, SCHEME>(L, out, rec, bmode, theta_x);
  return 0;
}

// Stage-1 shares from a linearisation given as Zbar and the nodal differences
// dZ_i = Z_i - Zbar (the double-float kernels).
template <class T, int SCHEME>
RD_HD int stage1_body_d(const T Zb[4], const T dZ[3][4], const T nx[3], const T ny[3], const T hl[3],
                        const Gas<T>& gas, T eps, T out[3][4], T rec[16], int bmode = BLEND_B, T theta_x = T(0)) {
  TriLin<T> L;
  int st = linearise_core(Zb, dZ, nx, ny, hl, gas, eps, L);
  if (st) return st;
  stage1_shares<T, SCHEME>(L, out, rec, bmode, theta_x);
  return 0;
}

template <class T, int SCHEME>
RD_HD void stage1_finish(const TriLin<T>& L, const T lda[3][4], T out[3][4], T rec[16], int bmode, T theta_x) {
  if (SCHEME == RD_N1) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) out[i][k] = L.phiN[i][k];
    return;
  }
  if (SCHEME == RD_LDA2) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) out[i][k] = lda[i][k];
  } else {
    blend(L.phiT, L.phiN, lda, out, bmode, theta_x);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) rec[4 * i + k] = L.phiN[i][k];
#pragma unroll
  for (int k = 0; k < 4; ++k) rec[12 + k] = L.phiT[k];
}

// Stage-1 shares from a linearisation: LDA distribution of phi^T (two-stage
// schemes), then the scheme's shares and the stage-2 record.
template <class T, int SCHEME>
RD_HD void stage1_shares(const TriLin<T>& L, T out[3][4], T rec[16], int bmode, T theta_x) {
  T lda[3][4];
  if (SCHEME != RD_N1) lda_apply(L, L.phiT, lda);
  stage1_finish<T, SCHEME>(L, lda, out, rec, bmode, theta_x);
}

// Stage 2 (Sec. 3.4): total residuals at (W^n, W*).
//   Phi^N_i   = |T|/3 (W*_i - W^n_i)/dt + (phi^N_i(W*) + phi^N_i(W^n)) / 2
//   Phi^T     = sum_j |T|/3 (W*_j - W^n_j)/dt + (phi^T(W^n) + phi^T(W*)) / 2
//   Phi^LDA_i = beta_i(W*) Phi^T     (m^LDA_ij = |T|/3 beta_i, global lumping)
//   Phi_i     = Theta Phi^N_i + (I - Theta) Phi^LDA_i, Theta from (Phi^T, Phi^N)
// Total residuals of stage 2 from the W* linearisation L, the stage-1 record
// and the mass term (m = |T|/3 (W* - W^n) / dt).
// dW[i][k] = W*_i - W^n_i (formed by the caller; the double-float kernels form it
// in double precision).
template <class T>
RD_HD void stage2_totals_dw(const TriLin<T>& L, const T dW[3][4], const T rec[16], T area, T idt, T PhiN[3][4],
                            T PhiT[4]) {
  const T q = area * (T(1) / T(3)) * idt;
#pragma unroll
  for (int k = 0; k < 4; ++k) PhiT[k] = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T m = dW[i][k] * q;
      PhiN[i][k] = m + (L.phiN[i][k] + rec[4 * i + k]) * T(0.5);
      PhiT[k] += m;
    }
#pragma unroll
  for (int k = 0; k < 4; ++k) PhiT[k] += (rec[12 + k] + L.phiT[k]) * T(0.5);
}

template <class T>
RD_HD void stage2_totals(const TriLin<T>& L, const T Wn[3][4], const T Ws[3][4], const T rec[16], T area, T idt,
                         T PhiN[3][4], T PhiT[4]) {
  const T q = area * (T(1) / T(3)) * idt;
#pragma unroll
  for (int k = 0; k < 4; ++k) PhiT[k] = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T m = (Ws[i][k] - Wn[i][k]) * q;
      PhiN[i][k] = m + (L.phiN[i][k] + rec[4 * i + k]) * T(0.5);
      PhiT[k] += m;
    }
#pragma unroll
  for (int k = 0; k < 4; ++k) PhiT[k] += (rec[12 + k] + L.phiT[k]) * T(0.5);
}

template <class T, int SCHEME>
RD_HD void stage2_shares(const TriLin<T>& L, const T PhiN[3][4], const T PhiT[4], const T dW[3][4], T area, T idt,
                         T out[3][4], int bmode, T theta_x, int sl);

template <class T, int SCHEME>
RD_HD int stage2_body(const T Zs[3][4], const T Wn[3][4], const T Ws[3][4], const T rec[16], const T nx[3],
                      const T ny[3], const T hl[3], T area, T dt, const Gas<T>& gas, T eps, T out[3][4],
                      int bmode = BLEND_B, T theta_x = T(0), int sl = 0) {
  TriLin<T> L;
  int st = linearise(Zs, nx, ny, hl, gas, eps, L);
  if (st) return st;
  T idt = rcp(dt);
  T PhiN[3][4], PhiT[4];
  stage2_totals(L, Wn, Ws, rec, area, idt, PhiN, PhiT);
  T dW[3][4];
  if (sl) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) dW[i][k] = Ws[i][k] - Wn[i][k];
  }
  stage2_shares<T, SCHEME>(L, PhiN, PhiT, dW, area, idt, out, bmode, theta_x, sl);
  return 0;
}

// Stage-2 shares from the W* linearisation given as Zbar* and dZ*_i = Z*_i - Zbar*,
// and dW_i = W*_i - W^n_i (the double-float kernels).
template <class T, int SCHEME>
RD_HD int stage2_body_d(const T Zbs[4], const T dZs[3][4], const T dW[3][4], const T rec[16], const T nx[3],
                        const T ny[3], const T hl[3], T area, T dt, const Gas<T>& gas, T eps, T out[3][4],
                        int bmode = BLEND_B, T theta_x = T(0), int sl = 0) {
  TriLin<T> L;
  int st = linearise_core(Zbs, dZs, nx, ny, hl, gas, eps, L);
  if (st) return st;
  T idt = rcp(dt);
  T PhiN[3][4], PhiT[4];
  stage2_totals_dw(L, dW, rec, area, idt, PhiN, PhiT);
  stage2_shares<T, SCHEME>(L, PhiN, PhiT, dW, area, idt, out, bmode, theta_x, sl);
  return 0;
}

template <class T, int SCHEME>
RD_HD void stage2_finish(const T PhiN[3][4], const T PhiT[4], const T lda[3][4], const T dW[3][4], T area, T idt,
                         T out[3][4], int bmode, T theta_x, int sl) {
  if (SCHEME == RD_LDA2) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) out[i][k] = lda[i][k];
  } else {
    blend(PhiT, PhiN, lda, out, bmode, theta_x);
  }
  if (sl) {
    // selective lumping: + sum_j (|T| delta_ij / 3 - |T| (delta_ij + 1) / 12) (W*_j - W^n_j) / dt
    //                    = |T| / 4 dW_i / dt - |T| / 12 sum_j dW_j / dt
    const T q = area * T(0.25) * idt, tw = area * (T(1) / T(12)) * idt;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T d0 = dW[0][k], d1 = dW[1][k], d2 = dW[2][k];
      T sum = tw * (d0 + d1 + d2);
      out[0][k] += q * d0 - sum;
      out[1][k] += q * d1 - sum;
      out[2][k] += q * d2 - sum;
    }
  }
}

template <class T, int SCHEME>
RD_HD void stage2_shares(const TriLin<T>& L, const T PhiN[3][4], const T PhiT[4], const T dW[3][4], T area, T idt,
                         T out[3][4], int bmode, T theta_x, int sl) {
  T lda[3][4];
  lda_apply(L, PhiT, lda);
  stage2_finish<T, SCHEME>(PhiN, PhiT, lda, dW, area, idt, out, bmode, theta_x, sl);
}

template <class T, int SCHEME>
RD_HD int stage1_body(const T Z[3][4], const T nx[3], const T ny[3], const T hl[3], T gamma, T eps, T out[3][4],
                      T rec[16]) {
  return stage1_body<T, SCHEME>(Z, nx, ny, hl, Gas<T>::of(gamma), eps, out, rec);
}
template <class T, int SCHEME>
RD_HD int stage2_body(const T Zs[3][4], const T Wn[3][4], const T Ws[3][4], const T rec[16], const T nx[3],
                      const T ny[3], const T hl[3], T area, T dt, T gamma, T eps, T out[3][4]) {
  return stage2_body<T, SCHEME>(Zs, Wn, Ws, rec, nx, ny, hl, area, dt, Gas<T>::of(gamma), eps, out);
}

// ---------------------------------------------------------------------------
// Stage-1 triangle kernel: share [nt][3][4]; rec [nt][16] (two-stage only);
// cfl [nt] = l_max^T max_j (|v_j| + c_j).
// ---------------------------------------------------------------------------
template <class T, int SCHEME>
__global__ void __launch_bounds__(256, (TriOcc<T, 1>::value)) k_tri_stage1(int nt, int nv, const int* __restrict__ tri, DevGeo<T> g,
                                                    const T* __restrict__ Z, const T* __restrict__ spd,
                                                    Gas<T> gas, T eps, T* __restrict__ share,
                                                    T* __restrict__ rec, T* __restrict__ cfl, DevCtl* ctl,
                                                    BlendArgs<T> ba = BlendArgs<T>()) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt || ctl->stop) return;
  int v[3];
  T nx[3], ny[3], hl[3], Zc[3][4];
  load_tri(t, nt, tri, g, v, nx, ny, hl);
#pragma unroll
  for (int c = 0; c < 3; ++c) load_vec4(Z, v[c], Zc[c]);
  {
    T s0 = __ldg(spd + v[0]), s1 = __ldg(spd + v[1]), s2 = __ldg(spd + v[2]);
    T lam = mag_less(s1, s0) ? s0 : s1;  // speeds are >= 0
    lam = mag_less(s2, lam) ? lam : s2;
    cfl[t] = __ldg(g.lmax + t) * lam;
  }
  T out[3][4], r[16];
  // SCHEME == RD_BMAX2 is the generic blend instantiation (Bmax, Bmin, Bx and
  // B with selective lumping, chosen at run time); RD_B2 is the plain B scheme.
  const int mode = SCHEME == RD_BMAX2 ? ba.mode : BLEND_B;
  T thx = T(0);
  if (SCHEME == RD_BMAX2 && mode == BLEND_X)
    thx = bx_theta(Zc, nx, ny, hl, __ldg(g.area + t), ba.L, vrange_of<T>(ba.vr));
  int st = stage1_body<T, SCHEME>(Zc, nx, ny, hl, gas, eps, out, r, mode, thx);
  if (st) {
    atomicOr(&ctl->status, st);
    return;
  }
  if (SCHEME != RD_N1) {
    T* rp = rec + (size_t)t * 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) st4(rp + 4 * k, r + 4 * k);
  }
  T* sp = share + (size_t)t * 12;
#pragma unroll
  for (int i = 0; i < 3; ++i) st4(sp + 4 * i, out[i]);
}

// Inspection variant: phi^N, phi^LDA, phi^B (each [nt][3][4]) and the CFL term.
template <class T>
__global__ void __launch_bounds__(256) k_tri_terms(int nt, int nv, const int* __restrict__ tri, DevGeo<T> g,
                                                   const T* __restrict__ Z, const T* __restrict__ spd,
                                                   T gamma, T eps, T* __restrict__ out, T* __restrict__ cfl,
                                                   DevCtl* ctl) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int v[3];
  T nx[3], ny[3], hl[3], Zc[3][4];
  load_tri(t, nt, tri, g, v, nx, ny, hl);
#pragma unroll
  for (int c = 0; c < 3; ++c) load_vec4(Z, v[c], Zc[c]);
  T s0 = spd[v[0]], s1 = spd[v[1]], s2 = spd[v[2]];
  T lam = s0 > s1 ? s0 : s1;
  lam = lam > s2 ? lam : s2;
  cfl[t] = g.lmax[t] * lam;
  TriLin<T> L;
  int st = linearise(Zc, nx, ny, hl, gamma, eps, L);
  if (st) {
    atomicOr(&ctl->status, st);
    return;
  }
  T lda[3][4], b[3][4];
  lda_apply(L, L.phiT, lda);
  blend(L.phiT, L.phiN, lda, b);
  size_t s3 = (size_t)nt * 12;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) {
      out[(size_t)t * 12 + 4 * i + k] = L.phiN[i][k];
      out[s3 + (size_t)t * 12 + 4 * i + k] = lda[i][k];
      out[2 * s3 + (size_t)t * 12 + 4 * i + k] = b[i][k];
    }
}

// ---------------------------------------------------------------------------
// Vertex gather of stage-1 shares and the CFL sums; dt by a two-level min.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

// Sum of the corner records of one vertex in CSR order (and, if CFL, of the
// triangles' CFL terms): indices and records of several corners are loaded
// before any is added, so the loads are in flight together; the sums keep
// the sequential CSR order.
template <class T, bool CFL>
__device__ __forceinline__ void gather_corners(int e0, int e1, const int* __restrict__ ent,
                                               const T* __restrict__ share, const T* __restrict__ cfl, T r[4],
                                               T& sig) {
  // 8 corners in flight for 16-byte float records, 2 for 32-byte double records
  constexpr int C = sizeof(T) == 4 ? 8 : 2;
  for (int eb = e0; eb < e1; eb += C) {
    int te[C];
    T q[C][4], c[C];
#pragma unroll
    for (int j = 0; j < C; ++j) te[j] = (eb + j < e1) ? __ldg(ent + eb + j) : -1;
#pragma unroll
    for (int j = 0; j < C; ++j)
      if (te[j] >= 0) {
        ld4(share + (size_t)te[j] * 4, q[j]);
        if (CFL) c[j] = __ldg(cfl + te[j] / 3);
      }
#pragma unroll
    for (int j = 0; j < C; ++j)
      if (te[j] >= 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) r[k] += q[j][k];
        if (CFL) sig += c[j];
      }
  }
}

// Block minimum of v (every thread of the block calls it; blockDim.x a
// multiple of 32, at most 1024); the result is valid in thread 0.
template <class T>
__device__ __forceinline__ T block_min(T v) {
  __shared__ T red_min[32];
  v = warp_min(v);
  if ((threadIdx.x & 31) == 0) red_min[threadIdx.x >> 5] = v;
  __syncthreads();
  T x = T(INFINITY);
  if (threadIdx.x < 32) {
    x = threadIdx.x < (blockDim.x >> 5) ? red_min[threadIdx.x] : T(INFINITY);
    x = warp_min(x);
  }
  return x;
}

// Second level of the dt reduction: each block stores its minimum of
// 2 V_i / sigma_i in partial[slot]; the last of the gridDim.x blocks to finish
// (ticket in the control block) takes the minimum over partial[0, count) and
// sets dt = CFL * min, clipped to t_end.  Every thread of the block calls it.
template <class T>
__device__ __forceinline__ void dt_finish(T ratio, T* __restrict__ partial, int slot, int count, T cflnum,
                                          DevCtl* ctl) {
  __shared__ bool last;
  T x = block_min(ratio);
  if (threadIdx.x == 0) {
    partial[slot] = x;
    __threadfence();
    unsigned int tk = atomicAdd(&ctl->ticket, 1u);
    last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  // last block: min over all block minima
  __threadfence();
  T m = T(INFINITY);
  for (int b = threadIdx.x; b < count; b += blockDim.x) {
    T y = ((volatile T*)partial)[b];
    m = y < m ? y : m;
  }
  __syncthreads();  // red_min of the first block_min is read before it is reused
  m = block_min(m);
  if (threadIdx.x == 0) {
    double dt = (double)(cflnum * m);
    if (ctl->t_end > 0.0) {
      double rem = ctl->t_end - ctl->t;
      if (dt > rem) dt = rem;
      if (!(rem > 0.0)) ctl->stop = 1;  // t_end reached: the rest of this step is a no-op
    }
    ctl->dt = (double)(T)dt;
    ctl->ticket = 0u;
  }
}

template <class T, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_gather_cfl(int nv, const int* __restrict__ ptr, const int* __restrict__ ent,
                                                      const T* __restrict__ share, const T* __restrict__ cfl,
                                                      const T* __restrict__ V, T* __restrict__ R1,
                                                      T* __restrict__ partial, T cflnum, DevCtl* ctl) {
  if (ctl->stop) return;
  int i = blockIdx.x * BLOCK + threadIdx.x;
  T ratio = T(INFINITY);
  if (i < nv) {
    T r[4] = {T(0), T(0), T(0), T(0)};
    T sig = T(0);
    gather_corners<T, true>(__ldg(ptr + i), __ldg(ptr + i + 1), ent, share, cfl, r, sig);
    st4(R1 + 4 * (size_t)i, r);
    ratio = T(2) * __ldg(V + i) / sig;
  }
  dt_finish(ratio, partial, blockIdx.x, gridDim.x, cflnum, ctl);
}

// Vertex state -> parameter vector Z and |v| + c; returns false if non-physical.
// One reciprocal of rho serves the four quotients (u, v, h and p / rho).
template <class T>
RD_HD bool vertex_Z(const T W[4], T gamma, T Z[4], T& spd, T* vmag = nullptr) {
  T rho = W[0];
  if (!positive(rho)) return false;
  const T ir = rcp(rho);
  T u = W[1] * ir, v = W[2] * ir;
  T p = (gamma - T(1)) * (W[3] - T(0.5) * rho * (u * u + v * v));
  if (!positive(p)) return false;
  T h = (W[3] + p) * ir;
  T sr = sqrt(rho);
  Z[0] = sr;
  Z[1] = sr * u;
  Z[2] = sr * v;
  Z[3] = sr * h;
  T q = sqrt(u * u + v * v);
  spd = q + sqrt(gamma * p * ir);
  if (vmag) *vmag = q;
  return true;
}

// Block-wide max and min of the non-negative vertex speeds |v| (Bx sensor),
// folded into vr[0] (max) and vr[1] (min) through their IEEE bit patterns (the
// integer order of non-negative doubles is their numeric order), one pair of
// atomics per block.  Every thread of the block calls it (blockDim a multiple
// of 32, at most 512); has = false contributes nothing.
__device__ __forceinline__ unsigned long long speed_bits(double q) { return (unsigned long long)__double_as_longlong(q); }
__device__ __forceinline__ unsigned long long speed_bits(float q) {
  // float -> double is exact; done here, once per block, off the per-thread path
  return (unsigned long long)__double_as_longlong((double)q);
}
template <class T>
__device__ __forceinline__ void vrange_fold(bool has, T q, unsigned long long* vr) {
  if (sizeof(T) == 4) {
    // reduce the 32-bit patterns (same order argument), widen only the block's result
    unsigned int h32 = has ? __float_as_uint((float)q) : 0u;
    unsigned int l32 = has ? h32 : 0x7f800000u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned int a = __shfl_xor_sync(0xffffffffu, h32, o), b = __shfl_xor_sync(0xffffffffu, l32, o);
      h32 = a > h32 ? a : h32;
      l32 = b < l32 ? b : l32;
    }
    __shared__ unsigned int s32[2][16];
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      s32[0][w] = h32;
      s32[1][w] = l32;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int j = 1; j < nw; ++j) {
        h32 = s32[0][j] > h32 ? s32[0][j] : h32;
        l32 = s32[1][j] < l32 ? s32[1][j] : l32;
      }
      atomicMax(vr, speed_bits(__uint_as_float(h32)));
      atomicMin(vr + 1, speed_bits(__uint_as_float(l32)));
    }
    return;
  }
  unsigned long long hi = has ? speed_bits(q) : 0ull;
  unsigned long long lo = has ? hi : 0x7ff0000000000000ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    hi = h2 > hi ? h2 : hi;
    lo = l2 < lo ? l2 : lo;
  }
  __shared__ unsigned long long sh[2][16];
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][w] = hi;
    sh[1][w] = lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 1; j < nw; ++j) {
      hi = sh[0][j] > hi ? sh[0][j] : hi;
      lo = sh[1][j] < lo ? sh[1][j] : lo;
    }
    atomicMax(vr, hi);
    atomicMin(vr + 1, lo);
  }
}

// Empty |v| range (max = +0, min = +inf) before a pass reduces into vr;
// skipped once the run has stopped, so that the last reduced range stays valid.
static __global__ void k_vr_reset(unsigned long long* vr, const DevCtl* ctl, int force) {
  if (force || !ctl->stop) {
    vr[0] = 0ull;
    vr[1] = 0x7ff0000000000000ull;
  }
}

// Boundary conditions of Sec. 3.5 as seen by the vertex update.
//   Walls: per internal vertex a CSR of wall-edge ends (the other vertex b, the
//   edge's outward unit normal and half length hl); the correction residual
//   hl (alpha f_self + (1 - alpha) f_other) with f = -(rho v_n, rho u v_n,
//   rho v v_n, rho h v_n) is added to R at the pass's state (Win), or, in
//   stage 2 (Wn != nullptr), as half of it at W* plus half at W^n.
//   Ghosts: the final update of a step writes the stored initial state of a
//   ghost vertex instead of its update.
template <class T>
struct WallArgs {
  const int* ptr = nullptr;
  const int* other = nullptr;
  const T* geo = nullptr;
  const T* Wn = nullptr;
  T alpha = T(0.75);
};
template <class T>
struct GhostArgs {
  const int* of = nullptr;
  const T* W = nullptr;
};

template <class T>
RD_HD void wall_flux(const T W[4], T nx, T ny, T gamma, T f[4]) {
  T rho = W[0];
  T u = W[1] / rho, v = W[2] / rho;
  T p = (gamma - T(1)) * (W[3] - T(0.5) * rho * (u * u + v * v));
  T vn = u * nx + v * ny;
  f[0] = -rho * vn;
  f[1] = -W[1] * vn;
  f[2] = -W[2] * vn;
  f[3] = -(W[3] + p) * vn;
}

template <class T>
__device__ __forceinline__ void wall_add(const WallArgs<T>& wa, const T* __restrict__ Ws, int i, T gamma, T weight,
                                         T r[4]) {
  const int e0 = __ldg(wa.ptr + i), e1 = __ldg(wa.ptr + i + 1);
  for (int e = e0; e < e1; ++e) {
    const int o = __ldg(wa.other + e);
    const T nx = __ldg(wa.geo + 3 * (size_t)e), ny = __ldg(wa.geo + 3 * (size_t)e + 1);
    const T hl = __ldg(wa.geo + 3 * (size_t)e + 2);
    T ws[4], wo[4], fs[4], fo[4];
    load_vec4(Ws, i, ws);
    load_vec4(Ws, o, wo);
    wall_flux(ws, nx, ny, gamma, fs);
    wall_flux(wo, nx, ny, gamma, fo);
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] += weight * hl * (wa.alpha * fs[k] + (T(1) - wa.alpha) * fo[k]);
  }
}

// W_out = W_in - dt/V R; Z_out = Z(W_out); spd_out (nullable) = |v| + c.
// If R2 != nullptr, W_in is W* and R = R2 gathered here from share (stage 2).
template <class T>
__global__ void __launch_bounds__(512) k_update(int nv, const T* __restrict__ Win, const T* __restrict__ R,
                                                const int* __restrict__ ptr, const int* __restrict__ ent,
                                                const T* __restrict__ share, const T* __restrict__ V, T gamma,
                                                T* __restrict__ Wout, T* __restrict__ Zout, T* __restrict__ spdout,
                                                DevCtl* ctl, const double* __restrict__ dtm = nullptr,
                                                const uint16_t* __restrict__ vmesh = nullptr,
                                                unsigned long long* __restrict__ vr_out = nullptr,
                                                WallArgs<T> wa = WallArgs<T>(), GhostArgs<T> ga = GhostArgs<T>(),
                                                float2* __restrict__ dw_df = nullptr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = i < nv && !ctl->stop;
  if (!act && !vr_out) return;
  bool has = false;
  T q = T(0);
  if (act) {
  T r[4];
  if (share) {
    r[0] = r[1] = r[2] = r[3] = T(0);
    T unused = T(0);
    gather_corners<T, false>(__ldg(ptr + i), __ldg(ptr + i + 1), ent, share, nullptr, r, unused);
  } else {
    load_vec4(R, i, r);
  }
  if (wa.ptr) {
    if (wa.Wn) {
      wall_add(wa, Win, i, gamma, T(0.5), r);
      wall_add(wa, wa.Wn, i, gamma, T(0.5), r);
    } else {
      wall_add(wa, Win, i, gamma, T(1), r);
    }
  }
  T dt = dtm ? (T)__ldg(dtm + __ldg(vmesh + i)) : (T)ctl->dt;
  T f = dt / __ldg(V + i);
  T W[4], Z[4], spd;
  load_vec4(Win, i, W);
#pragma unroll
  for (int k = 0; k < 4; ++k) W[k] = W[k] - f * r[k];
  if (ga.of) {
    const int gi = __ldg(ga.of + i);
    if (gi >= 0) load_vec4(ga.W, gi, W);
  }
  bool ok = vertex_Z(W, gamma, Z, spd, &q);
  st4(Wout + 4 * (size_t)i, W);
  st4(Zout + 4 * (size_t)i, Z);
  if (spdout) spdout[i] = spd;
  if constexpr (sizeof(T) == 8) {
    if (dw_df) {  // RD_DF64 stage 1: W* - W^n as double-float pairs for the stage-2 triangle kernel
      T w0[4];
      load_vec4(Win, i, w0);
      dfloat d[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) d[k] = dw::to_df(__dsub_rn(W[k], w0[k]));
      float4* o = reinterpret_cast<float4*>(dw_df + 4 * (size_t)i);
      o[0] = make_float4(d[0].hi, d[0].lo, d[1].hi, d[1].lo);
      o[1] = make_float4(d[2].hi, d[2].lo, d[3].hi, d[3].lo);
    }
  }
  if (!ok) {
    atomicOr(&ctl->status, ST_NONPHYS_VERTEX);
    ctl->stop = 1;
  }
  has = ok;
  }
  if (vr_out) vrange_fold(has, q, vr_out);
}

// Initial state of the ghost vertices: Wg[g] = W[ids[g]].
template <class T>
__global__ void k_ghost_capture(int n, const int* __restrict__ ids, const T* __restrict__ W, T* __restrict__ Wg) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  T w[4];
  load_vec4(W, __ldg(ids + g), w);
  st4(Wg + 4 * (size_t)g, w);
}

// Z and |v|+c of a freshly uploaded state.
template <class T>
__global__ void k_prepare(int nv, const T* __restrict__ W, T gamma, T* __restrict__ Z, T* __restrict__ spd,
                          DevCtl* ctl, unsigned long long* __restrict__ vr_out = nullptr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv && !vr_out) return;
  bool has = false;
  T q = T(0);
  if (i < nv) {
    T w[4], z[4], s;
    load_vec4(W, i, w);
    bool ok = vertex_Z(w, gamma, z, s, &q);
    st4(Z + 4 * (size_t)i, z);
    spd[i] = s;
    if (!ok) atomicOr(&ctl->status, ST_NONPHYS_VERTEX);
    has = ok;
  }
  if (vr_out) vrange_fold(has, q, vr_out);
}

// ---------------------------------------------------------------------------
// Stage-2 triangle kernel: total residuals at (W^n, W*) -> share [nt][3][4].
// ---------------------------------------------------------------------------
template <class T, int SCHEME>
__global__ void __launch_bounds__(256, (TriOcc<T, 2>::value)) k_tri_stage2(int nt, int nv, const int* __restrict__ tri, DevGeo<T> g,
                                                    const T* __restrict__ Zs, const T* __restrict__ Wn,
                                                    const T* __restrict__ Ws, const T* __restrict__ rec,
                                                    Gas<T> gas, T eps, T* __restrict__ share, DevCtl* ctl,
                                                    const double* __restrict__ dtm = nullptr,
                                                    const uint16_t* __restrict__ tmesh = nullptr,
                                                    BlendArgs<T> ba = BlendArgs<T>()) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt || ctl->stop) return;
  int v[3];
  T nx[3], ny[3], hl[3], Zc[3][4], wn[3][4], ws[3][4], r[16];
  load_tri(t, nt, tri, g, v, nx, ny, hl);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    load_vec4(Zs, v[c], Zc[c]);
    load_vec4(Wn, v[c], wn[c]);
    load_vec4(Ws, v[c], ws[c]);
  }
  const T* rp = rec + (size_t)t * 16;
#pragma unroll
  for (int k = 0; k < 4; ++k) ld4(rp + 4 * k, r + 4 * k);
  T out[3][4];
  T dt = dtm ? (T)__ldg(dtm + __ldg(tmesh + t)) : (T)ctl->dt;
  const T area = __ldg(g.area + t);
  const int mode = SCHEME == RD_BMAX2 ? ba.mode : BLEND_B;
  const int sl = (SCHEME == RD_BMAX2 || SCHEME == RD_LDA2) ? ba.sl : 0;
  T thx = T(0);
  if (SCHEME == RD_BMAX2 && mode == BLEND_X) thx = bx_theta(Zc, nx, ny, hl, area, ba.L, vrange_of<T>(ba.vr));
  int st = stage2_body<T, SCHEME>(Zc, wn, ws, r, nx, ny, hl, area, dt, gas, eps, out, mode, thx, sl);
  if (st) {
    atomicOr(&ctl->status, st);
    return;
  }
  T* sp = share + (size_t)t * 12;
#pragma unroll
  for (int i = 0; i < 3; ++i) st4(sp + 4 * i, out[i]);
}

// One thread: commit the step if nothing went wrong.
static __global__ void k_commit(DevCtl* ctl) {
  if (ctl->stop) return;
  if (ctl->status) {
    ctl->stop = 1;
    return;
  }
  ctl->t += ctl->dt;
  ctl->steps += 1;
  if (ctl->t_end > 0.0 && ctl->t >= ctl->t_end) ctl->stop = 1;
}

// Conserved totals: per-block partial sums of V_i W_i (fixed order), then a
// one-block pass in block order -> out[4] (double).
template <class T, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_conserved_partial(int nv, const T* __restrict__ W, const T* __restrict__ V,
                                                             double* __restrict__ partial) {
  __shared__ double red[4][BLOCK];
  int i = blockIdx.x * BLOCK + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = i < nv ? (double)V[i] * (double)W[4 * (size_t)i + k] : 0.0;
  __syncthreads();
  for (int s = BLOCK / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) partial[(size_t)blockIdx.x * 4 + k] = red[k][0];
}

static __global__ void k_conserved_final(int nblocks, const double* __restrict__ partial, double* __restrict__ out) {
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * 4 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Standalone CFL time step of a state in caller-owned device memory (Sec. 3.2):
//   dt = cfl * min_i 2 V_i / sum_{T containing i} l_max^T max_{j in T}(|v_j| + c_j)
// Per vertex: walk its CSR corners, recompute |v|+c of the three corners of each
// triangle, sum l_max * lambda_max; block minima to partial[], the last block
// reduces them into dt_out.  Scratch: partial[gridDim.x] and a DtScratchCtl.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T vertex_speed(const T* __restrict__ W, size_t nv, int i, T gamma, bool& ok) {
  T rho = __ldg(W + i), mx = __ldg(W + nv + i), my = __ldg(W + 2 * nv + i), e = __ldg(W + 3 * nv + i);
  T u = mx / rho, v = my / rho;
  T p = (gamma - T(1)) * (e - T(0.5) * rho * (u * u + v * v));
  ok = ok && (rho > T(0)) && (p > T(0));
  return sqrt(u * u + v * v) + sqrt(gamma * p / rho);
}

template <class T, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_cfl_dt(int nv, int nt, const T* __restrict__ W, const int* __restrict__ tri,
                                                  const T* __restrict__ lmax, const T* __restrict__ V,
                                                  const int* __restrict__ ptr, const int* __restrict__ ent, T gamma,
                                                  T cflnum, double* __restrict__ partial, DtScratchCtl* ctl,
                                                  double* __restrict__ dt_out) {
  __shared__ double red[BLOCK / 32];
  __shared__ bool last;
  int i = blockIdx.x * BLOCK + threadIdx.x;
  double ratio = INFINITY;
  bool ok = true;
  if (i < nv) {
    T sig = T(0);
    int e0 = __ldg(ptr + i), e1 = __ldg(ptr + i + 1);
    for (int e = e0; e < e1; ++e) {
      int t = __ldg(ent + e) / 3;
      T s0 = vertex_speed(W, (size_t)nv, __ldg(tri + t), gamma, ok);
      T s1 = vertex_speed(W, (size_t)nv, __ldg(tri + (size_t)nt + t), gamma, ok);
      T s2 = vertex_speed(W, (size_t)nv, __ldg(tri + 2 * (size_t)nt + t), gamma, ok);
      T lam = s0 > s1 ? s0 : s1;
      lam = lam > s2 ? lam : s2;
      sig += __ldg(lmax + t) * lam;
    }
    ratio = (double)(T(2) * __ldg(V + i) / sig);
  }
  if (!ok) atomicOr(&ctl->status, ST_NONPHYS_VERTEX);
  ratio = warp_min(ratio);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ratio;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < BLOCK / 32 ? red[threadIdx.x] : INFINITY;
    x = warp_min(x);
    if (threadIdx.x == 0) {
      partial[blockIdx.x] = x;
      __threadfence();
      unsigned int tk = atomicAdd(&ctl->ticket, 1u);
      last = (tk == gridDim.x - 1);
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double m = INFINITY;
  for (int b = threadIdx.x; b < gridDim.x; b += BLOCK) {
    double x = ((volatile double*)partial)[b];
    m = x < m ? x : m;
  }
  m = warp_min(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < BLOCK / 32 ? red[threadIdx.x] : INFINITY;
    x = warp_min(x);
    if (threadIdx.x == 0) {
      dt_out[0] = (double)(cflnum * (T)x);
      ctl->ticket = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// Batched form: many independent meshes concatenated into one vertex / triangle
// range, each with its own dt.  vmesh[i] is the mesh of vertex i.
// ---------------------------------------------------------------------------

// Gather of stage-1 shares (as k_gather_cfl) with a per-mesh min of 2 V_i / sigma_i:
// positive doubles order like their bit patterns, so the min is an atomicMin on
// the bits (exact and order-independent, hence deterministic).
template <class T>
__global__ void __launch_bounds__(512) k_gather_cfl_batch(int nv, const int* __restrict__ ptr,
                                                          const int* __restrict__ ent, const T* __restrict__ share,
                                                          const T* __restrict__ cfl, const T* __restrict__ V,
                                                          const uint16_t* __restrict__ vmesh, T* __restrict__ R1,
                                                          unsigned long long* __restrict__ mesh_min, DevCtl* ctl) {
  if (ctl->stop) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool act = i < nv;
  double ratio = INFINITY;
  int m = act ? (int)__ldg(vmesh + i) : -1;
  if (act) {
    T r[4] = {T(0), T(0), T(0), T(0)};
    T sig = T(0);
    int e0 = __ldg(ptr + i), e1 = __ldg(ptr + i + 1);
    for (int e = e0; e < e1; ++e) {
      int te = __ldg(ent + e);
      T q[4];
      ld4(share + (size_t)te * 4, q);
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] += q[k];
      sig += __ldg(cfl + te / 3);
    }
    st4(R1 + 4 * (size_t)i, r);
    ratio = (double)(T(2) * __ldg(V + i) / sig);
  }
  // one atomic per warp when the warp lies inside one mesh (the common case)
  int m0 = __shfl_sync(0xffffffffu, m, 0);
  bool uniform = __all_sync(0xffffffffu, m == m0 || m < 0);
  if (uniform) {
    double x = warp_min(ratio);
    if ((threadIdx.x & 31) == 0 && m0 >= 0) atomicMin(mesh_min + m0, (unsigned long long)__double_as_longlong(x));
  } else if (act) {
    atomicMin(mesh_min + m, (unsigned long long)__double_as_longlong(ratio));
  }
}

// dt of every mesh from its min, then reset the mins for the next step.
static __global__ void k_batch_dt(int n_mesh, double cflnum, unsigned long long* __restrict__ mesh_min,
                                  double* __restrict__ dtm, DevCtl* ctl) {
  if (ctl->stop) return;
  for (int m = threadIdx.x; m < n_mesh; m += blockDim.x) {
    double x = __longlong_as_double((long long)mesh_min[m]);
    dtm[m] = cflnum * x;
    mesh_min[m] = (unsigned long long)__double_as_longlong((double)INFINITY);
  }
}

// Per mesh: t += dt, steps++ (only if the step raised no error).
static __global__ void k_commit_batch(int n_mesh, const double* __restrict__ dtm, double* __restrict__ tm,
                                      long long* __restrict__ stepsm, DevCtl* ctl) {
  if (ctl->stop) return;
  if (ctl->status) {
    if (threadIdx.x == 0) ctl->stop = 1;
    return;
  }
  for (int m = threadIdx.x; m < n_mesh; m += blockDim.x) {
    tm[m] += dtm[m];
    stepsm[m] += 1;
  }
  if (threadIdx.x == 0) ctl->steps += 1;
}

// Caller-order double state -> internal-order T state (and back).
template <class T>
__global__ void k_permute_in(int nv, const int* __restrict__ vperm, const double* __restrict__ src,
                             T* __restrict__ dst, DevCtl* ctl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  int j = __ldg(vperm + i);
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double x = src[(size_t)k * nv + j];
    ok = ok && isfinite(x);
    dst[4 * (size_t)i + k] = (T)x;
  }
  if (!ok) atomicOr(&ctl->status, ST_NONPHYS_VERTEX);
}

// Caller order (component-major doubles, page-locked host memory read in place
// over the host link) -> internal order in T.  Thread j walks the caller's
// array contiguously, so every host read is coalesced; the writes scatter on
// the device through vinv (caller -> internal vertex).
template <class T>
__global__ void k_host_in(int nv, const int* __restrict__ vinv, const double* __restrict__ src, T* __restrict__ dst,
                          DevCtl* ctl) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const int i = __ldg(vinv + j);
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double x = src[(size_t)k * nv + j];
    ok = ok && isfinite(x);
    dst[4 * (size_t)i + k] = (T)x;
  }
  if (!ok) atomicOr(&ctl->status, ST_NONPHYS_VERTEX);
}

// Internal order in T -> caller order in page-locked host memory, written in
// place with coalesced host writes (the gathers are on the device).
template <class T>
__global__ void k_host_out(int nv, const int* __restrict__ vinv, const T* __restrict__ src, double* __restrict__ dst) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const int i = __ldg(vinv + j);
  T w[4];
  load_vec4(src, i, w);
#pragma unroll
  for (int k = 0; k < 4; ++k) dst[(size_t)k * nv + j] = (double)w[k];
}

template <class T>
__global__ void k_permute_out(int nv, const int* __restrict__ vperm, const T* __restrict__ src,
                              double* __restrict__ dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  int j = __ldg(vperm + i);
#pragma unroll
  for (int k = 0; k < 4; ++k) dst[(size_t)k * nv + j] = (double)src[4 * (size_t)i + k];
}

template <class Tsrc, class Tdst>
__global__ void k_convert(size_t n, const Tsrc* __restrict__ a, Tdst* __restrict__ b) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (Tdst)a[i];
}

}  // namespace rd
