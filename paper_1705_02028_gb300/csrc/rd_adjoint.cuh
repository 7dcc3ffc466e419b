// rd_adjoint.cuh -- hand-written reverse mode of the per-triangle bodies and the
// adjoint kernels of one time step (the step's dt is held fixed).
//
// Every reverse function below re-derives, by the chain rule, one primal
// function of rd_kernels.cuh; the primal values it needs are recomputed from
// the triangle's inputs (the forward kernels do not store intermediates).  The
// non-smooth branches of the N and B schemes -- the regularised |lambda| of
// each node and eigenvalue, the signs inside Theta and its max / 0-over-0
// guards -- are taken from a mask word recorded by the forward pass.
#pragma once

#include "rd_kernels.cuh"

namespace rd {

// ---------------------------------------------------------------------------
// branch masks (one 64-bit word per triangle and stage)
//   bits  0..8   |lambda_k| < delta (regularised branch), node i, eigenvalue k: bit 3i+k
//   bits  9..17  lambda_k < 0
//   bits 18..21  total residual t_k < 0          bits 22..25  t_k == 0
//   bits 26..29  sum_i |N_ik| > |t_k| (den = sum)  bits 30..33  den > 0
//   bits 34..45  N_ik < 0 (bit 34 + 4i + k)      bits 46..57  N_ik == 0
// ---------------------------------------------------------------------------
typedef unsigned long long Mask;

template <class T>
RD_HD Mask node_mask(const TriLin<T>& L, const T hl[3], T eps) {
  Mask m = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const NodeSys<T>& n = L.nd[i];
    T delta = eps * L.r.c * hl[i];
    T la[3] = {(n.w + L.r.c) * hl[i], (n.w - L.r.c) * hl[i], n.w * hl[i]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (fabs(la[k]) < delta) m |= 1ull << (3 * i + k);
      if (la[k] < T(0)) m |= 1ull << (9 + 3 * i + k);
    }
  }
  return m;
}

template <class T>
RD_HD Mask blend_mask(const T tot[4], const T N[3][4]) {
  Mask m = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T num = fabs(tot[k]);
    T D = fabs(N[0][k]) + fabs(N[1][k]) + fabs(N[2][k]);
    T den = D > num ? D : num;
    if (tot[k] < T(0)) m |= 1ull << (18 + k);
    if (tot[k] == T(0)) m |= 1ull << (22 + k);
    if (D > num) m |= 1ull << (26 + k);
    if (den > T(0)) m |= 1ull << (30 + k);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (N[i][k] < T(0)) m |= 1ull << (34 + 4 * i + k);
      if (N[i][k] == T(0)) m |= 1ull << (46 + 4 * i + k);
    }
  }
  return m;
}

RD_HD int mbit(Mask m, int b) { return (int)((m >> b) & 1ull); }

template <class T>
RD_HD T msign(Mask m, int neg_bit, int zero_bit) {
  return mbit(m, zero_bit) ? T(0) : (mbit(m, neg_bit) ? T(-1) : T(1));
}

// ---------------------------------------------------------------------------
// adjoint accumulators
// ---------------------------------------------------------------------------
template <class T>
struct RoeBar {
  T u, v, h, c, ic2h, i2c, alpha, g1u, g1v;
  RD_HD void zero() { u = v = h = c = ic2h = i2c = alpha = g1u = g1v = T(0); }
};

template <class T>
struct NodeBar {
  T w, l3[2], s1[2], s2[2], hp[2];
  RD_HD void zero() { w = l3[0] = l3[1] = s1[0] = s1[1] = s2[0] = s2[1] = hp[0] = hp[1] = T(0); }
};

// reverse of o = K^{+-} v (Kpm_apply): vb += (dK v/dv)^T ob, parameter bars accumulate
template <class T, bool PLUS>
RD_HD void Kpm_rev(const RoeState<T>& r, const NodeSys<T>& n, const T v[4], const T ob[4], T vb[4], RoeBar<T>& rb,
                   NodeBar<T>& nb) {
  const int j = PLUS ? 0 : 1;
  T A = r.alpha * v[0] - r.g1u * v[1] - r.g1v * v[2] + r.g1 * v[3];
  T B = n.nx * v[1] + n.ny * v[2] - n.w * v[0];
  T P = n.s1[j] * A + n.s2[j] * B;
  T Q = n.s2[j] * A + n.hp[j] * B;
  T l3 = n.l3[j];
  nb.l3[j] += ob[0] * v[0] + ob[1] * v[1] + ob[2] * v[2] + ob[3] * v[3];
#pragma unroll
  for (int k = 0; k < 4; ++k) vb[k] += l3 * ob[k];
  T Pb = ob[0] + r.u * ob[1] + r.v * ob[2] + r.h * ob[3];
  T Qb = n.nx * ob[1] + n.ny * ob[2] + n.w * ob[3];
  rb.u += ob[1] * P;
  rb.v += ob[2] * P;
  rb.h += ob[3] * P;
  nb.w += ob[3] * Q;
  nb.s1[j] += Pb * A;
  nb.s2[j] += Pb * B + Qb * A;
  nb.hp[j] += Qb * B;
  T Ab = n.s1[j] * Pb + n.s2[j] * Qb;
  T Bb = n.s2[j] * Pb + n.hp[j] * Qb;
  vb[0] += Ab * r.alpha - Bb * n.w;
  vb[1] += Bb * n.nx - Ab * r.g1u;
  vb[2] += Bb * n.ny - Ab * r.g1v;
  vb[3] += Ab * r.g1;
  rb.alpha += Ab * v[0];
  rb.g1u -= Ab * v[1];
  rb.g1v -= Ab * v[2];
  nb.w -= Bb * v[0];
}

// reverse of x = M^{-1} b: bb += M^{-T} xb, Mb -= (M^{-T} xb) x^T
template <class T>
RD_HD void solve_rev(const LU4<T>& lu, const T x[4], const T xb[4], T bb[4], T Mb[4][4]) {
  T z[4];
  lu.solve_t(xb, z);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    bb[r] += z[r];
#pragma unroll
    for (int c = 0; c < 4; ++c) Mb[r][c] -= z[r] * x[c];
  }
}

// reverse of the blend (Sec. 3.3.3): out = Theta N + (1 - Theta) lda
template <class T>
RD_HD void blend_rev(const T tot[4], const T N[3][4], const T lda[3][4], const T ob[3][4], Mask m, T totb[4],
                     T Nb[3][4], T ldab[3][4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T num = fabs(tot[k]);
    T D = fabs(N[0][k]) + fabs(N[1][k]) + fabs(N[2][k]);
    T den = D > num ? D : num;
    const T iden = rcp(den);
    T th = mbit(m, 30 + k) ? num * iden : T(0);
    T thb = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      thb += ob[i][k] * (N[i][k] - lda[i][k]);
      Nb[i][k] += th * ob[i][k];
      ldab[i][k] += (T(1) - th) * ob[i][k];
    }
    if (!mbit(m, 30 + k)) continue;
    T numb = thb * iden;
    T denb = -(thb * th) * iden;  // -thb num / den^2
    T Db = T(0);
    if (mbit(m, 26 + k)) Db = denb;
    else numb += denb;
#pragma unroll
    for (int i = 0; i < 3; ++i) Nb[i][k] += Db * msign<T>(m, 34 + 4 * i + k, 46 + 4 * i + k);
    totb[k] += numb * msign<T>(m, 18 + k, 22 + k);
  }
}

// reverse of lda_apply: out_i = -K_i^+ M^{-1} x  (y = M^{-1} x given)
template <class T>
RD_HD void lda_rev(const TriLin<T>& L, const T y[4], const T ldab[3][4], T xb[4], T Mb[4][4], RoeBar<T>& rb,
                   NodeBar<T> nb[3]) {
  T yb[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T ob[4] = {-ldab[i][0], -ldab[i][1], -ldab[i][2], -ldab[i][3]};
    Kpm_rev<T, true>(L.r, L.nd[i], y, ob, yb, rb, nb[i]);
  }
  solve_rev(L.lu, y, yb, xb, Mb);
}

// Reverse of linearise(): seeds phiNb (3x4) and phiTb (4) plus the bars already
// accumulated into Mb / rb / nb by later uses of the same linearisation.
// Accumulates into Zb_out (3x4).
template <class T>
RD_HD void linearise_rev(const T Z[3][4], const T nx[3], const T ny[3], const T hl[3], T gamma, T eps,
                         const TriLin<T>& L, Mask mask, const T phiNb[3][4], const T phiTb[4], T Mb[4][4],
                         RoeBar<T>& rb, NodeBar<T> nb[3], T Zb_out[3][4]) {
  const RoeState<T>& r = L.r;
  const T* Zb = L.Zb;
  const T g = r.g1 / gamma, ig = T(1) / gamma, third = T(1) / T(3);
  T Whb[3][4], winb[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) Whb[i][k] = T(0);
  // phi^N_i = K_i^+ (W^_i - win)
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T d[4], db[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = L.Wh[i][k] - L.win[k];
    Kpm_rev<T, true>(r, L.nd[i], d, phiNb[i], db, rb, nb[i]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Whb[i][k] += db[k];
      winb[k] -= db[k];
    }
  }
  // win = M^{-1} S
  T Sb[4] = {T(0), T(0), T(0), T(0)};
  solve_rev(L.lu, L.win, winb, Sb, Mb);
  // S = sum_i K_i^- W^_i
#pragma unroll
  for (int i = 0; i < 3; ++i) Kpm_rev<T, false>(r, L.nd[i], L.Wh[i], Sb, Whb[i], rb, nb[i]);
  // W^_i = dW/dZ(Zbar) Z_i
  T Zbb[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T* w = Whb[i];
    const T* z = Z[i];
    Zb_out[i][0] += T(2) * Zb[0] * w[0] + Zb[1] * w[1] + Zb[2] * w[2] + Zb[3] * ig * w[3];
    Zb_out[i][1] += Zb[0] * w[1] + g * Zb[1] * w[3];
    Zb_out[i][2] += Zb[0] * w[2] + g * Zb[2] * w[3];
    Zb_out[i][3] += Zb[0] * ig * w[3];
    Zbb[0] += T(2) * z[0] * w[0] + z[1] * w[1] + z[2] * w[2] + z[3] * ig * w[3];
    Zbb[1] += z[0] * w[1] + g * z[1] * w[3];
    Zbb[2] += z[0] * w[2] + g * z[2] * w[3];
    Zbb[3] += z[0] * ig * w[3];
  }
  // M = sum_j K_j^- assembled as L3 I + e P^T + sum_j d_j q_j^T
  {
    T L3b = Mb[0][0] + Mb[1][1] + Mb[2][2] + Mb[3][3];
    T S1 = T(0), Pw = T(0), Px = T(0), Py = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      S1 += L.nd[j].s1[1];
      Pw += L.nd[j].s2[1] * L.nd[j].w;
      Px += L.nd[j].s2[1] * L.nd[j].nx;
      Py += L.nd[j].s2[1] * L.nd[j].ny;
    }
    T P[4] = {S1 * r.alpha - Pw, Px - S1 * r.g1u, Py - S1 * r.g1v, S1 * r.g1};
    T Pb[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Pb[c] = Mb[0][c] + r.u * Mb[1][c] + r.v * Mb[2][c] + r.h * Mb[3][c];
      rb.u += Mb[1][c] * P[c];
      rb.v += Mb[2][c] * P[c];
      rb.h += Mb[3][c] * P[c];
    }
    T S1b = Pb[0] * r.alpha - Pb[1] * r.g1u - Pb[2] * r.g1v + Pb[3] * r.g1;
    rb.alpha += Pb[0] * S1;
    rb.g1u -= Pb[1] * S1;
    rb.g1v -= Pb[2] * S1;
    T Pwb = -Pb[0], Pxb = Pb[1], Pyb = Pb[2];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const NodeSys<T>& n = L.nd[j];
      T s2 = n.s2[1], hp = n.hp[1];
      T q[4] = {s2 * r.alpha - hp * n.w, hp * n.nx - s2 * r.g1u, hp * n.ny - s2 * r.g1v, s2 * r.g1};
      T qb[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        qb[c] = n.nx * Mb[1][c] + n.ny * Mb[2][c] + n.w * Mb[3][c];
        nb[j].w += Mb[3][c] * q[c];
      }
      nb[j].s2[1] += qb[0] * r.alpha - qb[1] * r.g1u - qb[2] * r.g1v + qb[3] * r.g1;
      nb[j].hp[1] += -qb[0] * n.w + qb[1] * n.nx + qb[2] * n.ny;
      rb.alpha += qb[0] * s2;
      nb[j].w -= qb[0] * hp;
      rb.g1u -= qb[1] * s2;
      rb.g1v -= qb[2] * s2;
      nb[j].l3[1] += L3b;
      nb[j].s1[1] += S1b;
      nb[j].s2[1] += Pwb * n.w + Pxb * n.nx + Pyb * n.ny;
      nb[j].w += Pwb * s2;
    }
  }
  // node eigen-split -> (u, v, c, ic2h, i2c)
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const NodeSys<T>& n = L.nd[i];
    T delta = eps * r.c * hl[i];
    T la[3] = {(n.w + r.c) * hl[i], (n.w - r.c) * hl[i], n.w * hl[i]};
    const bool reg = mbit(mask, 3 * i) || mbit(mask, 3 * i + 1) || mbit(mask, 3 * i + 2);
    const T idelta = reg ? rcp(delta) : T(0);
    T ab[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      ab[k] = mbit(mask, 3 * i + k) ? (la[k] * la[k] + delta * delta) * (T(0.5) * idelta) : fabs(la[k]);
    T lab[3] = {T(0), T(0), T(0)}, abb[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      T sg = j == 0 ? T(0.5) : T(-0.5);
      T l1 = la[0] * T(0.5) + sg * ab[0];
      T l2 = la[1] * T(0.5) + sg * ab[1];
      T l3 = la[2] * T(0.5) + sg * ab[2];
      T mu1 = l1 - l3, mu2 = l2 - l3;
      T sp = mu1 + mu2, sm = mu1 - mu2;
      T spb = nb[i].s1[j] * r.ic2h + nb[i].hp[j] * T(0.5);
      rb.ic2h += nb[i].s1[j] * sp;
      T smb = nb[i].s2[j] * r.i2c;
      rb.i2c += nb[i].s2[j] * sm;
      T mu1b = spb + smb, mu2b = spb - smb;
      T lb[3] = {mu1b, mu2b, nb[i].l3[j] - mu1b - mu2b};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        lab[k] += T(0.5) * lb[k];
        abb[k] += sg * lb[k];
      }
    }
    T deltab = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (mbit(mask, 3 * i + k)) {
        lab[k] += abb[k] * la[k] * idelta;
        deltab += abb[k] * (delta * delta - la[k] * la[k]) * (T(0.5) * idelta * idelta);
      } else {
        lab[k] += abb[k] * (mbit(mask, 9 + 3 * i + k) ? T(-1) : T(1));
      }
    }
    T wb = nb[i].w + hl[i] * (lab[0] + lab[1] + lab[2]);
    rb.c += hl[i] * (lab[0] - lab[1]) + eps * hl[i] * deltab;
    rb.u += wb * n.nx;
    rb.v += wb * n.ny;
  }
  // phi^T = dF/dZ(Zbar) gx + dG/dZ(Zbar) gy
  {
    const T* gx = L.gx;
    const T* gy = L.gy;
    const T* p = phiTb;
    T gxb[4] = {Zb[1] * p[0] + g * Zb[3] * p[1], Zb[0] * p[0] + (T(2) - g) * Zb[1] * p[1] + Zb[2] * p[2] + Zb[3] * p[3],
                -g * Zb[2] * p[1] + Zb[1] * p[2], g * Zb[0] * p[1] + Zb[1] * p[3]};
    T gyb[4] = {Zb[2] * p[0] + g * Zb[3] * p[2], Zb[2] * p[1] - g * Zb[1] * p[2],
                Zb[0] * p[0] + Zb[1] * p[1] + (T(2) - g) * Zb[2] * p[2] + Zb[3] * p[3], g * Zb[0] * p[2] + Zb[2] * p[3]};
    Zbb[0] += (gx[1] + gy[2]) * p[0] + g * gx[3] * p[1] + g * gy[3] * p[2];
    Zbb[1] += gx[0] * p[0] + ((T(2) - g) * gx[1] + gy[2]) * p[1] + (gx[2] - g * gy[1]) * p[2] + gx[3] * p[3];
    Zbb[2] += gy[0] * p[0] + (gy[1] - g * gx[2]) * p[1] + (gx[1] + (T(2) - g) * gy[2]) * p[2] + gy[3] * p[3];
    Zbb[3] += g * gx[0] * p[1] + g * gy[0] * p[2] + (gx[1] + gy[2]) * p[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T ax = nx[i] * hl[i], ay = ny[i] * hl[i];
#pragma unroll
      for (int k = 0; k < 4; ++k) Zb_out[i][k] += ax * gxb[k] + ay * gyb[k];
    }
  }
  // Roe state from Zbar
  {
    T iz = rcp(Zb[0]);
    T c2 = r.c * r.c;
    T cb = rb.c + rb.i2c * r.ic2h;
    T ic2hb = rb.ic2h + rb.i2c * r.c;
    T ic2b = T(0.5) * ic2hb;
    T c2b = -r.ic2 * r.ic2 * ic2b + cb * r.i2c;  // i2c = 1 / (2 c)
    T q2hb = r.g1 * rb.alpha - r.g1 * c2b;
    T hb = rb.h + r.g1 * c2b;
    T ub = rb.u + r.g1 * rb.g1u + r.u * q2hb;
    T vb = rb.v + r.g1 * rb.g1v + r.v * q2hb;
    (void)c2;
    Zbb[1] += iz * ub;
    Zbb[2] += iz * vb;
    Zbb[3] += iz * hb;
    T izb = Zb[1] * ub + Zb[2] * vb + Zb[3] * hb;
    Zbb[0] -= iz * iz * izb;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) Zb_out[i][k] += third * Zbb[k];
}

// Reverse of the stage-1 body (SCHEME RD_B2 / RD_LDA2 / RD_N1).  outb: adjoint of
// the three shares; recb (two-stage schemes): adjoint of (phi^N_0..2, phi^T).
// stage1_rev_lin takes the triangle's linearisation L (as linearise computes it
// from Z) instead of recomputing it.
template <class T, int SCHEME>
RD_HD int stage1_rev_lin(const TriLin<T>& L, const T Z[3][4], const T nx[3], const T ny[3], const T hl[3], T gamma,
                         T eps, Mask mask, const T outb[3][4], const T recb[16], T Zbar[3][4]) {
  T phiNb[3][4], phiTb[4] = {T(0), T(0), T(0), T(0)}, Mb[4][4];
  RoeBar<T> rb;
  rb.zero();
  NodeBar<T> nb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) nb[i].zero();
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) Mb[r][c] = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) phiNb[i][k] = T(0);
  if (SCHEME == RD_N1) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) phiNb[i][k] = outb[i][k];
  } else {
    T y[4], lda[3][4], ldab[3][4];
    L.lu.solve(L.phiT, y);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T o[4];
      Kpm_apply<T, true>(L.r, L.nd[i], y, o);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        lda[i][k] = -o[k];
        ldab[i][k] = T(0);
      }
    }
    if (SCHEME == RD_LDA2) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) ldab[i][k] = outb[i][k];
    } else {
      blend_rev(L.phiT, L.phiN, lda, outb, mask, phiTb, phiNb, ldab);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) phiNb[i][k] += recb[4 * i + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) phiTb[k] += recb[12 + k];
    lda_rev(L, y, ldab, phiTb, Mb, rb, nb);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) Zbar[i][k] = T(0);
  linearise_rev(Z, nx, ny, hl, gamma, eps, L, mask, phiNb, phiTb, Mb, rb, nb, Zbar);
  return 0;
}
template <class T, int SCHEME>
RD_HD int stage1_rev(const T Z[3][4], const T nx[3], const T ny[3], const T hl[3], T gamma, T eps, Mask mask,
                     const T outb[3][4], const T recb[16], T Zbar[3][4]) {
  TriLin<T> L;
  int st = linearise(Z, nx, ny, hl, gamma, eps, L);
  if (st) return st;
  return stage1_rev_lin<T, SCHEME>(L, Z, nx, ny, hl, gamma, eps, mask, outb, recb, Zbar);
}

// Reverse of the stage-2 body: outputs the adjoints of Z*, W^n, W* (3x4 each)
// and of the stage-1 record (16).
// stage2_rev_tot takes the stage-2 totals Phi^N_i, Phi^T (stage2_totals) and
// the mass factor q = |T| / (3 dt) as given; stage2_rev_lin forms them from
// W^n, W* and the record.
template <class T, int SCHEME>
RD_HD int stage2_rev_tot(const TriLin<T>& L, const T PhiN[3][4], const T PhiT[4], T q, const T Zs[3][4],
                         const T nx[3], const T ny[3], const T hl[3], T gamma, T eps, Mask mask, const T outb[3][4],
                         T Zsb[3][4], T Wnb[3][4], T Wsb[3][4], T recb[16]);
template <class T, int SCHEME>
RD_HD int stage2_rev_lin(const TriLin<T>& L, const T Zs[3][4], const T Wn[3][4], const T Ws[3][4], const T rec[16],
                         const T nx[3], const T ny[3], const T hl[3], T area, T dt, T gamma, T eps, Mask mask,
                         const T outb[3][4], T Zsb[3][4], T Wnb[3][4], T Wsb[3][4], T recb[16]) {
  const T q = area * (T(1) / T(3)) * rcp(dt);  // |T| / (3 dt), as in stage2_totals
  T PhiN[3][4], PhiT[4];
  stage2_totals(L, Wn, Ws, rec, area, rcp(dt), PhiN, PhiT);
  return stage2_rev_tot<T, SCHEME>(L, PhiN, PhiT, q, Zs, nx, ny, hl, gamma, eps, mask, outb, Zsb, Wnb, Wsb, recb);
}
template <class T, int SCHEME>
RD_HD int stage2_rev_tot(const TriLin<T>& L, const T PhiN[3][4], const T PhiT[4], T q, const T Zs[3][4],
                         const T nx[3], const T ny[3], const T hl[3], T gamma, T eps, Mask mask, const T outb[3][4],
                         T Zsb[3][4], T Wnb[3][4], T Wsb[3][4], T recb[16]) {
  T y[4], lda[3][4], ldab[3][4];
  L.lu.solve(PhiT, y);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T o[4];
    Kpm_apply<T, true>(L.r, L.nd[i], y, o);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      lda[i][k] = -o[k];
      ldab[i][k] = T(0);
    }
  }
  T PhiNb[3][4], PhiTb[4] = {T(0), T(0), T(0), T(0)}, Mb[4][4];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) PhiNb[i][k] = T(0);
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) Mb[r][c] = T(0);
  if (SCHEME == RD_LDA2) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) ldab[i][k] = outb[i][k];
  } else {
    blend_rev(PhiT, PhiN, lda, outb, mask, PhiTb, PhiNb, ldab);
  }
  RoeBar<T> rb;
  rb.zero();
  NodeBar<T> nb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) nb[i].zero();
  lda_rev(L, y, ldab, PhiTb, Mb, rb, nb);
  T phiNb[3][4], phiTb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    phiTb[k] = T(0.5) * PhiTb[k];
    recb[12 + k] = T(0.5) * PhiTb[k];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T mb = PhiNb[i][k] + PhiTb[k];
      phiNb[i][k] = T(0.5) * PhiNb[i][k];
      recb[4 * i + k] = T(0.5) * PhiNb[i][k];
      Wsb[i][k] = q * mb;
      Wnb[i][k] = -(q * mb);
      Zsb[i][k] = T(0);
    }
  linearise_rev(Zs, nx, ny, hl, gamma, eps, L, mask, phiNb, phiTb, Mb, rb, nb, Zsb);
  return 0;
}
template <class T, int SCHEME>
RD_HD int stage2_rev(const T Zs[3][4], const T Wn[3][4], const T Ws[3][4], const T rec[16], const T nx[3],
                     const T ny[3], const T hl[3], T area, T dt, T gamma, T eps, Mask mask, const T outb[3][4],
                     T Zsb[3][4], T Wnb[3][4], T Wsb[3][4], T recb[16]) {
  TriLin<T> L;
  int st = linearise(Zs, nx, ny, hl, gamma, eps, L);
  if (st) return st;
  return stage2_rev_lin<T, SCHEME>(L, Zs, Wn, Ws, rec, nx, ny, hl, area, dt, gamma, eps, mask, outb, Zsb, Wnb, Wsb,
                                   recb);
}

// Mask of a stage-1 / stage-2 evaluation (recomputes the primal of the triangle).
template <class T, int SCHEME>
RD_HD Mask stage1_mask(const T Z[3][4], const T nx[3], const T ny[3], const T hl[3], T gamma, T eps) {
  TriLin<T> L;
  if (linearise(Z, nx, ny, hl, gamma, eps, L)) return 0;
  Mask m = node_mask(L, hl, eps);
  if (SCHEME == RD_B2) m |= blend_mask(L.phiT, L.phiN);
  return m;
}

template <class T, int SCHEME>
RD_HD Mask stage2_mask(const T Zs[3][4], const T Wn[3][4], const T Ws[3][4], const T rec[16], const T nx[3],
                       const T ny[3], const T hl[3], T area, T dt, T gamma, T eps) {
  TriLin<T> L;
  if (linearise(Zs, nx, ny, hl, gamma, eps, L)) return 0;
  Mask m = node_mask(L, hl, eps);
  if (SCHEME != RD_B2) return m;
  T PhiN[3][4], PhiT[4];
  stage2_totals(L, Wn, Ws, rec, area, rcp(dt), PhiN, PhiT);  // as the masked forward kernel
  return m | blend_mask(PhiT, PhiN);
}

// A triangle's linearisation as LIN_WORDS scalars (the LU pivots packed into
// the last one), stored field-major (word w of triangle t at w * nt + t) by the
// forward re-run for the reverse kernels.
constexpr int LIN_WORDS = 12 + 3 * 11 + 16 + 4 + 4 + 12 + 4 + 4 + 4 + 12 + 4 + 1;
template <class T, class F>
__device__ __forceinline__ void lin_fields(TriLin<T>& L, F&& f) {
  int w = 0;
  RoeState<T>& r = L.r;
  f(w++, r.u); f(w++, r.v); f(w++, r.h); f(w++, r.c); f(w++, r.q2h); f(w++, r.ic2);
  f(w++, r.ic2h); f(w++, r.i2c); f(w++, r.g1); f(w++, r.alpha); f(w++, r.g1u); f(w++, r.g1v);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    NodeSys<T>& n = L.nd[i];
    f(w++, n.nx); f(w++, n.ny); f(w++, n.w);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      f(w++, n.l3[j]); f(w++, n.s1[j]); f(w++, n.s2[j]); f(w++, n.hp[j]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) f(w++, L.lu.a[a][b]);
#pragma unroll
  for (int k = 0; k < 4; ++k) f(w++, L.lu.rdiag[k]);
#pragma unroll
  for (int k = 0; k < 4; ++k) f(w++, L.phiT[k]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) f(w++, L.phiN[i][k]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    f(w++, L.Zb[k]); f(w++, L.gx[k]); f(w++, L.gy[k]); f(w++, L.win[k]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) f(w++, L.Wh[i][k]);
}
template <class T>
__device__ __forceinline__ void store_lin(TriLin<T>& L, T* __restrict__ out, int t, int nt) {
  lin_fields(L, [&](int w, T& x) { out[(size_t)w * nt + t] = x; });
  out[(size_t)(LIN_WORDS - 1) * nt + t] = T(L.lu.piv[0] + 4 * L.lu.piv[1] + 16 * L.lu.piv[2]);
}
template <class T>
__device__ __forceinline__ void load_lin(TriLin<T>& L, const T* __restrict__ in, int t, int nt) {
  lin_fields(L, [&](int w, T& x) { x = __ldg(in + (size_t)w * nt + t); });
  const int pk = (int)__ldg(in + (size_t)(LIN_WORDS - 1) * nt + t);
  L.lu.piv[0] = pk & 3;
  L.lu.piv[1] = (pk >> 2) & 3;
  L.lu.piv[2] = (pk >> 4) & 3;
}

// reverse of vertex_Z: Zb -> Wb += (dZ/dW)^T Zb
template <class T>
RD_HD void vertex_Z_rev(const T W[4], T gamma, const T Zb[4], T Wb[4]) {
  T rho = W[0];
  const T ir = rcp(rho);
  T u = W[1] * ir, v = W[2] * ir;
  T g1 = gamma - T(1);
  T p = g1 * (W[3] - T(0.5) * rho * (u * u + v * v));
  T h = (W[3] + p) * ir;
  T s = sqrt(rho), is = rcp(s);
  T Z1 = s * u, Z2 = s * v;
  Wb[0] += T(0.5) * is * Zb[0] - (Zb[1] * Z1 + Zb[2] * Z2) * (T(0.5) * ir) +
           Zb[3] * (T(0.5) * g1 * (u * u + v * v) - T(0.5) * h) * is;
  Wb[1] += (Zb[1] - Zb[3] * g1 * u) * is;
  Wb[2] += (Zb[2] - Zb[3] * g1 * v) * is;
  Wb[3] += Zb[3] * gamma * is;
}

}  // namespace rd
