// rd_oracle.cpp -- plain CPU oracle of the residual-distribution (RD) Euler step.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
// that the CUDA path is checked against.  Only tests/, __graft_entry__.smoke()
// and bench.py's cpu_baseline / reference legs may load it.  It shares no code,
// header, table or helper with the CUDA library, and it includes nothing from it.
//
// What it computes (Paardekooper 2017, "Multidimensional upwind hydrodynamics
// on unstructured meshes using GPUs I"):
//   * ideal-gas 2-D Euler equations, W = (rho, rho u, rho v, e)          (Sec. 3)
//   * Roe parameter vector Z = sqrt(rho) (1, u, v, h)          (Sec. 3.1.1, Sec. 3.2)
//   * piecewise-linear Z^h, cell residual phi^T = sum_i K_i Z_i with the
//     flux Jacobians dF/dZ evaluated at the nodal mean of Z      (Eqs. eqZh..eqLinearA)
//   * eigen-split K_i^{+-} = R Lambda^{+-} L                      (Sec. 3.2, App. A)
//   * N, LDA and blended B distributions, the Bmax / Bmin variants and the
//     shock-sensor blend Bx                                       (Sec. 3.3.1-3.3.3)
//   * forward-Euler update with the CFL time step                 (Eq. eqUpdate, Sec. 3.2)
//   * the explicit two-stage scheme with total residuals Phi^N, Phi^LDA,
//     mass matrices m^N, m^LDA and global or selective lumping    (Sec. 3.4, eqRK1/eqRK2)
//   * boundary conditions: ghost vertices held at their initial state
//     (non-reflecting / inflow) and weakly imposed reflecting walls   (Sec. 3.5)
//
// Everything is written in the paper's order and notation; no fusion, no
// reordering beyond what the formulas state.  All arithmetic is templated on the
// scalar type S so that the same source runs in double (the oracle proper),
// long double (round-off floor) and a forward-mode dual number (directional
// derivatives for the adjoint checks).
//
// Readings of points where the paper is silent or garbled:
//   (R1) K^{+-} act on the conservative linearised states W^_i = M(Zbar) Z_i,
//        M = dW/dZ; the K matrix of App. A is the conservative Jacobian.
//   (R2) n_i is the inward normal of the edge opposite node i, |n_i| = edge
//        length; K_i = (1/2)|n_i| K(n_i/|n_i|).
//   (R3) L = R^{-1} is obtained by numerically inverting the App. A eigenvector
//        matrix (App. A's printed inverse has sign typos).
//   (R4) |lambda| carries a Harten-type C^1 regularisation below
//        delta = eps * c * |n_i| / 2, so that N^ exists at stagnation.
//   (R5) Theta_kk = |phi^T_k| / max(sum_j |phi^N_jk|, |phi^T_k|), 0/0 -> 0
//        (the max only guards the triangle inequality against round-off).
//   (R6) Stage 2 blends total residuals; beta_i is evaluated at W*;
//        phi^N(W^n) and phi^T(W^n) are recomputed from W^n.
//   (R7) V_i = sum_{T containing i} |T|/3.
//   (R8) dt = CFL * min_i 2 V_i / sum_T l_max^T lambda_max^T, at W^n, used by
//        both stages.
//   (R9) Bx: theta = min(1, s^2 h_T / L) with s = max(0, -L div v / (|v|_max -
//        |v|_min)); div v of the piecewise-linear vertex velocities, h_T =
//        sqrt(2 |T|), L = max(Lx, Ly), |v| extremes over all vertices of the
//        state being distributed (W^n in stage 1, W* in stage 2); s = 0 when
//        |v|_max = |v|_min.  On the unit box theta = s^2 h as printed.
//   (R12) Ghost vertices are reset to their initial state at the start of
//        every step (the value entering the step); W* of a ghost vertex is
//        the ordinary stage-1 update.  "Initial" = the state passed to run().
//   (R13) The wall correction residual Phi^c is a spatial residual: it enters
//        stage 1 (and N1) at W^n and stage 2 as (Phi^c(W^n) + Phi^c(W*)) / 2,
//        like phi^T.  The wall's outward unit normal is minus the inward
//        normal of the edge in its triangle; h = (e + p) / rho.
//   (R10) Bmax / Bmin in stage 2 take max_k / min_k of the total-residual
//        Theta_kk of (R6); selective lumping adds its correction to the
//        blended total residual (it sums to zero over the triangle).
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared [-fopenmp]

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include <limits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace ora {

enum { OK = 0, EINVAL = 1, ENONPHYS = 4 };
enum { N1 = 0, B2 = 1, LDA2 = 2, BMAX2 = 3, BMIN2 = 4, BX2 = 5 };
enum { SELECTIVE_LUMPING = 0x100 };  // flag or-ed into the scheme code

// ---------------------------------------------------------------------------
// Forward-mode dual number (value + one directional derivative).
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double y) : v(x), d(y) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual& operator/=(Dual& a, Dual b) { a = a / b; return a; }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2 * s)); }
inline Dual fabs(Dual a) { return a.v < 0 ? -a : a; }
inline double val(Dual a) { return a.v; }

inline double val(double a) { return a; }
inline double val(long double a) { return (double)a; }
using std::sqrt;
using std::fabs;

template <class S> inline S smax(S a, S b) { return a < b ? b : a; }
template <class S> inline S smin(S a, S b) { return b < a ? b : a; }

// ---------------------------------------------------------------------------
// Mesh in the oracle's own form: geometry recomputed here from coordinates.
// ---------------------------------------------------------------------------
template <class S>
struct Mesh {
  int32_t nv = 0, nt = 0;
  std::vector<int32_t> tri;   // [nt][3]
  std::vector<S> n;           // [nt][3][2] inward normals, |n_i| = edge length
  std::vector<S> area;        // [nt]
  std::vector<S> lmax;        // [nt] longest edge
  std::vector<S> V;           // [nv] nodal volume (R7)
  S L = S(1);                 // domain size max(Lx, Ly) (R9)
  // boundary conditions (Sec. 3.5)
  std::vector<uint8_t> ghost;      // [nv] 1: state held at its initial value (empty: none)
  std::vector<int32_t> wall;       // [n_wall][2]: (triangle, corner) of the edge opposite the corner
  S alpha = S(0.75);               // wall-correction distribution parameter
};

// Geometry of every triangle from the (periodically shifted) corner positions.
template <class S>
int build_mesh(int32_t nv, const double* xy, int32_t nt, const int32_t* tri,
               const int8_t* shift, double Lx, double Ly, Mesh<S>& m) {
  m.nv = nv; m.nt = nt;
  m.L = S(Lx > Ly ? Lx : Ly);
  if (!(m.L > S(0))) m.L = S(1);
  m.tri.assign(tri, tri + 3 * (size_t)nt);
  m.n.assign(6 * (size_t)nt, S(0));
  m.area.assign(nt, S(0));
  m.lmax.assign(nt, S(0));
  m.V.assign(nv, S(0));
  for (int32_t t = 0; t < nt; ++t) {
    S x[3], y[3];
    for (int c = 0; c < 3; ++c) {
      int32_t v = tri[3 * t + c];
      if (v < 0 || v >= nv) return EINVAL;
      double sx = shift ? shift[6 * t + 2 * c] : 0, sy = shift ? shift[6 * t + 2 * c + 1] : 0;
      x[c] = S(xy[2 * v]) + S(sx) * S(Lx);
      y[c] = S(xy[2 * v + 1]) + S(sy) * S(Ly);
    }
    // inward normal of the edge opposite node c: rotate (x_{c+2} - x_{c+1}) by +90 deg
    for (int c = 0; c < 3; ++c) {
      int a = (c + 1) % 3, b = (c + 2) % 3;
      m.n[6 * t + 2 * c] = y[a] - y[b];
      m.n[6 * t + 2 * c + 1] = x[b] - x[a];
    }
    S A = S(0.5) * ((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]));
    if (!(A > S(0))) return EINVAL;  // counter-clockwise, non-degenerate only
    m.area[t] = A;
    S lm = S(0);
    for (int c = 0; c < 3; ++c) {
      S nx = m.n[6 * t + 2 * c], ny = m.n[6 * t + 2 * c + 1];
      lm = smax(lm, S(sqrt(nx * nx + ny * ny)));
    }
    m.lmax[t] = lm;
    for (int c = 0; c < 3; ++c) m.V[tri[3 * t + c]] += A / S(3);
  }
  for (int32_t i = 0; i < nv; ++i)
    if (!(m.V[i] > S(0))) return EINVAL;  // every vertex must belong to a triangle
  return OK;
}

// ---------------------------------------------------------------------------
// Primitive / parameter-vector conversions (Sec. 3, Sec. 3.1.1).
// ---------------------------------------------------------------------------
template <class S>
int primitive(const S W[4], S gamma, S& rho, S& u, S& v, S& p) {
  rho = W[0];
  if (!(rho > S(0))) return ENONPHYS;
  u = W[1] / rho;
  v = W[2] / rho;
  p = (gamma - S(1)) * (W[3] - S(0.5) * rho * (u * u + v * v));
  if (!(p > S(0))) return ENONPHYS;
  return OK;
}

// Z = sqrt(rho) (1, u, v, h), h = (e + p) / rho.
template <class S>
int parameter_vector(const S W[4], S gamma, S Z[4]) {
  S rho, u, v, p;
  int e = primitive(W, gamma, rho, u, v, p);
  if (e) return e;
  S h = (W[3] + p) / rho;
  S sr = sqrt(rho);
  Z[0] = sr; Z[1] = sr * u; Z[2] = sr * v; Z[3] = sr * h;
  return OK;
}

// ---------------------------------------------------------------------------
// Small dense linear algebra.
// ---------------------------------------------------------------------------
template <class S> void matvec(const S A[4][4], const S x[4], S y[4]) {
  for (int r = 0; r < 4; ++r) {
    S s = S(0);
    for (int c = 0; c < 4; ++c) s += A[r][c] * x[c];
    y[r] = s;
  }
}
template <class S> void matmul(const S A[4][4], const S B[4][4], S C[4][4]) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      S s = S(0);
      for (int k = 0; k < 4; ++k) s += A[r][k] * B[k][c];
      C[r][c] = s;
    }
}
// Gauss-Jordan inverse with partial pivoting.  Returns nonzero if singular.
template <class S> int invert4(const S Ain[4][4], S Ainv[4][4]) {
  S a[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      a[r][c] = Ain[r][c];
      a[r][c + 4] = (r == c) ? S(1) : S(0);
    }
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (!(fabs(a[piv][col]) > S(0))) return ENONPHYS;
    if (piv != col)
      for (int c = 0; c < 8; ++c) std::swap(a[piv][c], a[col][c]);
    S d = a[col][col];
    for (int c = 0; c < 8; ++c) a[col][c] = a[col][c] / d;
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      S f = a[r][col];
      for (int c = 0; c < 8; ++c) a[r][c] = a[r][c] - f * a[col][c];
    }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) Ainv[r][c] = a[r][c + 4];
  return OK;
}

// ---------------------------------------------------------------------------
// Flux Jacobians with respect to Z (Sec. 3.2, eqRes..eqLinearA).
// F(Z) = (Z1 Z2, Z2^2 + p, Z2 Z3, Z2 Z4), G(Z) = (Z1 Z3, Z2 Z3, Z3^2 + p, Z3 Z4),
// p = (gamma-1)/gamma (Z1 Z4 - (Z2^2 + Z3^2)/2): both quadratic in Z.
// ---------------------------------------------------------------------------
template <class S>
void flux_jacobians_Z(const S Z[4], S gamma, S A[4][4], S B[4][4]) {
  S g = (gamma - S(1)) / gamma;
  S dp[4] = {g * Z[3], -g * Z[1], -g * Z[2], g * Z[0]};
  S z = S(0);
  S Ar[4][4] = {{Z[1], Z[0], z, z},
                {dp[0], S(2) * Z[1] + dp[1], dp[2], dp[3]},
                {z, Z[2], Z[1], z},
                {z, Z[3], z, Z[1]}};
  S Br[4][4] = {{Z[2], z, Z[0], z},
                {z, Z[2], Z[1], z},
                {dp[0], dp[1], S(2) * Z[2] + dp[2], dp[3]},
                {z, z, Z[3], Z[2]}};
  std::memcpy(A, Ar, sizeof(Ar));
  std::memcpy(B, Br, sizeof(Br));
}

// dW/dZ at Z: W(Z) = (Z1^2, Z1 Z2, Z1 Z3, Z1 Z4/gamma + (gamma-1)/(2 gamma)(Z2^2 + Z3^2)).
template <class S>
void dWdZ(const S Z[4], S gamma, S M[4][4]) {
  S g = (gamma - S(1)) / gamma, z = S(0);
  S Mr[4][4] = {{S(2) * Z[0], z, z, z},
                {Z[1], Z[0], z, z},
                {Z[2], z, Z[0], z},
                {Z[3] / gamma, g * Z[1], g * Z[2], Z[0] / gamma}};
  std::memcpy(M, Mr, sizeof(Mr));
}

// ---------------------------------------------------------------------------
// App. A: K = A n_x + B n_y (conservative), its eigenvalues and right eigenvectors
// for a unit normal (nx, ny) at the state (u, v, h).
// ---------------------------------------------------------------------------
template <class S>
void K_matrix(S u, S v, S h, S gamma, S nx, S ny, S K[4][4]) {
  S g1 = gamma - S(1), g2 = gamma - S(2);
  S w = u * nx + v * ny;
  S alpha = g1 * (u * u + v * v) / S(2);
  S Kr[4][4] = {
      {S(0), nx, ny, S(0)},
      {alpha * nx - u * w, w - g2 * u * nx, u * ny - g1 * v * nx, g1 * nx},
      {alpha * ny - v * w, v * nx - g1 * u * ny, w - g2 * v * ny, g1 * ny},
      {(alpha - h) * w, h * nx - g1 * u * w, h * ny - g1 * v * w, gamma * w}};
  std::memcpy(K, Kr, sizeof(Kr));
}

template <class S>
void eigen_R(S u, S v, S h, S c, S gamma, S nx, S ny, S lam[4], S R[4][4]) {
  S g1 = gamma - S(1);
  S w = u * nx + v * ny;
  S alpha = g1 * (u * u + v * v) / S(2);
  lam[0] = w + c; lam[1] = w - c; lam[2] = w; lam[3] = w;
  // columns e1..e4
  S Rr[4][4] = {{S(1), S(1), S(0), S(1)},
                {u + c * nx, u - c * nx, -ny, u},
                {v + c * ny, v - c * ny, nx, v},
                {h + c * w, h - c * w, v * nx - u * ny, alpha / g1}};
  std::memcpy(R, Rr, sizeof(Rr));
}

// Regularised |lambda| (reading R4): C^1 Harten form below delta.
template <class S>
S abs_reg(S lam, S delta) {
  S a = fabs(lam);
  if (delta > S(0) && a < delta) return (lam * lam + delta * delta) / (S(2) * delta);
  return a;
}

// ---------------------------------------------------------------------------
// One triangle's linearisation and distributions (Sec. 3.2-3.3).
// ---------------------------------------------------------------------------
template <class S>
struct TriLin {
  S Zbar[4];
  S u, v, h, c;        // Roe state
  S What[3][4];        // W^_i = M(Zbar) Z_i
  S Kp[3][4][4], Km[3][4][4], K[3][4][4];
  S Nhat[4][4];
  S phiT[4];
  S phiN[3][4];
  S beta[3][4][4];
  S phiLDA[3][4];
  S theta[4];
  S phiB[3][4];
};

template <class S>
int linearise(const S Z[3][4], const S n[3][2], S gamma, S eps, TriLin<S>& o) {
  // nodal mean of Z (eqLinearA) and the Roe state it defines
  for (int k = 0; k < 4; ++k) o.Zbar[k] = (Z[0][k] + Z[1][k] + Z[2][k]) / S(3);
  if (!(o.Zbar[0] > S(0))) return ENONPHYS;
  o.u = o.Zbar[1] / o.Zbar[0];
  o.v = o.Zbar[2] / o.Zbar[0];
  o.h = o.Zbar[3] / o.Zbar[0];
  S c2 = (gamma - S(1)) * (o.h - (o.u * o.u + o.v * o.v) / S(2));
  if (!(c2 > S(0))) return ENONPHYS;
  o.c = sqrt(c2);

  // phi^T = sum_i K_i Z_i with K_i = (1/2) [A_x n_ix + A_y n_iy](Zbar)   (Sec. 3.2)
  S A[4][4], B[4][4];
  flux_jacobians_Z(o.Zbar, gamma, A, B);
  for (int k = 0; k < 4; ++k) o.phiT[k] = S(0);
  for (int i = 0; i < 3; ++i) {
    S KZ[4][4];
    for (int r = 0; r < 4; ++r)
      for (int q = 0; q < 4; ++q) KZ[r][q] = S(0.5) * (A[r][q] * n[i][0] + B[r][q] * n[i][1]);
    S t[4];
    matvec(KZ, Z[i], t);
    for (int k = 0; k < 4; ++k) o.phiT[k] += t[k];
  }

  // conservative linearised nodal states (reading R1)
  S M[4][4];
  dWdZ(o.Zbar, gamma, M);
  for (int i = 0; i < 3; ++i) matvec(M, Z[i], o.What[i]);

  // K_i = R Lambda L, K_i^{+-} = R Lambda^{+-} L  (Sec. 3.2, App. A, readings R2-R4)
  for (int i = 0; i < 3; ++i) {
    S len = sqrt(n[i][0] * n[i][0] + n[i][1] * n[i][1]);
    S nx = n[i][0] / len, ny = n[i][1] / len;
    S lam[4], R[4][4], L[4][4];
    eigen_R(o.u, o.v, o.h, o.c, gamma, nx, ny, lam, R);
    if (invert4(R, L)) return ENONPHYS;
    S delta = eps * o.c * len / S(2);
    S lp[4], lm[4], la[4];
    for (int k = 0; k < 4; ++k) {
      la[k] = lam[k] * len / S(2);
      S ab = abs_reg(la[k], delta);
      lp[k] = (la[k] + ab) / S(2);
      lm[k] = (la[k] - ab) / S(2);
    }
    for (int r = 0; r < 4; ++r)
      for (int q = 0; q < 4; ++q) {
        S sp = S(0), sm = S(0), s0 = S(0);
        for (int k = 0; k < 4; ++k) {
          sp += R[r][k] * lp[k] * L[k][q];
          sm += R[r][k] * lm[k] * L[k][q];
          s0 += R[r][k] * la[k] * L[k][q];
        }
        o.Kp[i][r][q] = sp;
        o.Km[i][r][q] = sm;
        o.K[i][r][q] = s0;
      }
  }

  // N^ = (sum_j K_j^-)^{-1}   (Sec. 3.3.1)
  S sumKm[4][4];
  for (int r = 0; r < 4; ++r)
    for (int q = 0; q < 4; ++q) sumKm[r][q] = o.Km[0][r][q] + o.Km[1][r][q] + o.Km[2][r][q];
  if (invert4(sumKm, o.Nhat)) return ENONPHYS;

  // N scheme: phi_i^N = K_i^+ (W^_i - N^ sum_j K_j^- W^_j)
  S s[4] = {S(0), S(0), S(0), S(0)};
  for (int j = 0; j < 3; ++j) {
    S t[4];
    matvec(o.Km[j], o.What[j], t);
    for (int k = 0; k < 4; ++k) s[k] += t[k];
  }
  S win[4];
  matvec(o.Nhat, s, win);
  for (int i = 0; i < 3; ++i) {
    S d[4];
    for (int k = 0; k < 4; ++k) d[k] = o.What[i][k] - win[k];
    matvec(o.Kp[i], d, o.phiN[i]);
  }

  // LDA scheme: beta_i = -K_i^+ N^, phi_i^LDA = beta_i phi^T   (Sec. 3.3.2)
  for (int i = 0; i < 3; ++i) {
    S P[4][4];
    matmul(o.Kp[i], o.Nhat, P);
    for (int r = 0; r < 4; ++r)
      for (int q = 0; q < 4; ++q) o.beta[i][r][q] = -P[r][q];
    matvec(o.beta[i], o.phiT, o.phiLDA[i]);
  }

  // B scheme: diagonal Theta, phi^B = Theta phi^N + (I - Theta) phi^LDA   (Sec. 3.3.3, R5)
  for (int k = 0; k < 4; ++k) {
    S num = fabs(o.phiT[k]);
    S den = smax(fabs(o.phiN[0][k]) + fabs(o.phiN[1][k]) + fabs(o.phiN[2][k]), num);
    o.theta[k] = den > S(0) ? num / den : S(0);
  }
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k)
      o.phiB[i][k] = o.theta[k] * o.phiN[i][k] + (S(1) - o.theta[k]) * o.phiLDA[i][k];
  return OK;
}

// Gather the three nodal Z vectors of triangle t from per-vertex Z.
template <class S>
void tri_Z(const Mesh<S>& m, const std::vector<S>& Zv, int32_t t, S Z[3][4], S n[3][2]) {
  for (int c = 0; c < 3; ++c) {
    int32_t v = m.tri[3 * t + c];
    for (int k = 0; k < 4; ++k) Z[c][k] = Zv[4 * (size_t)v + k];
    n[c][0] = m.n[6 * t + 2 * c];
    n[c][1] = m.n[6 * t + 2 * c + 1];
  }
}

template <class S>
int all_Z(const Mesh<S>& m, const std::vector<S>& W, S gamma, std::vector<S>& Zv) {
  Zv.assign(4 * (size_t)m.nv, S(0));
  for (int32_t i = 0; i < m.nv; ++i) {
    S Wi[4] = {W[4 * (size_t)i], W[4 * (size_t)i + 1], W[4 * (size_t)i + 2], W[4 * (size_t)i + 3]};
    int e = parameter_vector(Wi, gamma, &Zv[4 * (size_t)i]);
    if (e) return e;
  }
  return OK;
}

// CFL time step (Sec. 3.2, reading R8).
template <class S>
int time_step(const Mesh<S>& m, const std::vector<S>& W, S gamma, S cfl, S& dt) {
  std::vector<S> sig(m.nv, S(0)), spd(m.nv, S(0));
  for (int32_t i = 0; i < m.nv; ++i) {
    S Wi[4] = {W[4 * (size_t)i], W[4 * (size_t)i + 1], W[4 * (size_t)i + 2], W[4 * (size_t)i + 3]};
    S rho, u, v, p;
    int e = primitive(Wi, gamma, rho, u, v, p);
    if (e) return e;
    spd[i] = sqrt(u * u + v * v) + sqrt(gamma * p / rho);
  }
  for (int32_t t = 0; t < m.nt; ++t) {
    S lam = smax(smax(spd[m.tri[3 * t]], spd[m.tri[3 * t + 1]]), spd[m.tri[3 * t + 2]]);
    for (int c = 0; c < 3; ++c) sig[m.tri[3 * t + c]] += m.lmax[t] * lam;
  }
  S best = S(2) * m.V[0] / sig[0];
  for (int32_t i = 1; i < m.nv; ++i) best = smin(best, S(2) * m.V[i] / sig[i]);
  dt = cfl * best;
  return OK;
}

// Blend of N and LDA shares (Sec. 3.3.3): B uses the diagonal Theta; Bmax and
// Bmin put max_k Theta_kk or min_k Theta_kk on every diagonal entry; Bx uses
// the scalar theta of its shock sensor.  out_i = th phi^N_i + (1 - th) phi^LDA_i.
template <class S>
void blend_shares(int base, const S theta[4], S theta_x, const S N[3][4], const S LDA[3][4], S out[3][4]) {
  S th[4];
  for (int k = 0; k < 4; ++k) th[k] = theta[k];
  if (base == BMAX2 || base == BMIN2) {
    S e = theta[0];
    for (int k = 1; k < 4; ++k) e = base == BMAX2 ? smax(e, theta[k]) : smin(e, theta[k]);
    for (int k = 0; k < 4; ++k) th[k] = e;
  } else if (base == BX2) {
    for (int k = 0; k < 4; ++k) th[k] = theta_x;
  }
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k) out[i][k] = th[k] * N[i][k] + (S(1) - th[k]) * LDA[i][k];
}

// Range |v|_max - |v|_min of the vertex speeds of a state (Bx sensor, R9).
template <class S>
int speed_range(const std::vector<S>& W, S gamma, S& range) {
  S lo = S(0), hi = S(0);
  for (size_t i = 0; i < W.size() / 4; ++i) {
    S Wi[4] = {W[4 * i], W[4 * i + 1], W[4 * i + 2], W[4 * i + 3]};
    S rho, u, v, p;
    int e = primitive(Wi, gamma, rho, u, v, p);
    if (e) return e;
    S q = sqrt(u * u + v * v);
    lo = i == 0 ? q : smin(lo, q);
    hi = i == 0 ? q : smax(hi, q);
  }
  range = hi - lo;
  return OK;
}

// Bx blending coefficient of triangle t (Sec. 3.3.3, R9) from the vertex
// velocities u_c = rho u / rho, v_c = rho v / rho of the state being distributed.
template <class S>
S bx_theta(const Mesh<S>& m, int32_t t, const S W[3][4], S vrange) {
  if (!(vrange > S(0))) return S(0);
  // div v of the linear interpolant: grad phi_c = n_c / (2 |T|), n_c inward, |n_c| = edge length
  S div = S(0);
  for (int c = 0; c < 3; ++c) {
    S u = W[c][1] / W[c][0], v = W[c][2] / W[c][0];
    div += (u * m.n[6 * (size_t)t + 2 * c] + v * m.n[6 * (size_t)t + 2 * c + 1]) / (S(2) * m.area[t]);
  }
  S sens = -m.L * div / vrange;
  if (!(sens > S(0))) return S(0);
  S h = sqrt(S(2) * m.area[t]);
  return smin(S(1), sens * sens * h / m.L);
}

template <class S>
void tri_W(const Mesh<S>& m, const std::vector<S>& W, int32_t t, S out[3][4]) {
  for (int c = 0; c < 3; ++c)
    for (int k = 0; k < 4; ++k) out[c][k] = W[4 * (size_t)m.tri[3 * t + c] + k];
}

// Stage-1 / forward-Euler residuals: per triangle the share of each node.
template <class S>
int stage1_shares(const Mesh<S>& m, const std::vector<S>& W, S gamma, S eps, int scheme,
                  std::vector<S>& share, int nthreads) {
  const int base = scheme & 0xff;
  std::vector<S> Zv;
  int e = all_Z(m, W, gamma, Zv);
  if (e) return e;
  S vrange = S(0);
  if (base == BX2) {
    e = speed_range(W, gamma, vrange);
    if (e) return e;
  }
  share.assign(12 * (size_t)m.nt, S(0));
  int err = OK;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
  for (int32_t t = 0; t < m.nt; ++t) {
    S Z[3][4], n[3][2];
    tri_Z(m, Zv, t, Z, n);
    TriLin<S> o;
    int le = linearise(Z, n, gamma, eps, o);
    if (le) {
#pragma omp atomic write
      err = le;
      continue;
    }
    S out[3][4];
    if (base == N1 || base == LDA2) {
      for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 4; ++k) out[c][k] = base == N1 ? o.phiN[c][k] : o.phiLDA[c][k];
    } else {
      S thx = S(0);
      if (base == BX2) {
        S Wt[3][4];
        tri_W(m, W, t, Wt);
        thx = bx_theta(m, t, Wt, vrange);
      }
      blend_shares(base, o.theta, thx, o.phiN, o.phiLDA, out);
    }
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) share[12 * (size_t)t + 4 * c + k] = out[c][k];
  }
  return err;
}

// Stage-2 total residuals Phi_i (Sec. 3.4, reading R6).
template <class S>
struct TriStage2 {
  S PhiT[4];
  S PhiN[3][4];
  S PhiLDA[3][4];
  S theta[4];
  S Phi[3][4];
};

template <class S>
int stage2_triangle(const S Zn[3][4], const S Zs[3][4], const S Wn[3][4], const S Ws[3][4],
                    const S n[3][2], S area, S dt, S gamma, S eps, int scheme, TriStage2<S>& o,
                    S theta_x = S(0)) {
  const int base = scheme & 0xff;
  TriLin<S> ln, ls;
  int e = linearise(Zn, n, gamma, eps, ln);
  if (e) return e;
  e = linearise(Zs, n, gamma, eps, ls);
  if (e) return e;
  // Phi_i^N = |T|/3 (W*_i - W^n_i)/dt + (phi_i^N(W*) + phi_i^N(W^n))/2
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 4; ++k)
      o.PhiN[i][k] = area / S(3) * (Ws[i][k] - Wn[i][k]) / dt +
                     (ls.phiN[i][k] + ln.phiN[i][k]) / S(2);
  // Phi_i^LDA = sum_j m_ij^LDA (W*_j - W^n_j)/dt + beta_i/2 (phi(W^n) + phi(W*)),
  // m_ij^LDA = |T|/3 beta_i (eqMassMatrixLDA)
  for (int i = 0; i < 3; ++i) {
    S acc[4] = {S(0), S(0), S(0), S(0)};
    for (int j = 0; j < 3; ++j) {
      S dW[4], t[4];
      for (int k = 0; k < 4; ++k) dW[k] = (Ws[j][k] - Wn[j][k]) / dt;
      S mij[4][4];
      for (int r = 0; r < 4; ++r)
        for (int q = 0; q < 4; ++q) mij[r][q] = area / S(3) * ls.beta[i][r][q];
      matvec(mij, dW, t);
      for (int k = 0; k < 4; ++k) acc[k] += t[k];
    }
    S ph[4], t[4];
    for (int k = 0; k < 4; ++k) ph[k] = (ln.phiT[k] + ls.phiT[k]) / S(2);
    matvec(ls.beta[i], ph, t);
    for (int k = 0; k < 4; ++k) o.PhiLDA[i][k] = acc[k] + t[k];
  }
  // total residual of the triangle
  for (int k = 0; k < 4; ++k) {
    S s = S(0);
    for (int j = 0; j < 3; ++j) s += area / S(3) * (Ws[j][k] - Wn[j][k]) / dt;
    o.PhiT[k] = s + (ln.phiT[k] + ls.phiT[k]) / S(2);
  }
  // blend the total residuals in the same way as Sec. 3.3.3
  for (int k = 0; k < 4; ++k) {
    S num = fabs(o.PhiT[k]);
    S den = smax(fabs(o.PhiN[0][k]) + fabs(o.PhiN[1][k]) + fabs(o.PhiN[2][k]), num);
    o.theta[k] = (base == LDA2 || !(den > S(0))) ? S(0) : num / den;
  }
  blend_shares(base, o.theta, theta_x, o.PhiN, o.PhiLDA, o.Phi);
  // selective lumping: Phi_i += sum_j (|T| delta_ij / 3 - m^G_ij) (W*_j - W^n_j) / dt,
  // m^G_ij = |T| (delta_ij + 1) / 12 (Galerkin mass matrix)
  if (scheme & SELECTIVE_LUMPING) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        S d = i == j ? S(1) : S(0);
        S coef = area * d / S(3) - area * (d + S(1)) / S(12);
        for (int k = 0; k < 4; ++k) o.Phi[i][k] += coef * (Ws[j][k] - Wn[j][k]) / dt;
      }
  }
  return OK;
}

template <class S>
int stage2_shares(const Mesh<S>& m, const std::vector<S>& Wn, const std::vector<S>& Ws, S dt,
                  S gamma, S eps, int scheme, std::vector<S>& share, int nthreads) {
  std::vector<S> Zn, Zs;
  int e = all_Z(m, Wn, gamma, Zn);
  if (e) return e;
  e = all_Z(m, Ws, gamma, Zs);
  if (e) return e;
  S vrange = S(0);
  if ((scheme & 0xff) == BX2) {
    e = speed_range(Ws, gamma, vrange);
    if (e) return e;
  }
  share.assign(12 * (size_t)m.nt, S(0));
  int err = OK;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
  for (int32_t t = 0; t < m.nt; ++t) {
    S zn[3][4], zs[3][4], wn[3][4], ws[3][4], n[3][2];
    tri_Z(m, Zn, t, zn, n);
    tri_Z(m, Zs, t, zs, n);
    for (int c = 0; c < 3; ++c) {
      int32_t v = m.tri[3 * t + c];
      for (int k = 0; k < 4; ++k) {
        wn[c][k] = Wn[4 * (size_t)v + k];
        ws[c][k] = Ws[4 * (size_t)v + k];
      }
    }
    TriStage2<S> o;
    S thx = (scheme & 0xff) == BX2 ? bx_theta(m, t, ws, vrange) : S(0);
    int le = stage2_triangle(zn, zs, wn, ws, n, m.area[t], dt, gamma, eps, scheme, o, thx);
    if (le) {
#pragma omp atomic write
      err = le;
      continue;
    }
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) share[12 * (size_t)t + 4 * c + k] = o.Phi[c][k];
  }
  return err;
}

// Weak reflecting wall (Sec. 3.5): for every wall edge e = (a, b) with outward
// unit normal n, the correction flux F^c n_x + G^c n_y = -(rho v_n, rho u v_n,
// rho v v_n, rho h v_n) at each end, integrated by the trapezium rule and
// split with alpha:  Phi^c_a = |e|/2 (alpha f_a + (1 - alpha) f_b),
// Phi^c_b = |e|/2 ((1 - alpha) f_a + alpha f_b).  Added (times `weight`) to the
// per-vertex residual sums R.
template <class S>
int wall_residual(const Mesh<S>& m, const std::vector<S>& W, S gamma, S weight, std::vector<S>& R) {
  for (size_t w = 0; w < m.wall.size() / 2; ++w) {
    int32_t t = m.wall[2 * w], c = m.wall[2 * w + 1];
    int32_t a = m.tri[3 * (size_t)t + (c + 1) % 3], b = m.tri[3 * (size_t)t + (c + 2) % 3];
    S nx = -m.n[6 * (size_t)t + 2 * c], ny = -m.n[6 * (size_t)t + 2 * c + 1];
    S len = sqrt(nx * nx + ny * ny);
    nx = nx / len;
    ny = ny / len;
    S f[2][4];
    int32_t ends[2] = {a, b};
    for (int q = 0; q < 2; ++q) {
      const S* Wi = &W[4 * (size_t)ends[q]];
      S Wv[4] = {Wi[0], Wi[1], Wi[2], Wi[3]};
      S rho, u, v, p;
      int e = primitive(Wv, gamma, rho, u, v, p);
      if (e) return e;
      S vn = u * nx + v * ny;
      S h = (Wv[3] + p) / rho;
      f[q][0] = -rho * vn;
      f[q][1] = -rho * u * vn;
      f[q][2] = -rho * v * vn;
      f[q][3] = -rho * h * vn;
    }
    for (int k = 0; k < 4; ++k) {
      R[4 * (size_t)a + k] += weight * len / S(2) * (m.alpha * f[0][k] + (S(1) - m.alpha) * f[1][k]);
      R[4 * (size_t)b + k] += weight * len / S(2) * ((S(1) - m.alpha) * f[0][k] + m.alpha * f[1][k]);
    }
  }
  return OK;
}

// W_i <- W_i - dt/V_i sum_{T containing i} share_i   (eqUpdate, eqRK1, eqRK2)
template <class S>
void apply_update(const Mesh<S>& m, const std::vector<S>& Win, const std::vector<S>& share, S dt,
                  std::vector<S>& Wout, const std::vector<S>* extra = nullptr) {
  std::vector<S> R(4 * (size_t)m.nv, S(0));
  for (int32_t t = 0; t < m.nt; ++t)
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) R[4 * (size_t)m.tri[3 * t + c] + k] += share[12 * (size_t)t + 4 * c + k];
  if (extra)
    for (size_t i = 0; i < R.size(); ++i) R[i] += (*extra)[i];
  Wout.resize(Win.size());
  for (int32_t i = 0; i < m.nv; ++i)
    for (int k = 0; k < 4; ++k)
      Wout[4 * (size_t)i + k] = Win[4 * (size_t)i + k] - dt / m.V[i] * R[4 * (size_t)i + k];
}

// One full time step.  N1: forward Euler with the N scheme.  B2 / LDA2: the
// two-stage scheme (eqRK1, eqRK2).  dt_fixed > 0 overrides the CFL step.
template <class S>
int step(const Mesh<S>& m, std::vector<S>& W, S gamma, S cfl, S eps, int scheme, S dt_fixed,
         S& dt, int nthreads) {
  const int base = scheme & 0xff;
  if (base < N1 || base > BX2 || (scheme & ~(0xff | SELECTIVE_LUMPING))) return EINVAL;
  if (base == N1 && (scheme & SELECTIVE_LUMPING)) return EINVAL;
  if (dt_fixed > S(0)) {
    dt = dt_fixed;
  } else {
    int e = time_step(m, W, gamma, cfl, dt);
    if (e) return e;
  }
  std::vector<S> share, Ws, Wn1;
  int e = stage1_shares(m, W, gamma, eps, scheme, share, nthreads);
  if (e) return e;
  std::vector<S> wall_n, wall_2;
  if (!m.wall.empty()) {
    wall_n.assign(W.size(), S(0));
    e = wall_residual(m, W, gamma, S(1), wall_n);
    if (e) return e;
  }
  apply_update(m, W, share, dt, Ws, m.wall.empty() ? nullptr : &wall_n);
  if (base == N1) {
    W.swap(Ws);
    return OK;
  }
  e = stage2_shares(m, W, Ws, dt, gamma, eps, scheme, share, nthreads);
  if (e) return e;
  if (!m.wall.empty()) {
    // (Phi^c(W^n) + Phi^c(W*)) / 2   (R13)
    wall_2.assign(W.size(), S(0));
    e = wall_residual(m, W, gamma, S(0.5), wall_2);
    if (e) return e;
    e = wall_residual(m, Ws, gamma, S(0.5), wall_2);
    if (e) return e;
  }
  apply_update(m, Ws, share, dt, Wn1, m.wall.empty() ? nullptr : &wall_2);
  W.swap(Wn1);
  return OK;
}

// SoA (component-major) <-> AoS conversions for the C interface.
template <class S>
void soa_to_aos(const double* Wsoa, int32_t nv, std::vector<S>& W) {
  W.resize(4 * (size_t)nv);
  for (int32_t i = 0; i < nv; ++i)
    for (int k = 0; k < 4; ++k) W[4 * (size_t)i + k] = S(Wsoa[(size_t)k * nv + i]);
}
template <class S>
void aos_to_soa(const std::vector<S>& W, int32_t nv, double* Wsoa) {
  for (int32_t i = 0; i < nv; ++i)
    for (int k = 0; k < 4; ++k) Wsoa[(size_t)k * nv + i] = val(W[4 * (size_t)i + k]);
}

// Boundary description for run(): ghost [nv] (nullable), n_wall (triangle, corner) pairs.
struct Boundary {
  const uint8_t* ghost = nullptr;
  int32_t n_wall = 0;
  const int32_t* wall = nullptr;
  double alpha = 0.75;
};

template <class S>
int set_boundary(Mesh<S>& m, const Boundary* bc) {
  if (!bc) return OK;
  if (bc->ghost) m.ghost.assign(bc->ghost, bc->ghost + m.nv);
  for (int32_t w = 0; w < bc->n_wall; ++w) {
    int32_t t = bc->wall[2 * w], c = bc->wall[2 * w + 1];
    if (t < 0 || t >= m.nt || c < 0 || c > 2) return EINVAL;
  }
  m.wall.assign(bc->wall, bc->wall + 2 * (size_t)bc->n_wall);
  m.alpha = S(bc->alpha);
  return OK;
}

template <class S>
int run(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift, double Lx,
        double Ly, double* W_soa, int scheme, double cfl, double gamma, double eps, int32_t nsteps,
        const double* dt_fixed, double* dt_out, int nthreads, const Boundary* bc = nullptr) {
  Mesh<S> m;
  int e = build_mesh(nv, xy, nt, tri, shift, Lx, Ly, m);
  if (e) return e;
  e = set_boundary(m, bc);
  if (e) return e;
  std::vector<S> W;
  soa_to_aos(W_soa, nv, W);
  const std::vector<S> W0 = W;
  for (int32_t s = 0; s < nsteps; ++s) {
    // ghost vertices enter every step at their initial state (R12)
    if (!m.ghost.empty())
      for (int32_t i = 0; i < nv; ++i)
        if (m.ghost[i])
          for (int k = 0; k < 4; ++k) W[4 * (size_t)i + k] = W0[4 * (size_t)i + k];
    S dt;
    e = step(m, W, S(gamma), S(cfl), S(eps), scheme, dt_fixed ? S(dt_fixed[s]) : S(0), dt, nthreads);
    if (e) return e;
    if (dt_out) dt_out[s] = val(dt);
  }
  if (!m.ghost.empty())
    for (int32_t i = 0; i < nv; ++i)
      if (m.ghost[i])
        for (int k = 0; k < 4; ++k) W[4 * (size_t)i + k] = W0[4 * (size_t)i + k];
  aos_to_soa(W, nv, W_soa);
  return OK;
}

}  // namespace ora

// ===========================================================================
// C interface (ctypes).  W arrays are component-major: W[k * nv + i].
// xy: [nv][2], tri: [nt][3], shift: [nt][3][2] in periods (nullable).
// ===========================================================================
extern "C" {

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Advance W by nsteps full steps in double precision.  dt_fixed (nullable):
// per-step dt to use instead of the CFL step.  dt_out (nullable): dt of each step.
int ora_run(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift,
            double Lx, double Ly, double* W, int scheme, double cfl, double gamma, double eps,
            int32_t nsteps, const double* dt_fixed, double* dt_out, int nthreads) {
  return ora::run<double>(nv, xy, nt, tri, shift, Lx, Ly, W, scheme, cfl, gamma, eps, nsteps,
                          dt_fixed, dt_out, nthreads);
}

// Same in long double (round-off floor of the double oracle).
int ora_run_ld(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift,
               double Lx, double Ly, double* W, int scheme, double cfl, double gamma, double eps,
               int32_t nsteps, const double* dt_fixed, double* dt_out, int nthreads) {
  return ora::run<long double>(nv, xy, nt, tri, shift, Lx, Ly, W, scheme, cfl, gamma, eps, nsteps,
                               dt_fixed, dt_out, nthreads);
}

// Same as ora_run / ora_run_ld with boundary conditions (Sec. 3.5): ghost [nv]
// (nullable, 1 = held at the initial state), n_wall edges given as (triangle,
// corner) pairs naming the edge opposite the corner, alpha the wall split.
int ora_run_bc(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift,
               double Lx, double Ly, double* W, int scheme, double cfl, double gamma, double eps,
               int32_t nsteps, const double* dt_fixed, double* dt_out, int nthreads, const uint8_t* ghost,
               int32_t n_wall, const int32_t* wall, double alpha, int long_double) {
  ora::Boundary bc;
  bc.ghost = ghost;
  bc.n_wall = n_wall;
  bc.wall = wall;
  bc.alpha = alpha;
  if (long_double)
    return ora::run<long double>(nv, xy, nt, tri, shift, Lx, Ly, W, scheme, cfl, gamma, eps, nsteps, dt_fixed,
                                 dt_out, nthreads, &bc);
  return ora::run<double>(nv, xy, nt, tri, shift, Lx, Ly, W, scheme, cfl, gamma, eps, nsteps, dt_fixed, dt_out,
                          nthreads, &bc);
}

// Directional derivative of nsteps with a frozen dt sequence (dt_fixed, required):
// W (in/out, values) and dW (in/out, tangent) are both component-major.
int ora_run_tangent(int32_t nv, const double* xy, int32_t nt, const int32_t* tri,
                    const int8_t* shift, double Lx, double Ly, double* W, double* dW, int scheme,
                    double gamma, double eps, int32_t nsteps, const double* dt_fixed,
                    int nthreads) {
  if (!dt_fixed) return ora::EINVAL;
  ora::Mesh<ora::Dual> m;
  int e = ora::build_mesh(nv, xy, nt, tri, shift, Lx, Ly, m);
  if (e) return e;
  std::vector<ora::Dual> Wd(4 * (size_t)nv);
  for (int32_t i = 0; i < nv; ++i)
    for (int k = 0; k < 4; ++k)
      Wd[4 * (size_t)i + k] = ora::Dual(W[(size_t)k * nv + i], dW[(size_t)k * nv + i]);
  for (int32_t s = 0; s < nsteps; ++s) {
    ora::Dual dt;
    e = ora::step(m, Wd, ora::Dual(gamma), ora::Dual(0.0), ora::Dual(eps), scheme,
                  ora::Dual(dt_fixed[s]), dt, nthreads);
    if (e) return e;
  }
  for (int32_t i = 0; i < nv; ++i)
    for (int k = 0; k < 4; ++k) {
      W[(size_t)k * nv + i] = Wd[4 * (size_t)i + k].v;
      dW[(size_t)k * nv + i] = Wd[4 * (size_t)i + k].d;
    }
  return ora::OK;
}

// One operation of the dual-number type on scalars, for the closed-form unit
// checks of its derivative rules: op 0 a+b, 1 a-b, 2 a*b, 3 a/b, 4 sqrt(a),
// 5 |a|, 6 -a.  out = (value, derivative).
int ora_dual_eval(int op, double av, double ad, double bv, double bd, double* out) {
  const ora::Dual a(av, ad), b(bv, bd);
  ora::Dual r;
  switch (op) {
    case 0: r = a + b; break;
    case 1: r = a - b; break;
    case 2: r = a * b; break;
    case 3: r = a / b; break;
    case 4: r = ora::sqrt(a); break;
    case 5: r = ora::fabs(a); break;
    case 6: r = -a; break;
    default: return ora::EINVAL;
  }
  out[0] = r.v;
  out[1] = r.d;
  return ora::OK;
}

// CFL time step of state W.
int ora_time_step(int32_t nv, const double* xy, int32_t nt, const int32_t* tri,
                  const int8_t* shift, double Lx, double Ly, const double* W, double cfl,
                  double gamma, double* dt) {
  ora::Mesh<double> m;
  int e = ora::build_mesh(nv, xy, nt, tri, shift, Lx, Ly, m);
  if (e) return e;
  std::vector<double> Wv;
  ora::soa_to_aos(W, nv, Wv);
  return ora::time_step(m, Wv, gamma, cfl, *dt);
}

// Nodal volumes V_i (reading R7), per-triangle area and longest edge.
int ora_geometry(int32_t nv, const double* xy, int32_t nt, const int32_t* tri,
                 const int8_t* shift, double Lx, double Ly, double* V, double* area, double* lmax,
                 double* normals /*[nt][3][2]*/) {
  ora::Mesh<double> m;
  int e = ora::build_mesh(nv, xy, nt, tri, shift, Lx, Ly, m);
  if (e) return e;
  if (V) std::memcpy(V, m.V.data(), sizeof(double) * nv);
  if (area) std::memcpy(area, m.area.data(), sizeof(double) * nt);
  if (lmax) std::memcpy(lmax, m.lmax.data(), sizeof(double) * nt);
  if (normals) std::memcpy(normals, m.n.data(), sizeof(double) * 6 * (size_t)nt);
  return ora::OK;
}

}  // extern "C"

template <class S>
int triangle_terms_impl(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift,
                        double Lx, double Ly, const double* W, double gamma, double eps, double* phiT,
                        double* phiN, double* phiLDA, double* phiB) {
  ora::Mesh<S> m;
  int e = ora::build_mesh(nv, xy, nt, tri, shift, Lx, Ly, m);
  if (e) return e;
  std::vector<S> Wv, Zv;
  ora::soa_to_aos(W, nv, Wv);
  e = ora::all_Z(m, Wv, S(gamma), Zv);
  if (e) return e;
  for (int32_t t = 0; t < nt; ++t) {
    S Z[3][4], n[3][2];
    ora::tri_Z(m, Zv, t, Z, n);
    ora::TriLin<S> o;
    e = ora::linearise(Z, n, S(gamma), S(eps), o);
    if (e) return e;
    for (int k = 0; k < 4; ++k)
      if (phiT) phiT[4 * (size_t)t + k] = ora::val(o.phiT[k]);
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) {
        size_t ix = 12 * (size_t)t + 4 * c + k;
        if (phiN) phiN[ix] = ora::val(o.phiN[c][k]);
        if (phiLDA) phiLDA[ix] = ora::val(o.phiLDA[c][k]);
        if (phiB) phiB[ix] = ora::val(o.phiB[c][k]);
      }
  }
  return ora::OK;
}

extern "C" {

// Stage-1 shares evaluated in long double (round-off floor of the per-triangle terms).
int ora_triangle_terms_ld(int32_t nv, const double* xy, int32_t nt, const int32_t* tri,
                          const int8_t* shift, double Lx, double Ly, const double* W, double gamma,
                          double eps, double* phiT, double* phiN, double* phiLDA, double* phiB) {
  return triangle_terms_impl<long double>(nv, xy, nt, tri, shift, Lx, Ly, W, gamma, eps, phiT, phiN,
                                          phiLDA, phiB);
}

// Stage-1 quantities of every triangle at state W (component-major):
// phiT [nt][4], phiN/phiLDA/phiB [nt][3][4], beta [nt][3][4][4], theta [nt][4],
// Kp/Km [nt][3][4][4].  Any output pointer may be NULL.
int ora_triangle_terms(int32_t nv, const double* xy, int32_t nt, const int32_t* tri,
                       const int8_t* shift, double Lx, double Ly, const double* W, double gamma,
                       double eps, double* phiT, double* phiN, double* phiLDA, double* phiB,
                       double* beta, double* theta, double* Kp, double* Km) {
  ora::Mesh<double> m;
  int e = ora::build_mesh(nv, xy, nt, tri, shift, Lx, Ly, m);
  if (e) return e;
  std::vector<double> Wv, Zv;
  ora::soa_to_aos(W, nv, Wv);
  e = ora::all_Z(m, Wv, gamma, Zv);
  if (e) return e;
  for (int32_t t = 0; t < nt; ++t) {
    double Z[3][4], n[3][2];
    ora::tri_Z(m, Zv, t, Z, n);
    ora::TriLin<double> o;
    e = ora::linearise(Z, n, gamma, eps, o);
    if (e) return e;
    for (int k = 0; k < 4; ++k) {
      if (phiT) phiT[4 * (size_t)t + k] = o.phiT[k];
      if (theta) theta[4 * (size_t)t + k] = o.theta[k];
    }
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) {
        size_t ix = 12 * (size_t)t + 4 * c + k;
        if (phiN) phiN[ix] = o.phiN[c][k];
        if (phiLDA) phiLDA[ix] = o.phiLDA[c][k];
        if (phiB) phiB[ix] = o.phiB[c][k];
      }
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < 4; ++r)
        for (int q = 0; q < 4; ++q) {
          size_t ix = 48 * (size_t)t + 16 * c + 4 * r + q;
          if (beta) beta[ix] = o.beta[c][r][q];
          if (Kp) Kp[ix] = o.Kp[c][r][q];
          if (Km) Km[ix] = o.Km[c][r][q];
        }
  }
  return ora::OK;
}

// Stage-2 total residuals of every triangle for states Wn, Ws and step dt:
// PhiT [nt][4], PhiN/PhiLDA/Phi [nt][3][4], theta [nt][4].  Outputs nullable.
int ora_stage2_terms(int32_t nv, const double* xy, int32_t nt, const int32_t* tri,
                     const int8_t* shift, double Lx, double Ly, const double* Wn,
                     const double* Ws, double dt, double gamma, double eps, int scheme,
                     double* PhiT, double* PhiN, double* PhiLDA, double* Phi, double* theta);
int ora_stage2_terms_ld(int32_t nv, const double* xy, int32_t nt, const int32_t* tri,
                        const int8_t* shift, double Lx, double Ly, const double* Wn,
                        const double* Ws, double dt, double gamma, double eps, int scheme,
                        double* PhiT, double* PhiN, double* PhiLDA, double* Phi, double* theta);

}  // extern "C"

template <class S>
int stage2_terms_impl(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift, double Lx,
                      double Ly, const double* Wn, const double* Ws, double dt_d, double gamma_d, double eps_d,
                      int scheme, double* PhiT, double* PhiN, double* PhiLDA, double* Phi, double* theta) {
  ora::Mesh<S> m;
  int e = ora::build_mesh(nv, xy, nt, tri, shift, Lx, Ly, m);
  if (e) return e;
  const S dt = S(dt_d), gamma = S(gamma_d), eps = S(eps_d);
  std::vector<S> Wnv, Wsv, Zn, Zs;
  ora::soa_to_aos(Wn, nv, Wnv);
  ora::soa_to_aos(Ws, nv, Wsv);
  e = ora::all_Z(m, Wnv, gamma, Zn);
  if (e) return e;
  e = ora::all_Z(m, Wsv, gamma, Zs);
  if (e) return e;
  S vrange = S(0);
  if ((scheme & 0xff) == ora::BX2) {
    e = ora::speed_range(Wsv, gamma, vrange);
    if (e) return e;
  }
  for (int32_t t = 0; t < nt; ++t) {
    S zn[3][4], zs[3][4], wn[3][4], ws[3][4], n[3][2];
    ora::tri_Z(m, Zn, t, zn, n);
    ora::tri_Z(m, Zs, t, zs, n);
    for (int c = 0; c < 3; ++c) {
      int32_t v = m.tri[3 * t + c];
      for (int k = 0; k < 4; ++k) {
        wn[c][k] = Wnv[4 * (size_t)v + k];
        ws[c][k] = Wsv[4 * (size_t)v + k];
      }
    }
    ora::TriStage2<S> o;
    S thx = (scheme & 0xff) == ora::BX2 ? ora::bx_theta(m, t, ws, vrange) : S(0);
    e = ora::stage2_triangle(zn, zs, wn, ws, n, m.area[t], dt, gamma, eps, scheme, o, thx);
    if (e) return e;
    for (int k = 0; k < 4; ++k) {
      if (PhiT) PhiT[4 * (size_t)t + k] = ora::val(o.PhiT[k]);
      if (theta) theta[4 * (size_t)t + k] = ora::val(o.theta[k]);
    }
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) {
        size_t ix = 12 * (size_t)t + 4 * c + k;
        if (PhiN) PhiN[ix] = ora::val(o.PhiN[c][k]);
        if (PhiLDA) PhiLDA[ix] = ora::val(o.PhiLDA[c][k]);
        if (Phi) Phi[ix] = ora::val(o.Phi[c][k]);
      }
  }
  return ora::OK;
}

extern "C" {
int ora_stage2_terms(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift, double Lx,
                     double Ly, const double* Wn, const double* Ws, double dt, double gamma, double eps, int scheme,
                     double* PhiT, double* PhiN, double* PhiLDA, double* Phi, double* theta) {
  return stage2_terms_impl<double>(nv, xy, nt, tri, shift, Lx, Ly, Wn, Ws, dt, gamma, eps, scheme, PhiT, PhiN,
                                   PhiLDA, Phi, theta);
}
int ora_stage2_terms_ld(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift,
                        double Lx, double Ly, const double* Wn, const double* Ws, double dt, double gamma,
                        double eps, int scheme, double* PhiT, double* PhiN, double* PhiLDA, double* Phi,
                        double* theta) {
  return stage2_terms_impl<long double>(nv, xy, nt, tri, shift, Lx, Ly, Wn, Ws, dt, gamma, eps, scheme, PhiT,
                                        PhiN, PhiLDA, Phi, theta);
}
}  // extern "C"

template <class S>
int stage1_shares_impl(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift,
                       double Lx, double Ly, const double* W, double gamma, double eps, int scheme,
                       double* out, int nthreads) {
  ora::Mesh<S> m;
  int e = ora::build_mesh(nv, xy, nt, tri, shift, Lx, Ly, m);
  if (e) return e;
  std::vector<S> Wv, share;
  ora::soa_to_aos(W, nv, Wv);
  e = ora::stage1_shares(m, Wv, S(gamma), S(eps), scheme, share, nthreads);
  if (e) return e;
  for (size_t i = 0; i < share.size(); ++i) out[i] = ora::val(share[i]);
  return ora::OK;
}

extern "C" {

// Stage-1 (forward-Euler) shares of any scheme code at state W: out [nt][3][4].
int ora_stage1_shares(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift,
                      double Lx, double Ly, const double* W, double gamma, double eps, int scheme,
                      double* out, int nthreads) {
  return stage1_shares_impl<double>(nv, xy, nt, tri, shift, Lx, Ly, W, gamma, eps, scheme, out, nthreads);
}
int ora_stage1_shares_ld(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift,
                         double Lx, double Ly, const double* W, double gamma, double eps, int scheme,
                         double* out, int nthreads) {
  return stage1_shares_impl<long double>(nv, xy, nt, tri, shift, Lx, Ly, W, gamma, eps, scheme, out,
                                         nthreads);
}

// App. A pieces at one state and unit normal, for the algebra pins:
// K [4][4], lam [4], R [4][4] (columns = right eigenvectors), L = R^{-1} [4][4].
int ora_eigensystem(double u, double v, double h, double gamma, double nx, double ny, double* K,
                    double* lam, double* R, double* L) {
  double c2 = (gamma - 1) * (h - (u * u + v * v) / 2);
  if (!(c2 > 0)) return ora::ENONPHYS;
  double c = std::sqrt(c2);
  double Km[4][4], Rm[4][4], Lm[4][4];
  ora::K_matrix(u, v, h, gamma, nx, ny, Km);
  ora::eigen_R(u, v, h, c, gamma, nx, ny, lam, Rm);
  if (ora::invert4(Rm, Lm)) return ora::ENONPHYS;
  std::memcpy(K, Km, sizeof(Km));
  std::memcpy(R, Rm, sizeof(Rm));
  std::memcpy(L, Lm, sizeof(Lm));
  return ora::OK;
}

// Sum_i V_i W_i in double, in vertex order.
int ora_conserved(int32_t nv, const double* xy, int32_t nt, const int32_t* tri, const int8_t* shift,
                  double Lx, double Ly, const double* W, double* out4) {
  ora::Mesh<double> m;
  int e = ora::build_mesh(nv, xy, nt, tri, shift, Lx, Ly, m);
  if (e) return e;
  for (int k = 0; k < 4; ++k) {
    double s = 0;
    for (int32_t i = 0; i < nv; ++i) s += m.V[i] * W[(size_t)k * nv + i];
    out4[k] = s;
  }
  return ora::OK;
}

}  // extern "C"
