// Host build of the adjoint's per-triangle reverse code (the functions the
// reverse kernels call), checked by the dot-product test against central
// differences of the forward per-triangle code, for the CPU test suite.
//
// For n seeded random triangles (geometry, corner states) and random output
// adjoints and input directions, prints one line per scheme and stage:
//   <scheme> <stage> checked <k> skipped <s> max_rel <e>
// where e = max over triangles of |<out_bar, J dx> - <J^T out_bar, dx>| /
// (|<out_bar, J dx>| + |J^T out_bar| |dx|) with J dx from central differences
// (step 1e-6); triangles whose branch mask changes within the step are skipped.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

#include "rd_adjoint.cuh"

using namespace rd;

struct Tri {
  double nx[3], ny[3], hl[3], area;
  double W[3][4], Ws[3][4];
};

static void make_tri(std::mt19937_64& g, Tri& t) {
  std::uniform_real_distribution<double> U(0.0, 1.0);
  double x[3], y[3];
  for (;;) {
    for (int c = 0; c < 3; ++c) {
      x[c] = U(g);
      y[c] = U(g);
    }
    const double A = 0.5 * ((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]));
    if (A > 0.02) {
      t.area = A;
      break;
    }
  }
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    const double nxx = y[a] - y[b], nyy = x[b] - x[a], len = std::sqrt(nxx * nxx + nyy * nyy);
    t.nx[c] = nxx / len;
    t.ny[c] = nyy / len;
    t.hl[c] = len / 2.0;
  }
  const double gamma = 1.4;
  // a smooth field sampled at the corners, and W* = a nearby state
  const double r0 = 0.5 + 1.5 * U(g), u0 = 2.0 * U(g) - 1.0, v0 = 2.0 * U(g) - 1.0, p0 = 0.5 + 1.5 * U(g);
  for (int c = 0; c < 3; ++c) {
    const double rho = r0 * (1 + 0.2 * (U(g) - 0.5)), u = u0 + 0.2 * (U(g) - 0.5), v = v0 + 0.2 * (U(g) - 0.5);
    const double p = p0 * (1 + 0.2 * (U(g) - 0.5));
    t.W[c][0] = rho;
    t.W[c][1] = rho * u;
    t.W[c][2] = rho * v;
    t.W[c][3] = p / (gamma - 1) + 0.5 * rho * (u * u + v * v);
    const double f = 1 + 1e-2 * (U(g) - 0.5);
    for (int k = 0; k < 4; ++k) t.Ws[c][k] = t.W[c][k] * f;
  }
}

template <int SCHEME>
static void check(int n, unsigned long long seed) {
  const double gamma = 1.4, eps = 1e-6, dt = 1e-2, h = 1e-6;
  std::mt19937_64 g(seed);
  std::normal_distribution<double> N01(0.0, 1.0);
  int ok1 = 0, skip1 = 0, ok2 = 0, skip2 = 0;
  double e1 = 0.0, e2 = 0.0;
  for (int it = 0; it < n; ++it) {
    Tri t;
    make_tri(g, t);
    double Z[3][4], Zs[3][4], sp;
    for (int c = 0; c < 3; ++c) {
      vertex_Z(t.W[c], gamma, Z[c], sp);
      vertex_Z(t.Ws[c], gamma, Zs[c], sp);
    }
    // stage 1: Z -> (shares, record)
    {
      double dZ[3][4], ob[3][4], rb[16], Zp[3][4], Zm[3][4], op[3][4], om[3][4], rp[16], rm[16], Zbar[3][4];
      for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 4; ++k) {
          dZ[c][k] = N01(g);
          ob[c][k] = N01(g);
          Zp[c][k] = Z[c][k] + h * dZ[c][k];
          Zm[c][k] = Z[c][k] - h * dZ[c][k];
        }
      for (int k = 0; k < 16; ++k) rb[k] = SCHEME == RD_N1 ? 0.0 : N01(g);
      const Mask m0 = stage1_mask<double, SCHEME>(Z, t.nx, t.ny, t.hl, gamma, eps);
      if (stage1_mask<double, SCHEME>(Zp, t.nx, t.ny, t.hl, gamma, eps) != m0 ||
          stage1_mask<double, SCHEME>(Zm, t.nx, t.ny, t.hl, gamma, eps) != m0) {
        ++skip1;
      } else if (!stage1_body<double, SCHEME>(Zp, t.nx, t.ny, t.hl, gamma, eps, op, rp) &&
                 !stage1_body<double, SCHEME>(Zm, t.nx, t.ny, t.hl, gamma, eps, om, rm) &&
                 !stage1_rev<double, SCHEME>(Z, t.nx, t.ny, t.hl, gamma, eps, m0, ob, rb, Zbar)) {
        double lhs = 0.0, rhs = 0.0, nb = 0.0, nd = 0.0;
        for (int c = 0; c < 3; ++c)
          for (int k = 0; k < 4; ++k) {
            lhs += ob[c][k] * (op[c][k] - om[c][k]) / (2 * h);
            rhs += Zbar[c][k] * dZ[c][k];
            nb += Zbar[c][k] * Zbar[c][k];
            nd += dZ[c][k] * dZ[c][k];
          }
        if (SCHEME != RD_N1)
          for (int k = 0; k < 16; ++k) lhs += rb[k] * (rp[k] - rm[k]) / (2 * h);
        e1 = std::fmax(e1, std::fabs(lhs - rhs) / (std::fabs(lhs) + std::sqrt(nb * nd)));
        ++ok1;
      }
    }
    if (SCHEME == RD_N1) continue;
    // stage 2: (Z*, W^n, W*, record) -> shares
    {
      double rec[16], s1[3][4];
      if (stage1_body<double, SCHEME>(Z, t.nx, t.ny, t.hl, gamma, eps, s1, rec)) continue;
      double dZs[3][4], dWn[3][4], dWs[3][4], drec[16], ob[3][4];
      for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 4; ++k) {
          dZs[c][k] = N01(g);
          dWn[c][k] = N01(g) * 1e-2;
          dWs[c][k] = N01(g) * 1e-2;
          ob[c][k] = N01(g);
        }
      for (int k = 0; k < 16; ++k) drec[k] = N01(g) * 1e-2;
      double o[2][3][4];
      Mask ms[2];
      for (int s = 0; s < 2; ++s) {
        const double sg = s == 0 ? h : -h;
        double a[3][4], b[3][4], c2[3][4], r[16];
        for (int c = 0; c < 3; ++c)
          for (int k = 0; k < 4; ++k) {
            a[c][k] = Zs[c][k] + sg * dZs[c][k];
            b[c][k] = t.W[c][k] + sg * dWn[c][k];
            c2[c][k] = t.Ws[c][k] + sg * dWs[c][k];
          }
        for (int k = 0; k < 16; ++k) r[k] = rec[k] + sg * drec[k];
        ms[s] = stage2_mask<double, SCHEME>(a, b, c2, r, t.nx, t.ny, t.hl, t.area, dt, gamma, eps);
        stage2_body<double, SCHEME>(a, b, c2, r, t.nx, t.ny, t.hl, t.area, dt, gamma, eps, o[s]);
      }
      const Mask m0 = stage2_mask<double, SCHEME>(Zs, t.W, t.Ws, rec, t.nx, t.ny, t.hl, t.area, dt, gamma, eps);
      double Zsb[3][4], Wnb[3][4], Wsb[3][4], recb[16];
      if (ms[0] != m0 || ms[1] != m0) {
        ++skip2;
      } else if (!stage2_rev<double, SCHEME>(Zs, t.W, t.Ws, rec, t.nx, t.ny, t.hl, t.area, dt, gamma, eps, m0, ob,
                                             Zsb, Wnb, Wsb, recb)) {
        double lhs = 0.0, rhs = 0.0, nb = 0.0, nd = 0.0;
        for (int c = 0; c < 3; ++c)
          for (int k = 0; k < 4; ++k) {
            lhs += ob[c][k] * (o[0][c][k] - o[1][c][k]) / (2 * h);
            rhs += Zsb[c][k] * dZs[c][k] + Wnb[c][k] * dWn[c][k] + Wsb[c][k] * dWs[c][k];
            nb += Zsb[c][k] * Zsb[c][k] + Wnb[c][k] * Wnb[c][k] + Wsb[c][k] * Wsb[c][k];
            nd += dZs[c][k] * dZs[c][k] + dWn[c][k] * dWn[c][k] + dWs[c][k] * dWs[c][k];
          }
        for (int k = 0; k < 16; ++k) {
          rhs += recb[k] * drec[k];
          nb += recb[k] * recb[k];
          nd += drec[k] * drec[k];
        }
        e2 = std::fmax(e2, std::fabs(lhs - rhs) / (std::fabs(lhs) + std::sqrt(nb * nd)));
        ++ok2;
      }
    }
  }
  const char* name = SCHEME == RD_N1 ? "N1" : SCHEME == RD_B2 ? "B2" : "LDA2";
  std::printf("%s 1 checked %d skipped %d max_rel %.3e\n", name, ok1, skip1, e1);
  if (SCHEME != RD_N1) std::printf("%s 2 checked %d skipped %d max_rel %.3e\n", name, ok2, skip2, e2);
}

int main(int argc, char** argv) {
  const int n = argc > 1 ? std::atoi(argv[1]) : 500;
  check<RD_N1>(n, 1);
  check<RD_B2>(n, 2);
  check<RD_LDA2>(n, 3);
  return 0;
}
