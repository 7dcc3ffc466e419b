// Host build of the triangle kernels' per-triangle code (the same functions the
// CUDA kernels run, compiled for the CPU), for the CPU test that holds them to
// the oracle's per-triangle shares without a GPU.  Scheme codes + 16 select the
// double-float bodies of the RD_DF64 kernels (Zbar, Z_i - Zbar and W*_i - W^n_i
// formed in double, the rest in double-float), as rd_df64_kernels.cuh calls them.
//
// Input (binary): nv, nt, Lx, Ly, has_shift, xy, tri, shift as in
// tile_plan_check.cpp, then gamma, eps, dt (double), scheme (int32: 0 N1,
// 1 B2, 2 LDA2), W^n and W* ([4][nv] double, component-major, caller order).
// Output (binary): stage-1 shares [nt][3][4], then (two-stage schemes) the
// stage-2 shares [nt][3][4], both in the caller's triangle and corner order.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "rd_dfloat.cuh"
#include "rd_internal.h"
#include "rd_kernels.cuh"

template <int SCHEME>
static int run_df(const rd::HostMesh& h, const std::vector<double>& Wn, const std::vector<double>& Ws, double gamma,
                  double eps, double dt, std::vector<double>& s1, std::vector<double>& s2) {
  using rd::dfloat;
  const int nt = h.nt, nv = h.nv;
  rd::Gas<dfloat> gas;
  gas.gamma = dfloat(gamma);
  gas.g1 = dfloat(gamma - 1.0);
  gas.g = dfloat((gamma - 1.0) / gamma);
  gas.ig = dfloat(1.0 / gamma);
  for (int t = 0; t < nt; ++t) {
    double Zn[3][4], Zs[3][4], wn[3][4], ws[3][4];
    dfloat nx[3], ny[3], hl[3];
    for (int c = 0; c < 3; ++c) {
      const int vi = h.tri[(size_t)c * nt + t], vc = h.vperm[vi];
      for (int k = 0; k < 4; ++k) {
        wn[c][k] = Wn[(size_t)k * nv + vc];
        ws[c][k] = Ws[(size_t)k * nv + vc];
      }
      double sp;
      if (!rd::vertex_Z(wn[c], gamma, Zn[c], sp) || !rd::vertex_Z(ws[c], gamma, Zs[c], sp)) return 2;
      nx[c] = dfloat(h.nx[(size_t)c * nt + t]);
      ny[c] = dfloat(h.ny[(size_t)c * nt + t]);
      hl[c] = dfloat(h.hl[(size_t)c * nt + t]);
    }
    dfloat Zb[4], dZ[3][4], Zbs[4], dZs[3][4], dW[3][4], out[3][4], rec[16];
    for (int k = 0; k < 4; ++k) {
      const double zb = (Zn[0][k] + Zn[1][k] + Zn[2][k]) * (1.0 / 3.0);
      const double zs = (Zs[0][k] + Zs[1][k] + Zs[2][k]) * (1.0 / 3.0);
      Zb[k] = dfloat(zb);
      Zbs[k] = dfloat(zs);
      for (int c = 0; c < 3; ++c) {
        dZ[c][k] = dfloat(Zn[c][k] - zb);
        dZs[c][k] = dfloat(Zs[c][k] - zs);
        dW[c][k] = dfloat(ws[c][k] - wn[c][k]);
      }
    }
    if (rd::stage1_body_d<dfloat, SCHEME>(Zb, dZ, nx, ny, hl, gas, dfloat(eps), out, rec)) return 3;
    const size_t tc = (size_t)h.tperm[t];
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) s1[12 * tc + 4 * c + k] = (double)out[c][k];
    if (SCHEME == RD_N1) continue;
    if (rd::stage2_body_d<dfloat, SCHEME>(Zbs, dZs, dW, rec, nx, ny, hl, dfloat(h.area[t]), dfloat(dt), gas,
                                          dfloat(eps), out))
      return 4;
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) s2[12 * tc + 4 * c + k] = (double)out[c][k];
  }
  return 0;
}

template <int SCHEME>
static int run(const rd::HostMesh& h, const std::vector<double>& Wn, const std::vector<double>& Ws, double gamma,
               double eps, double dt, std::vector<double>& s1, std::vector<double>& s2) {
  const int nt = h.nt, nv = h.nv;
  const rd::Gas<double> gas = rd::Gas<double>::of(gamma);
  for (int t = 0; t < nt; ++t) {
    double Zn[3][4], Zs[3][4], wn[3][4], ws[3][4], nx[3], ny[3], hl[3];
    for (int c = 0; c < 3; ++c) {
      const int vi = h.tri[(size_t)c * nt + t], vc = h.vperm[vi];
      for (int k = 0; k < 4; ++k) {
        wn[c][k] = Wn[(size_t)k * nv + vc];
        ws[c][k] = Ws[(size_t)k * nv + vc];
      }
      double sp;
      if (!rd::vertex_Z(wn[c], gamma, Zn[c], sp) || !rd::vertex_Z(ws[c], gamma, Zs[c], sp)) return 2;
      nx[c] = h.nx[(size_t)c * nt + t];
      ny[c] = h.ny[(size_t)c * nt + t];
      hl[c] = h.hl[(size_t)c * nt + t];
    }
    double out[3][4], rec[16];
    if (rd::stage1_body<double, SCHEME>(Zn, nx, ny, hl, gas, eps, out, rec)) return 3;
    const size_t tc = (size_t)h.tperm[t];
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) s1[12 * tc + 4 * c + k] = out[c][k];
    if (SCHEME == RD_N1) continue;
    if (rd::stage2_body<double, SCHEME>(Zs, wn, ws, rec, nx, ny, hl, h.area[t], dt, gas, eps, out)) return 4;
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 4; ++k) s2[12 * tc + 4 * c + k] = out[c][k];
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t nv = 0, nt = 0, has_shift = 0, scheme = 0;
  double Lx = 0, Ly = 0, gamma = 0, eps = 0, dt = 0;
  bool ok = std::fread(&nv, 4, 1, f) == 1 && std::fread(&nt, 4, 1, f) == 1 && std::fread(&Lx, 8, 1, f) == 1 &&
            std::fread(&Ly, 8, 1, f) == 1 && std::fread(&has_shift, 4, 1, f) == 1;
  std::vector<double> xy(2 * (size_t)nv), Wn(4 * (size_t)nv), Ws(4 * (size_t)nv);
  std::vector<int32_t> tri(3 * (size_t)nt);
  std::vector<int8_t> sh(6 * (size_t)nt);
  ok = ok && std::fread(xy.data(), 8, xy.size(), f) == xy.size() &&
       std::fread(tri.data(), 4, tri.size(), f) == tri.size();
  if (ok && has_shift) ok = std::fread(sh.data(), 1, sh.size(), f) == sh.size();
  ok = ok && std::fread(&gamma, 8, 1, f) == 1 && std::fread(&eps, 8, 1, f) == 1 && std::fread(&dt, 8, 1, f) == 1 &&
       std::fread(&scheme, 4, 1, f) == 1 && std::fread(Wn.data(), 8, Wn.size(), f) == Wn.size() &&
       std::fread(Ws.data(), 8, Ws.size(), f) == Ws.size();
  std::fclose(f);
  if (!ok) return 2;
  rd::HostMesh h;
  if (rd::build_host_mesh(nv, xy.data(), nt, tri.data(), has_shift ? sh.data() : nullptr, Lx, Ly, RD_ORDER_MORTON, h))
    return 1;
  std::vector<double> s1(12 * (size_t)nt, 0.0), s2(12 * (size_t)nt, 0.0);
  const bool df = (scheme & 16) != 0;
  scheme &= 15;
  int rc;
  if (df)
    rc = scheme == 0 ? run_df<RD_N1>(h, Wn, Ws, gamma, eps, dt, s1, s2)
         : scheme == 1 ? run_df<RD_B2>(h, Wn, Ws, gamma, eps, dt, s1, s2)
                       : run_df<RD_LDA2>(h, Wn, Ws, gamma, eps, dt, s1, s2);
  else
    rc = scheme == 0 ? run<RD_N1>(h, Wn, Ws, gamma, eps, dt, s1, s2)
         : scheme == 1 ? run<RD_B2>(h, Wn, Ws, gamma, eps, dt, s1, s2)
                       : run<RD_LDA2>(h, Wn, Ws, gamma, eps, dt, s1, s2);
  if (rc) return rc;
  FILE* o = std::fopen(argv[2], "wb");
  if (!o) return 2;
  std::fwrite(s1.data(), 8, s1.size(), o);
  if (scheme != 0) std::fwrite(s2.data(), 8, s2.size(), o);
  std::fclose(o);
  return 0;
}
