// rd_probe.cu -- measurement helpers: an FMA-throughput probe (the ALU peak the
// triangle kernels are held against) and an exact count of the floating-point
// operations of the per-triangle bodies (the same source as the kernels,
// instantiated on a counting scalar type).
#include <cuda_runtime.h>

#include <cmath>

#include "rd_internal.h"
#include "rd_kernels.cuh"

namespace {

// ---------------------------------------------------------------------------
// counting scalar
// ---------------------------------------------------------------------------
struct Counts {
  long long add = 0, mul = 0, div = 0, sqrt = 0;
};
Counts g_cnt;

struct Flop {
  double v;
  Flop() : v(0) {}
  Flop(double x) : v(x) {}
};
inline Flop operator+(Flop a, Flop b) { ++g_cnt.add; return Flop(a.v + b.v); }
inline Flop operator-(Flop a, Flop b) { ++g_cnt.add; return Flop(a.v - b.v); }
inline Flop operator-(Flop a) { return Flop(-a.v); }
inline Flop operator*(Flop a, Flop b) { ++g_cnt.mul; return Flop(a.v * b.v); }
inline Flop operator/(Flop a, Flop b) { ++g_cnt.div; return Flop(a.v / b.v); }
inline Flop& operator+=(Flop& a, Flop b) { a = a + b; return a; }
inline Flop& operator-=(Flop& a, Flop b) { a = a - b; return a; }
inline Flop& operator*=(Flop& a, Flop b) { a = a * b; return a; }
inline bool operator<(Flop a, Flop b) { return a.v < b.v; }
inline bool operator>(Flop a, Flop b) { return a.v > b.v; }
inline bool operator<=(Flop a, Flop b) { return a.v <= b.v; }
inline bool operator>=(Flop a, Flop b) { return a.v >= b.v; }
inline Flop fabs(Flop a) { return Flop(std::fabs(a.v)); }
inline Flop sqrt(Flop a) { ++g_cnt.sqrt; return Flop(std::sqrt(a.v)); }

// a representative interior triangle of a 64^2 regular mesh with a smooth,
// moving state (no entropy-fix branch taken)
void sample(Flop Z[3][4], Flop Zs[3][4], Flop Wn[3][4], Flop Ws[3][4], Flop nx[3], Flop ny[3], Flop hl[3],
            Flop& area) {
  const double gamma = 1.4, h = 1.0 / 64;
  const double rho[3] = {1.9, 2.0, 1.95}, u[3] = {0.45, 0.5, 0.48}, v[3] = {0.01, -0.004, 0.007},
               p[3] = {2.5, 2.49, 2.51};
  for (int i = 0; i < 3; ++i) {
    for (int s = 0; s < 2; ++s) {
      double r = rho[i] * (1 + 0.001 * s), e = 0.5 * r * (u[i] * u[i] + v[i] * v[i]) + p[i] / (gamma - 1);
      double W[4] = {r, r * u[i], r * v[i], e};
      double hh = (e + p[i]) / r, sr = std::sqrt(r);
      Flop* Zd = s ? Zs[i] : Z[i];
      Flop* Wd = s ? Ws[i] : Wn[i];
      Zd[0] = sr; Zd[1] = sr * u[i]; Zd[2] = sr * v[i]; Zd[3] = sr * hh;
      for (int k = 0; k < 4; ++k) Wd[k] = W[k];
    }
  }
  // triangle (0,0), (h,0), (h,h): inward unit normals and half edge lengths
  const double n[3][2] = {{-h, 0.0}, {h, -h}, {0.0, h}};
  for (int c = 0; c < 3; ++c) {
    double len = std::sqrt(n[c][0] * n[c][0] + n[c][1] * n[c][1]);
    nx[c] = n[c][0] / len;
    ny[c] = n[c][1] / len;
    hl[c] = len / 2;
  }
  area = 0.5 * h * h;
}

template <int SCHEME>
void count(int stage, Counts& out) {
  Flop Z[3][4], Zs[3][4], Wn[3][4], Ws[3][4], nx[3], ny[3], hl[3], area, o[3][4], rec[16];
  sample(Z, Zs, Wn, Ws, nx, ny, hl, area);
  const rd::Gas<Flop> gas = rd::Gas<Flop>::of(Flop(1.4));  // formed on the host, once per launch
  g_cnt = Counts();
  rd::stage1_body<Flop, SCHEME>(Z, nx, ny, hl, gas, Flop(1e-6), o, rec);
  if (stage == 2) {
    g_cnt = Counts();
    rd::stage2_body<Flop, SCHEME>(Zs, Wn, Ws, rec, nx, ny, hl, area, Flop(1e-3), gas, Flop(1e-6), o);
  }
  out = g_cnt;
}

// ---------------------------------------------------------------------------
// FMA throughput probe: 8 independent FMA chains per thread.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T seed, T* out) {
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed + T(threadIdx.x + j) * T(1e-7);
  const T m = T(0.9999999), c = T(1e-7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int probe(int iters, double* flops_per_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RD_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RD_ECUDA;
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) {
    cudaGetLastError();
    return RD_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_probe<T><<<blocks, threads>>>(iters / 4, T(1), out);  // warm-up
  cudaEventRecord(e0);
  k_fma_probe<T><<<blocks, threads>>>(iters, T(1), out);
  cudaEventRecord(e1);
  int rc = RD_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = RD_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  cudaGetLastError();
  if (rc == RD_OK) *flops_per_s = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
  return rc;
}

}  // namespace

extern "C" int rd_count_flops(int32_t scheme, int32_t stage, double out[4]) {
  if (!out || (stage != 1 && stage != 2)) return RD_EINVAL;
  if (stage == 2 && scheme == RD_N1) return RD_EINVAL;
  Counts c;
  switch (scheme) {
    case RD_N1: count<RD_N1>(stage, c); break;
    case RD_B2: count<RD_B2>(stage, c); break;
    case RD_LDA2: count<RD_LDA2>(stage, c); break;
    default: return RD_EINVAL;
  }
  out[0] = (double)c.add;
  out[1] = (double)c.mul;
  out[2] = (double)c.div;
  out[3] = (double)c.sqrt;
  return RD_OK;
}

extern "C" int rd_probe_fma_peak(int32_t precision, double* flops_per_s) {
  if (!flops_per_s) return RD_EINVAL;
  if (precision == RD_FP64) return probe<double>(20000, flops_per_s);
  if (precision == RD_FP32) return probe<float>(400000, flops_per_s);
  return RD_EINVAL;
}

namespace {
// Element-wise evaluation of the triangle kernels' own device arithmetic
// helpers, so that tests can hold them against CUDA's IEEE operations.
__global__ void k_math_eval(int fn, long long n, const double* __restrict__ x, double* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = x[i];
  double r = 0.0;
  switch (fn) {
    case RD_MATH_RCP: r = rd::rcp(a); break;
    default: break;
  }
  out[i] = r;
}
}  // namespace

extern "C" int rd_math_eval(int32_t fn, int64_t n, const double* x, double* out, void* cuda_stream) {
  if (fn != RD_MATH_RCP || n < 0 || (n > 0 && (!x || !out))) return RD_EINVAL;
  if (n == 0) return RD_OK;
  const int threads = 256;
  const long long blocks = (n + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return RD_EINVAL;
  k_math_eval<<<(unsigned)blocks, threads, 0, (cudaStream_t)cuda_stream>>>(fn, n, x, out);
  if (cudaGetLastError() != cudaSuccess) return RD_ECUDA;
  if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) {
    cudaGetLastError();
    return RD_ECUDA;
  }
  return RD_OK;
}
