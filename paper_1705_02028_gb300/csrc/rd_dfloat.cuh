// rd_dfloat.cuh -- double-float ("double-word") arithmetic: a value is the
// unevaluated sum hi + lo of two IEEE single-precision numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits.
//
// GB300 executes FP32 at 64 times its FP64 rate, so the triangle kernels can
// run their per-triangle algebra in this type on the FP32 pipe.  The building
// blocks are the classical error-free transformations:
//   * two_sum (Knuth, TAOCP vol. 2, Sec. 4.2.2): s + e = a + b exactly;
//   * fast_two_sum (Dekker 1971), valid when |a| >= |b| or a = 0;
//   * two_prod with a fused multiply-add: p + e = a * b exactly;
// and the double-word sum and product whose error bounds are proved by
// Joldes, Muller and Popescu (ACM TOMS 44, 2017): the "accurate" sum
// (relative error <= 3 u^2) and the product using FMAs (<= 5 u^2), u = 2^-24.
// The reciprocal and square root are one Newton step in double-word arithmetic
// from the single-precision hardware results (Newton's iteration for 1/x and
// for sqrt(x)); a / b is a * (1 / b).
//
// Every single-precision operation is written with an explicit rounding
// intrinsic on the device (__fadd_rn, __fmul_rn, __fmaf_rn), which the
// compiler may neither contract into an FMA nor reorder: the transformations
// rely on each operation being rounded separately.  On the host (the CPU
// build of the kernels' per-triangle code) the same sequence of IEEE single
// operations gives bitwise the same results when compiled without contraction
// (-ffp-contract=off), with std::fma for the fused operations.
#pragma once

#include <cmath>
#include <cstdint>

#ifndef RD_HD
#define RD_HD __host__ __device__ __forceinline__
#endif

namespace rd {
// The type and its functions live in a nested namespace: argument-dependent
// lookup finds them for double-float arguments, while unqualified calls of
// sqrt / fabs on float and double arguments inside namespace rd still see the
// standard overloads.
namespace dw {

namespace dfo {
RD_HD float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
RD_HD float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
RD_HD float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
RD_HD float fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
// single-precision reciprocal and square root, correctly rounded
RD_HD float rcp(float a) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(a);
#else
  return 1.0f / a;
#endif
}
RD_HD float sqrt(float a) {
#ifdef __CUDA_ARCH__
  return __fsqrt_rn(a);
#else
  return std::sqrt(a);
#endif
}
}  // namespace dfo

struct dfloat {
  float hi, lo;
  dfloat() = default;
  RD_HD constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // from double: hi = double rounded to single, lo = the rest rounded to single
  RD_HD dfloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  RD_HD dfloat(int x) : dfloat((double)x) {}
  RD_HD explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth)
RD_HD dfloat two_sum(float a, float b) {
  const float s = dfo::add(a, b);
  const float bb = dfo::sub(s, a);
  const float e = dfo::add(dfo::sub(a, dfo::sub(s, bb)), dfo::sub(b, bb));
  return dfloat(s, e);
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
RD_HD dfloat fast_two_sum(float a, float b) {
  const float s = dfo::add(a, b);
  const float e = dfo::sub(b, dfo::sub(s, a));
  return dfloat(s, e);
}
// p + e = a * b exactly (FMA)
RD_HD dfloat two_prod(float a, float b) {
  const float p = dfo::mul(a, b);
  return dfloat(p, dfo::fma(a, b, -p));
}

RD_HD dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }

#ifndef RD_DF_ACCURATE_ADD
#define RD_DF_ACCURATE_ADD 0
#endif
#if RD_DF_ACCURATE_ADD
// accurate double-word sum
RD_HD dfloat operator+(dfloat x, dfloat y) {
  const dfloat s = two_sum(x.hi, y.hi);
  const dfloat t = two_sum(x.lo, y.lo);
  const float c = dfo::add(s.lo, t.hi);
  const dfloat v = fast_two_sum(s.hi, c);
  const float w = dfo::add(t.lo, v.lo);
  return fast_two_sum(v.hi, w);
}
#else
// double-word sum with one error-free transformation (Dekker's add2): the error
// is below about 2 u^2 (|x| + |y|), i.e. of the order of the operands' own
// representation error, which is what every later operation of the triangle
// algebra sees anyway; half the operations of the accurate sum.
RD_HD dfloat operator+(dfloat x, dfloat y) {
  const dfloat s = two_sum(x.hi, y.hi);
  const float e = dfo::add(s.lo, dfo::add(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}
#endif
RD_HD dfloat operator-(dfloat x, dfloat y) { return x + (-y); }

// double-word product with FMAs
RD_HD dfloat operator*(dfloat x, dfloat y) {
  const dfloat c = two_prod(x.hi, y.hi);
  const float tl0 = dfo::mul(x.lo, y.lo);
  const float tl1 = dfo::fma(x.hi, y.lo, tl0);
  const float cl2 = dfo::fma(x.lo, y.hi, tl1);
  const float cl3 = dfo::add(c.lo, cl2);
  return fast_two_sum(c.hi, cl3);
}

// 1 / y: r0 = 1 / hi in single precision, then r = r0 + r0 e with the residual
// e = 1 - y r0 formed exactly in its leading part (fma) and corrected by lo.
RD_HD dfloat rcp(dfloat y) {
  const float r0 = dfo::rcp(y.hi);
  float e = dfo::fma(-y.hi, r0, 1.0f);
  e = dfo::fma(-y.lo, r0, e);
  return fast_two_sum(r0, dfo::mul(r0, e));
}
RD_HD dfloat operator/(dfloat x, dfloat y) { return x * rcp(y); }

// sqrt(x): s0 = sqrt(hi) in single precision, then s = s0 + (x - s0^2) / (2 s0)
// with x - s0^2 formed from the exact square.
RD_HD dfloat sqrt(dfloat x) {
  if (!(x.hi > 0.0f)) return dfloat(dfo::sqrt(x.hi), 0.0f);
  const float s0 = dfo::sqrt(x.hi);
  const dfloat p = two_prod(s0, s0);
  const float d = dfo::add(dfo::sub(dfo::sub(x.hi, p.hi), p.lo), x.lo);
  return fast_two_sum(s0, dfo::mul(d, dfo::mul(0.5f, dfo::rcp(s0))));
}

RD_HD dfloat fabs(dfloat a) { return a.hi < 0.0f ? -a : a; }

RD_HD dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
RD_HD dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
RD_HD dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

// Order of normalised double-words: by hi, then by lo.
RD_HD bool operator<(dfloat a, dfloat b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
RD_HD bool operator>(dfloat a, dfloat b) { return b < a; }
RD_HD bool operator<=(dfloat a, dfloat b) { return !(b < a); }
RD_HD bool operator>=(dfloat a, dfloat b) { return !(a < b); }

#if defined(__CUDACC__)
// double -> double-float (hi = x rounded to single, lo = the rest rounded to
// single) and back, with the double operations written as non-contractible
// intrinsics so that every kernel forms the same bits.
__device__ __forceinline__ dfloat to_df(double x) {
  const float h = __double2float_rn(x);
  return dfloat(h, __double2float_rn(__dsub_rn(x, (double)h)));
}
__device__ __forceinline__ double from_df(dfloat a) { return __dadd_rn((double)a.hi, (double)a.lo); }
#endif

}  // namespace dw
using dw::dfloat;

}  // namespace rd
