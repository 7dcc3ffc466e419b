// Host build of the double-float operations the RD_DF64 triangle kernels use
// (rd_dfloat.cuh), for the CPU test that holds them to their error bounds.
// Input (binary): n (int32), then n pairs (a, b) of doubles.  Each is split
// into a double-float (hi = a rounded to single, lo = the rest rounded to
// single).  Output (binary): for each pair the values of a + b, a - b, a * b,
// a / b, sqrt(|a|) as (hi, lo) float pairs, then the exact-transformation
// residual checks two_sum and two_prod of the two his as (s, e) float pairs.
#include <cmath>
#include <cstdio>
#include <vector>

#include "rd_dfloat.cuh"

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int n = 0;
  if (std::fread(&n, 4, 1, f) != 1 || n < 0) return 2;
  std::vector<double> ab(2 * (size_t)n);
  if (std::fread(ab.data(), 8, ab.size(), f) != ab.size()) return 2;
  std::fclose(f);
  std::vector<float> out(14 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const rd::dfloat a(ab[2 * i]), b(ab[2 * i + 1]);
    const rd::dfloat r[5] = {a + b, a - b, a * b, a / b, sqrt(fabs(a))};
    for (int k = 0; k < 5; ++k) {
      out[14 * (size_t)i + 2 * k] = r[k].hi;
      out[14 * (size_t)i + 2 * k + 1] = r[k].lo;
    }
    const rd::dfloat s = rd::dw::two_sum(a.hi, b.hi), p = rd::dw::two_prod(a.hi, b.hi);
    out[14 * (size_t)i + 10] = s.hi;
    out[14 * (size_t)i + 11] = s.lo;
    out[14 * (size_t)i + 12] = p.hi;
    out[14 * (size_t)i + 13] = p.lo;
  }
  FILE* o = std::fopen(argv[2], "wb");
  if (!o) return 2;
  std::fwrite(out.data(), 4, out.size(), o);
  std::fclose(o);
  return 0;
}
