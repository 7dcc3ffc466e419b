"""The FP64 triangle kernels divide with their own reciprocal (the hardware's
approximate reciprocal refined by two Newton-Raphson steps, Newton's method for
1/x: r <- r + r (1 - x r)); it is held here against CUDA's IEEE division 1.0/x
on the same device, on random doubles over the whole range where the fast path
is taken, and on the edges that take the IEEE path."""
import numpy as np
import pytest

from tests._gpu import require_gpu

pytestmark = pytest.mark.gpu


def _bits_to_double(b):
    return np.asarray(b, dtype=np.uint64).view(np.float64)


def _ulp_distance(a, b):
    """|a - b| in units in the last place for finite doubles of the same sign."""
    ia = a.view(np.int64).astype(np.int64)
    ib = b.view(np.int64).astype(np.int64)
    return np.abs(ia - ib)


def test_rcp_against_ieee_division_on_random_doubles():
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    rng = np.random.default_rng(11)
    n = 1 << 21
    exp = rng.integers(24, 2023, size=n, dtype=np.uint64)          # biased exponents of the fast path
    man = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    sign = rng.integers(0, 2, size=n, dtype=np.uint64)
    x = _bits_to_double((sign << np.uint64(63)) | (exp << np.uint64(52)) | man)
    # exact powers of two and mantissas next to them
    x[:4096] = _bits_to_double((rng.integers(24, 2023, 4096, dtype=np.uint64) << np.uint64(52)))
    x[4096:8192] = _bits_to_double((rng.integers(24, 2023, 4096, dtype=np.uint64) << np.uint64(52)) |
                                   np.uint64((1 << 52) - 1))
    xd = torch.tensor(x, device="cuda")
    got = binding.math_eval("rcp", xd).cpu().numpy()
    ieee = (1.0 / xd).cpu().numpy()
    ulp = _ulp_distance(got, ieee)
    mism_rand = int((ulp[8192:] != 0).sum())
    mism_pow2 = int((ulp[:4096] != 0).sum())
    mism_ones = int((ulp[4096:8192] != 0).sum())
    print(f"rcp vs IEEE 1/x: random mantissas {mism_rand} of {n - 8192} differ, powers of two {mism_pow2} of 4096, "
          f"all-ones mantissas {mism_ones} of 4096; max {int(ulp.max())} ulp")
    # two Newton steps from the hardware approximation leave the result within one ulp
    # of the correctly rounded 1/x (measured: bitwise equal on random mantissas and on
    # powers of two; one ulp on mantissas of all ones, just below a power of two)
    assert int(ulp.max()) <= 1
    assert mism_rand <= (n - 8192) // 10000
    assert mism_pow2 == 0


def test_rcp_edges_take_the_ieee_division():
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    vals = [0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, 2.2250738585072014e-308,
            1.7976931348623157e308, -1.7976931348623157e308]
    for e in (1, 23, 24, 2022, 2023, 2046):                      # biased exponents around the fast range
        for m in (0, 1, (1 << 52) - 1):
            for s in (0, 1):
                vals.append(float(_bits_to_double([(s << 63) | (e << 52) | m])[0]))
    x = np.array(vals)
    xd = torch.tensor(x, device="cuda")
    got = binding.math_eval("rcp", xd).cpu().numpy()
    ieee = (1.0 / xd).cpu().numpy()
    for xi, g, r in zip(x, got, ieee):
        if np.isnan(r):
            assert np.isnan(g), xi
        else:
            assert g.view(np.uint64) == r.view(np.uint64) or abs(int(g.view(np.int64)) - int(r.view(np.int64))) <= 1, xi
    # outside the fast range the IEEE path is taken: bitwise equal there
    e = (x.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF)
    slow = (e < 24) | (e > 2022)
    fin = slow & ~np.isnan(ieee)
    assert np.array_equal(got[fin].view(np.uint64), ieee[fin].view(np.uint64))
