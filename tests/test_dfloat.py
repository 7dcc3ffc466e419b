"""Double-float arithmetic of the RD_DF64 triangle kernels (rd_dfloat.cuh, host
build of the same source): the error-free transformations are exact; the sum
(one error-free transformation, Dekker's add2) errs by at most 3 u^2 (|a| +
|b|), the order of its operands' own representation error; the product (with
FMAs), quotient and square root stay within 5, 8 and 8 u^2 relative (the
product's bound is Joldes, Muller & Popescu 2017's), u = 2^-24; all measured
against exact rational arithmetic."""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from paper_1705_02028_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
U2 = Fraction(1, 2 ** 48)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if not nvcc:
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("df") / "dfloat_host_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off", "-I", build.CSRC,
                    os.path.join(HERE, "dfloat_host_check.cu"), "-o", out], check=True)
    return out


def _run(harness, ab, tmp_path):
    src, dst = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(src, "wb") as f:
        f.write(struct.pack("<i", len(ab)))
        f.write(np.ascontiguousarray(ab, dtype=np.float64).tobytes())
    subprocess.run([harness, src, dst], check=True)
    return np.fromfile(dst, dtype=np.float32).reshape(len(ab), 7, 2)


def _split(x):
    hi = np.float32(x)
    lo = np.float32(x - np.float64(hi))
    return Fraction(float(hi)) + Fraction(float(lo))


def test_double_float_operations_within_their_error_bounds(harness, tmp_path):
    rng = np.random.default_rng(5)
    n = 3000
    a = rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))
    b = rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))
    b[:300] = -a[:300] * (1 + rng.uniform(-1e-6, 1e-6, 300))   # near-cancelling sums
    b[300:400] = a[300:400]
    out = _run(harness, np.stack([a, b], axis=1), tmp_path)
    worst = np.zeros(5)
    for i in range(n):
        A, B = _split(a[i]), _split(b[i])
        exact = [A + B, A - B, A * B, A / B]
        for k in range(4):
            got = Fraction(float(out[i, k, 0])) + Fraction(float(out[i, k, 1]))
            # sum and difference: error relative to |a| + |b|; product and quotient: to the result
            ref = abs(A) + abs(B) if k < 2 else abs(exact[k])
            if ref != 0:
                worst[k] = max(worst[k], float(abs(got - exact[k]) / ref / U2))
        # sqrt: compare its square with |A| (relative error of sqrt ~ half that)
        s = Fraction(float(out[i, 4, 0])) + Fraction(float(out[i, 4, 1]))
        worst[4] = max(worst[4], float(abs(s * s - abs(A)) / abs(A) / U2) / 2.0)
        # error-free transformations: exact
        ah, bh = Fraction(float(np.float32(a[i]))), Fraction(float(np.float32(b[i])))
        assert Fraction(float(out[i, 5, 0])) + Fraction(float(out[i, 5, 1])) == ah + bh
        assert Fraction(float(out[i, 6, 0])) + Fraction(float(out[i, 6, 1])) == ah * bh
    print("worst relative error in units of u^2 (add, sub, mul, div, sqrt):", np.round(worst, 3))
    assert worst[0] <= 3 and worst[1] <= 3 and worst[2] <= 5 and worst[3] <= 8 and worst[4] <= 8


def test_normalised_outputs(harness, tmp_path):
    """Every result is normalised: |lo| <= ulp(hi) / 2, so the order by (hi, lo) is numeric."""
    rng = np.random.default_rng(6)
    ab = rng.standard_normal((2000, 2)) * 10.0 ** rng.uniform(-8, 8, (2000, 2))
    out = _run(harness, ab, tmp_path).astype(np.float64)
    hi, lo = out[:, :5, 0], out[:, :5, 1]
    ulp = np.spacing(np.abs(hi).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(lo) <= ulp / 2 + 0.0)
