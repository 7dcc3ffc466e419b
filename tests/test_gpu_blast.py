"""GPU parity on the strong-shock tests of Secs. 5.1.3, 5.2.3 and 5.2.4 (the
oracle is pinned on them in tests/test_oracle_blast.py): planar and
cylindrical blast waves (gamma = 5/3, near-vacuum pre-shock gas) and the
two-dimensional Riemann problem on a box with ghost boundaries, each run to
its final time with the last step clipped (rd_run's t_end), against the
long-double oracle.  Bar: 1e-12, or, where the oracle's own double run
departs from its long-double run by more (round-off amplified by strong
shocks and the Bmax blend), at least as close as the oracle's double run."""
import os

import numpy as np
import pytest

import oracle
from tests._gpu import rel_max_err, require_gpu
from tests.test_oracle_blast import G53, cylindrical_blast, mirror, planar_blast, riemann2d, run_to_time

pytestmark = pytest.mark.gpu
NTH = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def rd():
    require_gpu()
    from paper_1705_02028_gb300 import binding
    return binding


CASES = {
    "planar_N1": (lambda: planar_blast(200), "N1", 10.0, G53),
    "cylindrical_N1": (lambda: cylindrical_blast(64), "N1", 0.4, G53),
    "riemann2d_N1": (lambda: riemann2d(48), "N1", 0.8, 1.4),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_strong_shock_problems_match_the_oracle(rd, case, precision):
    make, scheme, T, gamma = CASES[case]
    mesh, W0 = make()
    m = rd.Mesh(mesh, reorder="morton")
    s = rd.State(m, W0, scheme=scheme, precision=precision, gamma=gamma)
    done = s.run(1_000_000, t_end=T)
    t, n = s.time()
    assert t == pytest.approx(T, rel=1e-14)
    Wg = s.get()
    Wld, nld = run_to_time(mesh, W0, scheme, T, gamma, nthreads=NTH, long_double=True)
    Wd, _ = run_to_time(mesh, W0, scheme, T, gamma, nthreads=NTH)
    err, floor = rel_max_err(Wg, Wld), rel_max_err(Wd, Wld)
    print(f"{case} {precision}: {done} steps (oracle {nld}), vs oracle(ld) {err:.2e}, "
          f"oracle(double) vs oracle(ld) {floor:.2e}")
    assert done == nld
    assert err < max(1e-12, floor)
    if case.startswith("riemann2d"):
        assert np.abs(Wg - mirror(mesh, Wg)).max() < 1e-13 * np.abs(Wg).max()


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_riemann2d_bmax_first_steps(rd, precision):
    """The Bmax blend on the two-dimensional Riemann problem over its first 60 steps
    (later, the blend's round-off amplification -- it breaks the x <-> y symmetry
    at 4e-3 by t = 0.8 even in the oracle -- changes the dt sequence itself)."""
    mesh, W0 = riemann2d(48)
    m = rd.Mesh(mesh, reorder="morton")
    s = rd.State(m, W0, scheme="BMAX2", precision=precision)
    assert s.run(60) == 60
    Wld, _ = oracle.run(mesh, W0, "BMAX2", nsteps=60, nthreads=NTH, long_double=True)
    Wd, _ = oracle.run(mesh, W0, "BMAX2", nsteps=60, nthreads=NTH)
    err, floor = rel_max_err(s.get(), Wld), rel_max_err(Wd, Wld)
    print(f"riemann2d BMAX2 {precision}, 60 steps: vs oracle(ld) {err:.2e}, oracle(double) vs oracle(ld) {floor:.2e}")
    assert err < max(1e-12, floor)
