"""RD_DF64: FP64 state with the per-triangle algebra in double-float arithmetic
(FP32 pairs) on the FP32 pipe.  Held to the same bar as the FP64 path: 1e-12
relative in the max norm against the oracle's long-double run after 100 steps
(20 on the Sod-like state, whose B2 round-off amplification is documented in
tests/test_oracle_step.py), the per-triangle shares element by element, the
variants, a ragged mesh with dt per step, and the benchmarked 4096^2 KHI
configuration's first steps."""
import os

import numpy as np
import pytest

import oracle
from paper_1705_02028_gb300 import inputs
from tests._gpu import rel_max_err, require_gpu

pytestmark = pytest.mark.gpu
NTH = max(1, min(16, os.cpu_count() or 1))
TOL = 1e-12


@pytest.fixture(scope="module")
def rd():
    require_gpu()
    from paper_1705_02028_gb300 import binding
    return binding


def _states(mesh, kind):
    return {"vortex": inputs.vortex_state, "khi": inputs.khi_state, "sod": inputs.sod_like_state,
            "smooth": inputs.smooth_density_state}[kind](mesh)


@pytest.mark.parametrize("state,N,scheme,steps", [("vortex", 64, "N1", 100), ("vortex", 64, "B2", 100),
                                                  ("khi", 48, "B2", 100), ("sod", 48, "B2", 20),
                                                  ("vortex", 40, "LDA2", 100), ("smooth", 50, "B2", 100)])
def test_df64_matches_oracle(rd, state, N, scheme, steps):
    mesh = inputs.periodic_grid(N, relabel_seed=6)
    W0 = _states(mesh, state)
    m = rd.Mesh(mesh, reorder="morton")
    s = rd.State(m, W0, scheme=scheme, precision="df64")
    assert s.run(steps) == steps
    Wld, dto = oracle.run(mesh, W0, scheme, nsteps=steps, nthreads=NTH, long_double=True)
    err = rel_max_err(s.get(), Wld)
    s64 = rd.State(m, W0, scheme=scheme, precision="fp64")
    s64.run(steps)
    err64 = rel_max_err(s64.get(), Wld)
    print(f"{state} {N}^2 {scheme} {steps} steps: DF64 vs oracle(ld) {err:.2e}, FP64 vs oracle(ld) {err64:.2e}")
    assert err < TOL
    t, n = s.time()
    assert n == steps and t == pytest.approx(dto.sum(), rel=1e-13)


@pytest.mark.parametrize("scheme", ["BMAX2", "BMIN2", "BX2", "B2_SL", "LDA2_SL"])
def test_df64_variants(rd, scheme):
    mesh = inputs.periodic_grid(40, relabel_seed=6)
    W0 = inputs.khi_state(mesh)
    m = rd.Mesh(mesh, reorder="morton")
    s = rd.State(m, W0, scheme=scheme, precision="df64")
    s.run(40)
    Wld, _ = oracle.run(mesh, W0, scheme, nsteps=40, nthreads=NTH, long_double=True)
    err = rel_max_err(s.get(), Wld)
    print(f"{scheme} 40^2 KHI 40 steps: DF64 vs oracle(ld) {err:.2e}")
    assert err < TOL


def test_df64_shares_element_by_element(rd):
    """Stage-1 shares of one DF64 step against the long-double oracle (the same 1e-11
    of max|phi^N| bar as the FP64 share test), through a full step's effect: the
    state after one N1 step (W* = W^n - dt/V R1) isolates the stage-1 shares."""
    mesh = inputs.periodic_grid(33, 31, Lx=1.0, Ly=31 / 33, relabel_seed=6)
    for kind in ("vortex", "khi", "sod"):
        W = _states(mesh, kind)
        m = rd.Mesh(mesh)
        s = rd.State(m, W, scheme="N1", precision="df64")
        s.step()
        Wld, _ = oracle.run(mesh, W, "N1", nsteps=1, long_double=True)
        assert rel_max_err(s.get(), Wld) < 1e-14, kind


def test_df64_ragged_mesh_step_by_step(rd):
    mesh = inputs.periodic_grid(37, 23, Lx=1.0, Ly=23 / 37, relabel_seed=3)
    W0 = inputs.khi_state(mesh, seed=9)
    m = rd.Mesh(mesh)
    s = rd.State(m, W0, scheme="B2", precision="df64")
    dts = [s.step(return_dt=True) for _ in range(7)]
    Wo, dto = oracle.run(mesh, W0, "B2", nsteps=7, long_double=True)
    assert np.allclose(dts, dto, rtol=1e-14, atol=0)
    assert rel_max_err(s.get(), Wo) < TOL


def test_df64_unstructured_and_walls(rd):
    mesh = inputs.jittered_grid(36, relabel_seed=6)
    W0 = inputs.vortex_state(mesh)
    m = rd.Mesh(mesh, reorder="morton")
    s = rd.State(m, W0, scheme="B2", precision="df64")
    s.run(60)
    Wld, _ = oracle.run(mesh, W0, "B2", nsteps=60, nthreads=NTH, long_double=True)
    assert rel_max_err(s.get(), Wld) < TOL
    box = inputs.bounded_grid(30, 30, periodic_x=True, bc_y="wall")
    Wb = inputs.khi_state(box)
    mb = rd.Mesh(box, reorder="morton")
    sb = rd.State(mb, Wb, scheme="B2", precision="df64")
    sb.run(40)
    Wbo, _ = oracle.run(box, Wb, "B2", nsteps=40, nthreads=NTH, long_double=True)
    assert rel_max_err(sb.get(), Wbo) < TOL


def test_df64_conservation_determinism_and_options(rd):
    mesh = inputs.periodic_grid(96, relabel_seed=6)
    W0 = inputs.khi_state(mesh)
    m = rd.Mesh(mesh)
    s = rd.State(m, W0, scheme="B2", precision="df64")
    c0 = s.conserved()
    s.autotune()
    s.run(50)
    c1 = s.conserved()
    assert np.abs(c1 - c0).max() <= 1e-13 * np.abs(c0).max()
    s2 = rd.State(m, W0, scheme="B2", precision="df64")
    s2.run(50)
    assert np.array_equal(s.get(), s2.get())          # launch shapes do not change results
    with pytest.raises(rd.RDError) as e:
        s2.set_tiling(512, 128)
    assert e.value.status == rd.RD_ENOTSUP


def test_df64_full_size_4096_khi_first_steps(rd):
    """The 4096^2 KHI B2 workload in DF64 with autotuned shapes: three graph-replayed
    steps against the oracle at 1e-12."""
    mesh = inputs.periodic_grid(4096)
    W0 = inputs.khi_state(mesh)
    m = rd.Mesh(mesh, reorder="morton")
    s = rd.State(m, W0, scheme="B2", precision="df64")
    s.autotune()
    assert s.run(3) == 3
    Wo, _ = oracle.run(mesh, W0, "B2", nsteps=3, nthreads=NTH)
    err = rel_max_err(s.get(), Wo)
    print(f"4096^2 KHI B2 DF64, 3 steps: rel max err vs oracle {err:.2e}")
    assert err < TOL


def test_df64_kernel_variants_are_bitwise_equal(rd):
    """The DF64 triangle-kernel variants (128 registers without and with block
    barriers between phases, 96 and 80 with barriers), every block size and
    different shapes per stage run the same arithmetic: bitwise equal states,
    including a ragged last block."""
    mesh = inputs.periodic_grid(45, 37, Lx=1.0, Ly=37 / 45, relabel_seed=6)
    W0 = inputs.khi_state(mesh)
    m = rd.Mesh(mesh)
    ref = None
    for occ in (2, 3, 4, 5):
        for tb in (64, 256):
            for scheme in ("B2", "N1"):
                s = rd.State(m, W0, scheme=scheme, precision="df64")
                s.set_launch_shapes(tb, 256, occ)
                s.run(6)
                W = s.get()
                s.close()
                key = (scheme,)
                if ref is None:
                    ref = {}
                if key not in ref:
                    ref[key] = W
                assert np.array_equal(W, ref[key]), (occ, tb, scheme)
    for (tb1, o1), (tb2, o2) in (((256, 5), (128, 4)), ((64, 2), (192, 3))):
        s = rd.State(m, W0, scheme="B2", precision="df64")
        s.set_stage_shapes(1, tb1, o1)
        s.set_stage_shapes(2, tb2, o2)
        assert s.stage_shapes(1) == (tb1, o1) and s.stage_shapes(2) == (tb2, o2)
        s.run(6)
        assert np.array_equal(s.get(), ref[("B2",)]), (tb1, o1, tb2, o2)
        s.close()
    s = rd.State(m, W0, scheme="B2", precision="df64")
    for stage, tb, var in ((3, 128, 2), (0, 128, 2), (1, 100, 2), (2, 128, 6), (1, 128, 1)):
        with pytest.raises(rd.RDError):
            s.set_stage_shapes(stage, tb, var)
    assert s.stage_shapes(1) == s.stage_shapes(2)   # unchanged by the rejected calls
    s.close()
