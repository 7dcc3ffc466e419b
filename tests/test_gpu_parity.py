"""GPU path vs the CPU oracle, element by element, through the C ABI.

Tolerance: the FP64 path must match the oracle to 1e-12 relative in the max
norm (per component, scaled by max(max|W_k|, max|e|)) after 100 steps.  The
reference is the oracle's long-double instantiation (same source): its double
instantiation carries its own round-off of up to ~5e-13 on the B2 vortex after
100 steps, which is printed beside each result.  On the Sod-like state the B2
scheme amplifies round-off (the oracle's own double and long-double runs part
by ~1e-3 within 60 steps, see tests/test_oracle_step.py), so that state is
compared at 1e-12 over its first 20 steps (10 at 1024^2).
The FP32 path reports its L1 density error against the FP64 oracle.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import exact
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


def make_state(rd, mesh, W, scheme, precision="fp64", reorder="morton", eps=1e-6):
    m = rd.Mesh(mesh, reorder=reorder)
    s = rd.State(m, W, scheme=scheme, precision=precision, eps_fix=eps)
    return m, s


@pytest.mark.parametrize("state", ["vortex", "khi", "sod"])
def test_stage1_shares_element_by_element(rd, state):
    mesh = inputs.periodic_grid(33, 31, Lx=1.0, Ly=31 / 33, relabel_seed=6)
    W = {"vortex": inputs.vortex_state, "khi": inputs.khi_state, "sod": inputs.sod_like_state}[state](mesh)
    m, s = make_state(rd, mesh, W, "B2")
    ref = oracle.triangle_terms_ld(mesh, W)
    g = oracle.geometry(mesh)
    rho, u, v, p = inputs.primitives(W)
    spd = np.hypot(u, v) + np.sqrt(1.4 * p / rho)
    cfl_ref = g["lmax"] * spd[mesh.tri].max(axis=1)
    # Per-triangle shares come out of a 4x4 solve whose condition number reaches
    # ~1e3 on these states, so their round-off is ~1e3 eps of the largest
    # intermediate K_i W^_i (10-100x the largest share): the oracle's own double
    # shares differ from its long-double ones by up to 5.4e-13 of max|phi^N| on
    # the KHI state.  Tolerance: 1e-11 of max|phi^N|.
    scale = np.abs(ref["phiN"]).max()
    for which, key in (("N", "phiN"), ("LDA", "phiLDA"), ("B", "phiB")):
        out, cfl = s.triangle_shares(which)
        assert np.abs(out - ref[key]).max() <= 1e-11 * scale, which
    assert np.allclose(cfl, cfl_ref, rtol=1e-14)


@pytest.mark.parametrize("reorder", ["none", "morton", "rcm"])
def test_n1_vortex_64_100_steps(rd, reorder):
    """64x64 periodic vortex, N scheme + forward Euler, CFL 0.8, 100 steps."""
    mesh = inputs.periodic_grid(64, relabel_seed=6)
    W0 = inputs.vortex_state(mesh)
    m, s = make_state(rd, mesh, W0, "N1", reorder=reorder)
    assert s.run(100) == 100
    Wg = s.get()
    Wo, dto = oracle.run(mesh, W0, "N1", nsteps=100, nthreads=NTH, long_double=True)
    assert rel_max_err(Wg, Wo) < TOL
    t, n = s.time()
    assert n == 100 and t == pytest.approx(dto.sum(), rel=1e-13)


@pytest.mark.parametrize("state,N,scheme,steps", [("vortex", 64, "B2", 100), ("khi", 48, "B2", 100),
                                                  ("sod", 48, "B2", 20), ("vortex", 40, "LDA2", 100)])
def test_two_stage(rd, state, N, scheme, steps):
    mesh = inputs.periodic_grid(N, relabel_seed=6)
    W0 = {"vortex": inputs.vortex_state, "khi": inputs.khi_state, "sod": inputs.sod_like_state}[state](mesh)
    m, s = make_state(rd, mesh, W0, scheme)
    assert s.run(steps) == steps
    Wg = s.get()
    Wld, _ = oracle.run(mesh, W0, scheme, nsteps=steps, nthreads=NTH, long_double=True)
    Wd, _ = oracle.run(mesh, W0, scheme, nsteps=steps, nthreads=NTH)
    err, floor = rel_max_err(Wg, Wld), rel_max_err(Wd, Wld)
    print(f"{state} {N}^2 {scheme} {steps} steps: GPU vs oracle(ld) {err:.2e}, oracle(double) vs oracle(ld) {floor:.2e}")
    assert err < TOL


def test_step_by_step_dt_and_ragged_sizes(rd):
    """Non-square ragged mesh (sizes not multiples of the block sizes), dt per step."""
    mesh = inputs.periodic_grid(37, 23, Lx=1.0, Ly=23 / 37, relabel_seed=3)
    W0 = inputs.khi_state(mesh, seed=9)
    m, s = make_state(rd, mesh, W0, "B2")
    dts = [s.step(return_dt=True) for _ in range(7)]
    Wo, dto = oracle.run(mesh, W0, "B2", nsteps=7, long_double=True)
    assert np.allclose(dts, dto, rtol=1e-14, atol=0)
    assert rel_max_err(s.get(), Wo) < TOL


def test_tiny_and_degenerate_meshes(rd):
    """2x2 periodic mesh (every triangle wraps) and a uniform state at rest."""
    mesh = inputs.periodic_grid(2, relabel_seed=1)
    m, s = make_state(rd, mesh, inputs.uniform_state(mesh), "B2")
    s.run(10)
    assert np.abs(s.get() - inputs.uniform_state(mesh)).max() < 1e-14
    mesh3 = inputs.periodic_grid(3, 2, Lx=1.0, Ly=2 / 3)
    W3 = inputs.vortex_state(mesh3)
    m3, s3 = make_state(rd, mesh3, W3, "B2")
    s3.run(20)
    Wo, _ = oracle.run(mesh3, W3, "B2", nsteps=20, long_double=True)
    assert rel_max_err(s3.get(), Wo) < TOL


def test_conservation_and_determinism(rd):
    mesh = inputs.periodic_grid(96, relabel_seed=6)
    W0 = inputs.khi_state(mesh)
    m, s = make_state(rd, mesh, W0, "B2")
    c0 = s.conserved()
    co = oracle.conserved(mesh, W0)
    assert np.allclose(c0, co, rtol=1e-13)
    s.run(50)
    c1 = s.conserved()
    assert np.abs(c1 - c0).max() <= 1e-13 * np.abs(c0).max()
    W1 = s.get()
    m2, s2 = make_state(rd, mesh, W0, "B2")
    s2.run(50)
    assert np.array_equal(W1, s2.get())


def test_checkpoint_resume_is_bitwise(rd):
    mesh = inputs.periodic_grid(40, relabel_seed=2)
    W0 = inputs.vortex_state(mesh)
    m, s = make_state(rd, mesh, W0, "B2")
    s.run(20)
    ref = s.get()
    m2, s2 = make_state(rd, mesh, W0, "B2")
    s2.run(9)
    mid = s2.get()
    m3, s3 = make_state(rd, mesh, mid, "B2")
    s3.run(11)
    assert np.array_equal(s3.get(), ref)


def test_t_end_clips_last_step(rd):
    mesh = inputs.periodic_grid(32)
    W0 = inputs.vortex_state(mesh)
    m, s = make_state(rd, mesh, W0, "B2")
    done = s.run(1000, t_end=0.0123)
    t, n = s.time()
    assert t == pytest.approx(0.0123, rel=1e-15, abs=1e-17)
    assert done == n and n < 1000
    assert s.run(5, t_end=0.0123) == 0


def test_nonphysical_state_is_reported(rd):
    mesh = inputs.periodic_grid(16)
    W0 = inputs.uniform_state(mesh)
    W0[3, 7] = -1.0
    with pytest.raises(rd.RDError) as e:
        make_state(rd, mesh, W0, "B2")
    assert e.value.status == rd.RD_ENONPHYSICAL
    # a CFL far beyond stability drives the state non-physical; the last good state is kept
    mesh = inputs.periodic_grid(24)
    W0 = inputs.sod_like_state(mesh)
    m = rd.Mesh(mesh)
    s = rd.State(m, W0, scheme="N1", cfl=25.0)
    with pytest.raises(rd.RDError) as e:
        s.run(50)
    assert e.value.status == rd.RD_ENONPHYSICAL
    _, n = s.time()
    Wk = s.get()
    rho, u, v, p = inputs.primitives(Wk)
    assert np.all(np.isfinite(Wk)) and rho.min() > 0 and p.min() > 0
    assert n < 50
    # the library stays usable: a new state on the same mesh runs normally
    s2 = rd.State(m, W0, scheme="N1")
    assert s2.run(3) == 3


def test_fp32_l1_density_error(rd):
    mesh = inputs.periodic_grid(64, relabel_seed=6)
    W0 = inputs.vortex_state(mesh)
    m, s = make_state(rd, mesh, W0, "B2", precision="fp32")
    s.run(100)
    W32 = s.get()
    Wo, _ = oracle.run(mesh, W0, "B2", nsteps=100, nthreads=NTH)
    l1 = exact.l1_error(oracle.geometry(mesh)["V"], W32[0], Wo[0])
    print(f"FP32 L1 density error vs FP64 oracle (64^2 vortex, B2, 100 steps): {l1:.3e}")
    assert l1 < 2e-6


def test_full_size_1024_sod_like_b2(rd):
    """1024x1024 (2.1M triangles) Sod-like B2: 10 full steps against the oracle."""
    mesh = inputs.periodic_grid(1024, relabel_seed=6)
    W0 = inputs.sod_like_state(mesh)
    m, s = make_state(rd, mesh, W0, "B2")
    s.run(10)
    Wo, _ = oracle.run(mesh, W0, "B2", nsteps=10, nthreads=NTH, long_double=True)
    assert rel_max_err(s.get(), Wo) < TOL


def test_full_size_4096_khi_b2_first_five_steps(rd):
    """4096x4096 (33.5M triangles) KHI B2: the first five full steps and each step's dt
    against the oracle (about 7 s per oracle step on 16 host threads)."""
    mesh = inputs.periodic_grid(4096)
    W0 = inputs.khi_state(mesh)
    m, s = make_state(rd, mesh, W0, "B2")
    dts = [s.step(return_dt=True) for _ in range(5)]
    Wo, dto = oracle.run(mesh, W0, "B2", nsteps=5, nthreads=NTH)
    assert np.allclose(dts, dto, rtol=1e-14, atol=0)
    err = rel_max_err(s.get(), Wo)
    print(f"4096^2 KHI B2, 5 steps: rel max err vs oracle {err:.2e}")
    assert err < TOL


def test_full_size_1024_sod_like_fp32_l1_over_500_steps(rd):
    """1024x1024 Sod-like B2 over the full 500 steps: the FP32 path's L1 density error
    against the FP64 oracle, printed beside the FP64 path's own L1 distance to the
    oracle (B2 amplifies round-off on this state, so even FP64 parts from the oracle
    over 500 steps; the L1 norm, not the max norm, is the stated measure here)."""
    mesh = inputs.periodic_grid(1024, relabel_seed=6)
    W0 = inputs.sod_like_state(mesh)
    Wo, _ = oracle.run(mesh, W0, "B2", nsteps=500, nthreads=NTH)
    V = oracle.geometry(mesh)["V"]
    out = {}
    for prec in ("fp32", "fp64"):
        m, s = make_state(rd, mesh, W0, "B2", precision=prec)
        assert s.run(500) == 500
        out[prec] = exact.l1_error(V, s.get()[0], Wo[0])
        s.close()
        m.close()
    print(f"1024^2 Sod-like B2, 500 steps: L1 density error vs FP64 oracle: FP32 {out['fp32']:.3e}, "
          f"FP64 {out['fp64']:.3e}")
    assert out["fp32"] < 5e-3
    assert out["fp64"] < out["fp32"]


def test_full_size_4096_in_the_benchmarked_configuration(rd):
    """The configuration bench.py times: 4096^2 KHI B2 with the autotuned launch shapes
    (and tiling), two steps through the captured CUDA graph of rd_run, FP64 against the
    oracle at 1e-12 and FP32 by its L1 density error."""
    mesh = inputs.periodic_grid(4096)
    W0 = inputs.khi_state(mesh)
    m = rd.Mesh(mesh, reorder="morton")
    s = rd.State(m, W0, scheme="B2")
    shapes = s.autotune()
    assert s.run(2) == 2
    Wo, dto = oracle.run(mesh, W0, "B2", nsteps=2, nthreads=NTH)
    err = rel_max_err(s.get(), Wo)
    print(f"4096^2 B2, shapes {shapes}, 2 graph steps: rel max err {err:.2e}")
    assert err < TOL
    s.close()
    s32 = rd.State(m, W0, scheme="B2", precision="fp32")
    s32.autotune()  # may keep the tiled step (rd_state_set_tiling)
    assert s32.run(2) == 2
    l1 = exact.l1_error(oracle.geometry(mesh)["V"], s32.get()[0], Wo[0])
    print(f"4096^2 B2 FP32 (tiling {s32.tiling()}), 2 graph steps: L1 density error vs the FP64 oracle {l1:.2e}")
    assert l1 < 1e-6
