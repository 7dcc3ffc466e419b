"""Pins of the oracle's time stepping (Sec. 3.2 eqUpdate, Sec. 3.4 eqRK1/eqRK2)."""
import numpy as np
import pytest

import oracle
from paper_1705_02028_gb300 import inputs


def test_geometry_of_regular_grid():
    N = 8
    mesh = inputs.periodic_grid(N, relabel_seed=3)
    g = oracle.geometry(mesh)
    h = 1.0 / N
    assert np.allclose(g["area"], 0.5 * h * h, rtol=1e-14)
    assert np.allclose(g["V"], h * h, rtol=1e-14)            # 6 triangles x |T|/3
    assert np.allclose(g["lmax"], np.sqrt(2.0) * h, rtol=1e-14)
    assert np.allclose(g["normals"].sum(axis=1), 0.0, atol=1e-15)


@pytest.mark.parametrize("vel", [(0.0, 0.0), (0.5, 1.5)])
def test_cfl_time_step_closed_form(vel):
    """Uniform state on the regular grid: dt = CFL h / (3 sqrt(2) (|v| + c))."""
    N = 10
    mesh = inputs.periodic_grid(N)
    rho, p = 1.2, 0.8
    W = inputs.uniform_state(mesh, rho=rho, u=vel[0], v=vel[1], p=p)
    s = np.hypot(*vel) + np.sqrt(1.4 * p / rho)
    expect = 0.8 * (1.0 / N) / (3.0 * np.sqrt(2.0) * s)
    assert oracle.time_step(mesh, W, cfl=0.8) == pytest.approx(expect, rel=1e-14)


@pytest.mark.parametrize("scheme", ["N1", "B2", "LDA2"])
@pytest.mark.parametrize("vel", [(0.0, 0.0), (1.0, 1.0)])
def test_uniform_flow_is_preserved(scheme, vel):
    mesh = inputs.periodic_grid(12, relabel_seed=2)
    W0 = inputs.uniform_state(mesh, rho=1.0, u=vel[0], v=vel[1], p=1.0)
    W, _ = oracle.run(mesh, W0, scheme, nsteps=100)
    assert np.abs(W - W0).max() < 1e-13


@pytest.mark.parametrize("scheme", ["N1", "B2"])
@pytest.mark.parametrize("state", ["vortex", "sod", "khi"])
def test_conservation_on_periodic_mesh(scheme, state):
    mesh = inputs.periodic_grid(24, relabel_seed=4)
    W0 = {"vortex": inputs.vortex_state, "sod": inputs.sod_like_state,
          "khi": inputs.khi_state}[state](mesh)
    c0 = oracle.conserved(mesh, W0)
    W, _ = oracle.run(mesh, W0, scheme, nsteps=100, nthreads=4)
    c1 = oracle.conserved(mesh, W)
    scale = np.abs(c0).max()
    assert np.abs(c1 - c0).max() < 2e-14 * scale


def test_stage2_total_residuals_sum_to_triangle_total():
    mesh = inputs.periodic_grid(10, relabel_seed=7)
    Wn = inputs.vortex_state(mesh)
    dt = oracle.time_step(mesh, Wn)
    Ws, _ = oracle.run(mesh, Wn, "N1", nsteps=1)  # some nearby admissible state as W*
    t = oracle.stage2_terms(mesh, Wn, Ws, dt)
    sc = np.abs(t["PhiN"]).max()
    assert np.allclose(t["PhiN"].sum(axis=1), t["PhiT"], atol=1e-12 * sc)
    assert np.allclose(t["PhiLDA"].sum(axis=1), t["PhiT"], atol=1e-12 * sc)
    assert np.allclose(t["Phi"].sum(axis=1), t["PhiT"], atol=1e-12 * sc)
    assert np.all(t["theta"] >= 0) and np.all(t["theta"] <= 1 + 1e-14)


def test_stage2_with_Wstar_equal_Wn_reduces_to_stage1():
    """W* = W^n: Phi^N_i = phi^N_i(W^n) and Phi^LDA_i = beta_i phi^T (Sec. 3.4)."""
    mesh = inputs.periodic_grid(8, relabel_seed=9)
    Wn = inputs.khi_state(mesh, seed=5)
    s1 = oracle.triangle_terms(mesh, Wn)
    s2 = oracle.stage2_terms(mesh, Wn, Wn, 1e-3)
    assert np.allclose(s2["PhiN"], s1["phiN"], rtol=1e-13, atol=1e-15)
    assert np.allclose(s2["PhiLDA"], s1["phiLDA"], rtol=1e-13, atol=1e-15)
    assert np.allclose(s2["Phi"], s1["phiB"], rtol=1e-12, atol=1e-15)


def test_threads_are_bitwise_deterministic():
    mesh = inputs.periodic_grid(16, relabel_seed=1)
    W0 = inputs.khi_state(mesh)
    a, _ = oracle.run(mesh, W0, "B2", nsteps=5, nthreads=1)
    b, _ = oracle.run(mesh, W0, "B2", nsteps=5, nthreads=4)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("state", ["vortex", "khi"])
def test_round_off_floor_long_double(state):
    """double vs long double oracle: the achievable parity floor is far below 1e-12."""
    mesh = inputs.periodic_grid(16, relabel_seed=1)
    W0 = {"vortex": inputs.vortex_state, "khi": inputs.khi_state}[state](mesh)
    a, da = oracle.run(mesh, W0, "B2", nsteps=20)
    b, db = oracle.run(mesh, W0, "B2", nsteps=20, long_double=True)
    scale = np.abs(b).max(axis=1, keepdims=True)
    assert (np.abs(a - b) / scale).max() < 1e-13


def test_relabelling_does_not_change_the_solution():
    """The scheme is defined per triangle; vertex / triangle labels only change round-off."""
    m0 = inputs.periodic_grid(12)
    m1 = inputs.periodic_grid(12, relabel_seed=8)
    a, _ = oracle.run(m0, inputs.vortex_state(m0), "B2", nsteps=10)
    b, _ = oracle.run(m1, inputs.vortex_state(m1), "B2", nsteps=10)
    a_by_orig = a[:, np.argsort(m0.orig_vertex)]
    b_by_orig = b[:, np.argsort(m1.orig_vertex)]
    assert np.abs(a_by_orig - b_by_orig).max() < 1e-13


def test_nonphysical_state_is_rejected():
    mesh = inputs.periodic_grid(6)
    W0 = inputs.uniform_state(mesh)
    W0[3, 5] = -1.0
    with pytest.raises(oracle.OracleError):
        oracle.run(mesh, W0, "B2", nsteps=1)


def test_b2_amplifies_round_off_on_sod_like_state():
    """Evidence for the parity policy: on the Sod-like state the blended two-stage
    scheme (Theta from the total residuals, Sec. 3.4) amplifies round-off -- the
    oracle's own double and long-double runs part -- while N1 and LDA2 stay at
    round-off.  On the smooth KHI state B2 stays at round-off too."""
    mesh = inputs.periodic_grid(32, relabel_seed=6)
    W0 = inputs.sod_like_state(mesh)

    def floor(scheme, n, W=W0):
        a, _ = oracle.run(mesh, W, scheme, nsteps=n, nthreads=4)
        b, _ = oracle.run(mesh, W, scheme, nsteps=n, nthreads=4, long_double=True)
        sc = np.maximum(np.abs(b).max(axis=1), np.abs(b[3]).max())
        return float((np.abs(a - b).max(axis=1) / sc).max())

    assert floor("N1", 60) < 1e-14
    assert floor("B2", 15) < 1e-13
    assert floor("B2", 60) > 1e-8
    assert floor("B2", 60, inputs.khi_state(mesh)) < 1e-13
