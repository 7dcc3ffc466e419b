"""Physics pins of the oracle against closed-form solutions (Sec. 5 of the paper).

* isentropic vortex (Sec. 5.2.1): exact translation; observed order ~1 for N1,
  ~2 for LDA2 and approaching 2 for B2,
* linear sound wave (Sec. 5.1.1): order 1 for N, ~2 for B/LDA near h ~ 0.01,
* Sod shock tube on a triangulated strip (Sec. 5.1.2): L1 against the exact
  Riemann solution, N1 monotone, sublinear convergence.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1705_02028_gb300 import inputs

NTH = max(1, min(8, os.cpu_count() or 1))
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_exact_riemann_solver_matches_printed_sod_star_state():
    g = json.load(open(os.path.join(GOLDEN, "sod_star_state.json")))
    ps, us = exact.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert ps == pytest.approx(g["p_star"], abs=6e-6)
    assert us == pytest.approx(g["u_star"], abs=6e-6)
    rho, u, p = exact.riemann_exact((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), np.array([0.5, 1.2]))
    assert rho[0] == pytest.approx(g["rho_star_left"], abs=6e-6)
    assert rho[1] == pytest.approx(g["rho_star_right"], abs=6e-6)


def test_vortex_initial_state_is_in_radial_equilibrium():
    """dp/dr = rho r Omega^2 for the closed form of Sec. 5.2.1 (paper units)."""
    r = np.linspace(0.3, 3.0, 50)
    d = 1e-6
    beta, g = 5.0, 1.4

    def prim(rr):
        rho, u, v, p = inputs.vortex_primitives(0.5 + rr / 10.0, 0.5, u0=0.0, v0=0.0)
        return rho, v, p

    rho, vt, p = prim(r)
    _, _, pp = prim(r + d)
    _, _, pm = prim(r - d)
    dpdr = (pp - pm) / (2 * d)
    omega = beta * np.exp((1 - r * r) / 2) / (2 * np.pi)
    assert np.allclose(vt, omega * r, rtol=1e-12)
    assert np.allclose(dpdr, rho * r * omega ** 2, rtol=1e-7)


def _vortex_l1(N, scheme, T=0.05):
    m = inputs.periodic_grid(N)
    W0 = inputs.vortex_state(m)
    n = int(np.ceil(T / oracle.time_step(m, W0)))
    W, _ = oracle.run(m, W0, scheme, nsteps=n, dt_fixed=np.full(n, T / n), nthreads=NTH)
    ex = inputs.vortex_state(m, t=T)
    return exact.l1_error(oracle.geometry(m)["V"], W[0], ex[0])


@pytest.mark.slow
def test_vortex_convergence_orders():
    e = {s: [_vortex_l1(N, s) for N in (64, 128)] for s in ("N1", "B2", "LDA2")}
    order = {s: np.log2(v[0] / v[1]) for s, v in e.items()}
    assert 0.8 < order["N1"] < 1.2, order
    assert order["LDA2"] > 1.8, order
    assert order["B2"] > 1.45, order
    assert e["B2"][1] < e["N1"][1] / 3


def _sound_l1(Nx, scheme, T=1.0):
    m = inputs.periodic_grid(Nx, 4, Lx=1.0, Ly=4.0 / Nx)
    W0 = inputs.sound_wave_state(m)
    n = int(np.ceil(T / oracle.time_step(m, W0)))
    W, _ = oracle.run(m, W0, scheme, nsteps=n, dt_fixed=np.full(n, T / n), nthreads=NTH)
    ex = inputs.sound_wave_state(m, t=T)
    return exact.l1_error(oracle.geometry(m)["V"], W[0], ex[0])


def test_sound_wave_convergence_orders():
    e = {s: [_sound_l1(N, s) for N in (32, 64, 128)] for s in ("N1", "B2")}
    oN = np.log2(e["N1"][1] / e["N1"][2])
    oB = np.log2(e["B2"][1] / e["B2"][2])
    assert 0.8 < oN < 1.2
    assert oB > 1.7
    assert max(e["N1"]) < 1e-4 * 0.5  # far below the wave amplitude 1e-4


def _sod(Nx, scheme, T=0.2):
    m = inputs.periodic_grid(2 * Nx, 4, Lx=2.0, Ly=4.0 / Nx)
    W = inputs.sod_strip_state(m)
    t = 0.0
    while t < T - 1e-14:
        dt = min(oracle.time_step(m, W), T - t)
        W, _ = oracle.run(m, W, scheme, nsteps=1, dt_fixed=[dt])
        t += dt
    x = m.xy[:, 0]
    sel = x <= 1.0
    r, _, _ = exact.riemann_exact((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x[sel] - 0.5) / T)
    return exact.l1_error(oracle.geometry(m)["V"][sel], W[0][sel], r), W, m


def test_sod_strip_against_exact_riemann_solution():
    eN1, WN, m = _sod(50, "N1")
    eN2, _, _ = _sod(100, "N1")
    eB1, WB, _ = _sod(50, "B2")
    eB2, _, _ = _sod(100, "B2")
    # N scheme is monotone: no new extrema (Sec. 5.1.2)
    assert WN[0].min() >= 0.125 - 1e-12 and WN[0].max() <= 1.0 + 1e-12
    # B scheme: only very minor overshoots
    assert WB[0].max() < 1.0 + 2e-3 and WB[0].min() > 0.125 - 5e-3
    # sublinear convergence, B better than N
    for a, b in ((eN1, eN2), (eB1, eB2)):
        order = np.log2(a / b)
        assert 0.35 < order < 1.05
    assert eB2 < eN2
    assert eN2 < 0.025 and eB2 < 0.012
    # the strip stays y-invariant: all rows identical
    rho = WN[0][np.argsort(m.orig_vertex)].reshape(4, -1)
    assert np.abs(rho - rho[0]).max() < 1e-13
