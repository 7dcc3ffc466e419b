"""Pins of the scheme variants of Sec. 3.3.3 and Sec. 3.4 in the oracle: the
Bmax / Bmin blends (every diagonal entry of Theta set to max_k or min_k
Theta_kk), the Bx blend with its shock sensor (reading R9: theta = min(1,
s^2 h_T / L), s = max(0, -L div v / (|v|_max - |v|_min))), and selective
lumping (the anti-diffusive correction with the Galerkin mass matrix)."""
import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1705_02028_gb300 import inputs

VARIANTS = ["BMAX2", "BMIN2", "BX2", "B2_SL", "LDA2_SL", "BMAX2_SL", "BMIN2_SL", "BX2_SL"]


@pytest.mark.parametrize("scheme", VARIANTS)
@pytest.mark.parametrize("vel", [(0.0, 0.0), (0.8, -0.3)])
def test_uniform_flow_is_preserved(scheme, vel):
    mesh = inputs.jittered_grid(11, 9, relabel_seed=2)
    W0 = inputs.uniform_state(mesh, rho=1.1, u=vel[0], v=vel[1], p=0.7)
    W, _ = oracle.run(mesh, W0, scheme, nsteps=40)
    assert np.abs(W - W0).max() < 1e-13


@pytest.mark.parametrize("scheme", VARIANTS)
@pytest.mark.parametrize("state", ["sod", "khi"])
def test_conservation(scheme, state):
    if state == "sod" and scheme.startswith("LDA2"):
        pytest.skip("LDA is not positivity preserving at the Sod discontinuity")
    mesh = inputs.periodic_grid(20, relabel_seed=4)
    W0 = {"sod": inputs.sod_like_state, "khi": inputs.khi_state}[state](mesh)
    c0 = oracle.conserved(mesh, W0)
    W, _ = oracle.run(mesh, W0, scheme, nsteps=60, nthreads=4)
    assert np.abs(oracle.conserved(mesh, W) - c0).max() < 2e-14 * np.abs(c0).max()


def _weights(phi, N, L):
    """Per triangle and component: w with phi - L = w (N - L), where N - L is not tiny."""
    d = N - L
    big = np.abs(d) > 1e-8 * np.abs(d).max()
    w = np.where(big, (phi - L) / np.where(big, d, 1.0), np.nan)
    return w, big


def test_bmax_bmin_blend_weights_bracket_theta():
    """Bmax and Bmin are blends of N and LDA with one weight per triangle, equal to
    the largest and the smallest of the B scheme's per-component weights."""
    mesh = inputs.periodic_grid(16, relabel_seed=1)
    W = inputs.khi_state(mesh)
    Wn, _ = oracle.run(mesh, W, "N1", nsteps=5)        # a state with structure at every triangle
    N = oracle.stage1_shares(mesh, Wn, "N1")
    L = oracle.stage1_shares(mesh, Wn, "LDA2")
    wB, big = _weights(oracle.stage1_shares(mesh, Wn, "B2"), N, L)
    theta = np.nanmean(wB, axis=1)                        # (nt, 4): Theta_kk, same over the 3 nodes
    assert np.nanmax(np.nanstd(wB, axis=1)) < 1e-6
    for name, pick in (("BMAX2", np.nanmax), ("BMIN2", np.nanmin)):
        w, _ = _weights(oracle.stage1_shares(mesh, Wn, name), N, L)
        wt = w.reshape(mesh.nt, -1)
        ok = np.isfinite(wt).sum(axis=1) > 0
        spread = np.nanmax(wt[ok], axis=1) - np.nanmin(wt[ok], axis=1)
        assert spread.max() < 1e-6, name                   # one scalar weight per triangle
        full = np.isfinite(theta).all(axis=1) & ok
        assert np.allclose(np.nanmean(wt[full], axis=1), pick(theta[full], axis=1), atol=1e-6), name
    assert np.all((theta[np.isfinite(theta)] >= -1e-9) & (theta[np.isfinite(theta)] <= 1 + 1e-9))


def _divergence(mesh, W):
    """div v of the piecewise-linear vertex velocities, from corner coordinates (2x2 solve)."""
    P = mesh.xy[mesh.tri] + mesh.shift * np.array([mesh.Lx, mesh.Ly])
    u = (W[1] / W[0])[mesh.tri]
    v = (W[2] / W[0])[mesh.tri]
    E = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]], axis=1)        # (nt, 2, 2) edge vectors
    gu = np.linalg.solve(E, np.stack([u[:, 1] - u[:, 0], u[:, 2] - u[:, 0]], axis=1)[..., None])[..., 0]
    gv = np.linalg.solve(E, np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]], axis=1)[..., None])[..., 0]
    area = 0.5 * np.abs(E[:, 0, 0] * E[:, 1, 1] - E[:, 0, 1] * E[:, 1, 0])
    return gu[:, 0] + gv[:, 1], area


def test_bx_sensor():
    """Bx is LDA where the flow expands (div v >= 0) and blends towards N with
    theta = min(1, s^2 h / L) where it compresses."""
    mesh = inputs.jittered_grid(20, relabel_seed=3)
    Wn, _ = oracle.run(mesh, inputs.sod_like_state(mesh), "B2", nsteps=8)
    N = oracle.stage1_shares(mesh, Wn, "N1")
    L = oracle.stage1_shares(mesh, Wn, "LDA2")
    X = oracle.stage1_shares(mesh, Wn, "BX2")
    div, area = _divergence(mesh, Wn)
    rho, u, v, p = inputs.primitives(Wn)
    q = np.hypot(u, v)
    s = np.maximum(0.0, -1.0 * div / (q.max() - q.min()))
    theta = np.minimum(1.0, s * s * np.sqrt(2.0 * area) / 1.0)
    expand = div > 1e-9
    assert expand.sum() > 10 and (div < -1e-9).sum() > 10
    assert np.array_equal(X[expand], L[expand])
    pred = theta[:, None, None] * N + (1 - theta[:, None, None]) * L
    assert np.abs(X - pred).max() < 1e-9 * np.abs(N).max()
    assert (theta > 0.5).sum() > 0 and (theta == 1.0).sum() > 0


def test_bx_equals_lda_without_compression():
    """A density pattern carried by a uniform velocity: div v = 0 and |v|_max =
    |v|_min, so the sensor vanishes and the Bx shares are the LDA shares bitwise."""
    mesh = inputs.jittered_grid(16, relabel_seed=1)
    W0 = inputs.smooth_density_state(mesh)
    assert np.array_equal(oracle.stage1_shares(mesh, W0, "BX2"), oracle.stage1_shares(mesh, W0, "LDA2"))


def test_selective_lumping_correction_closed_form():
    """Phi^SL_i - Phi_i = sum_j (|T| delta_ij / 3 - |T| (delta_ij + 1) / 12) dW_j / dt
    = |T| / 4 dW_i / dt - |T| / 12 sum_j dW_j / dt, which sums to zero over the triangle."""
    mesh = inputs.jittered_grid(9, 8, relabel_seed=5)
    Wn = inputs.vortex_state(mesh)
    dt = oracle.time_step(mesh, Wn)
    Ws, _ = oracle.run(mesh, Wn, "N1", nsteps=1)
    g = oracle.geometry(mesh)
    for base in ("B2", "LDA2", "BMIN2"):
        a = oracle.stage2_terms(mesh, Wn, Ws, dt, scheme=base)["Phi"]
        b = oracle.stage2_terms(mesh, Wn, Ws, dt, scheme=base + "_SL")["Phi"]
        dW = (Ws - Wn).T[mesh.tri] / dt                      # (nt, 3, 4)
        A = g["area"][:, None, None]
        corr = A / 4 * dW - A / 12 * dW.sum(axis=1, keepdims=True)
        assert np.abs((b - a) - corr).max() < 1e-12 * np.abs(a).max(), base
        assert np.abs((b - a).sum(axis=1)).max() < 1e-12 * np.abs(a).max()


def test_sod_strip_blend_ordering():
    """Sod tube (Sec. 5.1.2; 100 cells, t = 0.2): Bmax favours N (no overshoot,
    total variation close to N's), Bmin favours LDA (overshoots, largest total
    variation of the blends); the B scheme sits in between."""
    Nx, T = 100, 0.2
    m = inputs.periodic_grid(2 * Nx, 4, Lx=2.0, Ly=4.0 / Nx)
    W0 = inputs.sod_strip_state(m)
    x, y = m.xy[:, 0], m.xy[:, 1]
    row = (y == y.min()) & (x <= 1.0)
    order = np.argsort(x[row])
    tv, top = {}, {}
    for sch in ("N1", "BMAX2", "B2", "BMIN2"):
        n = int(np.ceil(T / oracle.time_step(m, W0)))
        W, _ = oracle.run(m, W0, sch, nsteps=n, dt_fixed=np.full(n, T / n), nthreads=4)
        r = W[0][row][order]
        tv[sch] = np.abs(np.diff(r)).sum()
        top[sch] = r.max()
    assert tv["N1"] <= tv["BMAX2"] < tv["B2"] < tv["BMIN2"], tv
    assert top["BMAX2"] < 1.0 + 1e-3 < top["BMIN2"], top
