"""Pins of the oracle's forward-mode derivative (run_tangent, the dual-number
instantiation of the step of Sec. 3.4 with the dt sequence held fixed).

The derivative the adjoint checks rely on is pinned here against things that
do not share its arithmetic: the closed-form derivative rules of each dual
operation, and central differences of the plain double-precision rollout
(oracle.run with the same frozen dt sequence), on maps that are C^1 (N1 and
LDA2 away from the |lambda| kinks; the B blend's Theta has kinks wherever a
residual component changes sign).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1705_02028_gb300 import inputs


@pytest.mark.parametrize("a,da,b,db", [(1.7, 0.3, -2.9, 1.1), (-0.4, -2.0, 0.25, 0.5), (3.0e5, 1e-3, 7e-4, -2.0)])
def test_dual_rules_closed_form(a, da, b, db):
    """d(a+b), d(a-b), d(ab), d(a/b) = (a'b - ab')/b^2, d(-a)."""
    assert oracle.dual_eval("add", a, da, b, db) == pytest.approx((a + b, da + db), rel=1e-15)
    assert oracle.dual_eval("sub", a, da, b, db) == pytest.approx((a - b, da - db), rel=1e-15)
    assert oracle.dual_eval("mul", a, da, b, db) == pytest.approx((a * b, da * b + a * db), rel=1e-15)
    q, dq = oracle.dual_eval("div", a, da, b, db)
    assert q == pytest.approx(a / b, rel=1e-15)
    assert dq == pytest.approx((da * b - a * db) / (b * b), rel=1e-13)
    assert oracle.dual_eval("neg", a, da) == (-a, -da)


@pytest.mark.parametrize("a,da", [(2.25, 0.6), (1e-6, 3.0), (7.0e4, -1.5)])
def test_dual_sqrt_closed_form(a, da):
    s, ds = oracle.dual_eval("sqrt", a, da)
    assert s == pytest.approx(math.sqrt(a), rel=1e-15)
    assert ds == pytest.approx(da / (2.0 * math.sqrt(a)), rel=1e-14)


def test_dual_fabs_sign():
    """d|a| = sign(a) a' away from 0; at a = 0 the oracle takes the right-hand branch (+a')."""
    assert oracle.dual_eval("fabs", -1.5, 0.7) == (1.5, -0.7)
    assert oracle.dual_eval("fabs", 2.5, 0.7) == (2.5, 0.7)
    assert oracle.dual_eval("fabs", 2.5, -0.7) == (2.5, -0.7)
    assert oracle.dual_eval("fabs", 0.0, -0.7) == (0.0, -0.7)


def _drifting_state(mesh, kind):
    """A smooth state moving obliquely (u = 1, v = 0.35), so that no edge normal is
    orthogonal to the flow: there u.n = 0 puts an eigenvalue inside the C^1
    regularisation of |lambda|, whose curvature (1 / delta, delta ~ 1e-6) would
    dominate a finite difference with h = 1e-6."""
    if kind == "smooth":
        rho, _, _, p = inputs.primitives(inputs.smooth_density_state(mesh))
    else:
        rho, _, _, p = inputs.primitives(inputs.vortex_state(mesh))
    return inputs.conserved(rho, np.full_like(rho, 1.0), np.full_like(rho, 0.35), p)


def _direction(mesh, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((4, mesh.nv))
    return d / np.abs(d).max()


@pytest.mark.parametrize("scheme", ["N1", "LDA2"])
@pytest.mark.parametrize("state", ["smooth", "vortex"])
def test_tangent_matches_central_differences(scheme, state):
    """run_tangent == (run(W0 + h d) - run(W0 - h d)) / 2h with the dt sequence frozen,
    on a relabelled 6x6 periodic mesh over 5 steps (h = 1e-6, truncation ~h^2)."""
    mesh = inputs.periodic_grid(6, relabel_seed=6)
    W0 = _drifting_state(mesh, state)
    _, dts = oracle.run(mesh, W0, scheme, nsteps=5)
    d = _direction(mesh, 5) * np.abs(W0).max(axis=1, keepdims=True)
    W, dW = oracle.run_tangent(mesh, W0, d, dts, scheme)
    Wref, _ = oracle.run(mesh, W0, scheme, nsteps=5, dt_fixed=dts)
    assert np.array_equal(W, Wref)  # the value part is the plain rollout
    h = 1e-6
    Wp, _ = oracle.run(mesh, W0 + h * d, scheme, nsteps=5, dt_fixed=dts)
    Wm, _ = oracle.run(mesh, W0 - h * d, scheme, nsteps=5, dt_fixed=dts)
    fd = (Wp - Wm) / (2.0 * h)
    scale = np.abs(dW).max(axis=1, keepdims=True)
    err = float((np.abs(dW - fd) / scale).max())
    assert err < 1e-7, err


def test_tangent_is_linear_in_the_direction():
    """The tangent of a + b equals the sum of the tangents (forward mode is linear)."""
    mesh = inputs.periodic_grid(6, relabel_seed=6)
    W0 = inputs.vortex_state(mesh)
    _, dts = oracle.run(mesh, W0, "B2", nsteps=3)
    a = _direction(mesh, 7)
    b = _direction(mesh, 8)
    _, da = oracle.run_tangent(mesh, W0, a, dts, "B2")
    _, db = oracle.run_tangent(mesh, W0, b, dts, "B2")
    _, dab = oracle.run_tangent(mesh, W0, 2.0 * a - b, dts, "B2")
    assert np.abs(dab - (2.0 * da - db)).max() < 1e-11 * np.abs(dab).max()
