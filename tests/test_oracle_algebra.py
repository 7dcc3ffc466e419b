"""Pins of the oracle's Appendix-A algebra and per-triangle distributions.

Everything here checks the oracle against mathematics it does not share code
with: the textbook conservative Euler flux (differentiated by complex step),
Simpson quadrature of the boundary flux, and the invariants that the paper's
definitions imply (Sec. 3.2-3.3, App. A).
"""
import numpy as np
import pytest

import oracle
from paper_1705_02028_gb300 import inputs

GAMMA = 1.4


def euler_flux_n(W, nx, ny, gamma=GAMMA):
    """Conservative Euler flux F nx + G ny (textbook form), works for complex W."""
    rho, mx, my, e = W
    u, v = mx / rho, my / rho
    p = (gamma - 1.0) * (e - 0.5 * rho * (u * u + v * v))
    un = u * nx + v * ny
    return np.array([rho * un, mx * un + p * nx, my * un + p * ny, (e + p) * un])


def flux_jacobian_cs(W, nx, ny, gamma=GAMMA):
    """dF.n/dW by complex step (exact to rounding)."""
    J = np.zeros((4, 4))
    hstep = 1e-30
    for k in range(4):
        Wc = np.array(W, dtype=np.complex128)
        Wc[k] += 1j * hstep
        J[:, k] = euler_flux_n(Wc, nx, ny, gamma).imag / hstep
    return J


def random_states(n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.2, 3.0, n)
    u = rng.uniform(-2.0, 2.0, n)
    v = rng.uniform(-2.0, 2.0, n)
    p = rng.uniform(0.1, 3.0, n)
    th = rng.uniform(0, 2 * np.pi, n)
    return rho, u, v, p, np.cos(th), np.sin(th)


def test_K_is_flux_jacobian_and_eigensystem():
    for rho, u, v, p, nx, ny in zip(*random_states(40, 11)):
        W = inputs.conserved(np.array([rho]), u, v, p)[:, 0]
        h = (W[3] + p) / rho
        K, lam, R, L = oracle.eigensystem(u, v, h, nx, ny)
        J = flux_jacobian_cs(W, nx, ny)
        assert np.allclose(K, J, rtol=1e-13, atol=1e-13 * np.abs(J).max())
        c = np.sqrt(GAMMA * p / rho)
        w = u * nx + v * ny
        assert np.allclose(lam, [w + c, w - c, w, w], rtol=1e-14, atol=1e-14)
        # right eigenvectors: K R = R diag(lam); L = R^{-1}
        assert np.allclose(K @ R, R * lam[None, :], atol=1e-12 * np.abs(K).max() * np.abs(R).max())
        assert np.allclose(L @ R, np.eye(4), atol=1e-12)
        assert np.allclose(R @ L, np.eye(4), atol=1e-12)


def one_triangle(x, y):
    """A non-periodic single-triangle mesh (counter-clockwise corners)."""
    return inputs.Mesh(xy=np.array(list(zip(x, y)), dtype=np.float64),
                       tri=np.array([[0, 1, 2]], dtype=np.int32),
                       shift=np.zeros((1, 3, 2), dtype=np.int8), Lx=1.0, Ly=1.0,
                       orig_vertex=np.arange(3))


def to_Z(W):
    rho, u, v, p = inputs.primitives(W)
    h = (W[3] + p) / rho
    s = np.sqrt(rho)
    return np.stack([s, s * u, s * v, s * h])


def from_Z(Z, gamma=GAMMA):
    z1, z2, z3, z4 = Z
    rho = z1 * z1
    u, v, h = z2 / z1, z3 / z1, z4 / z1
    p = (gamma - 1.0) / gamma * (rho * h - 0.5 * rho * (u * u + v * v))
    return inputs.conserved(np.atleast_1d(rho), u, v, p)[:, 0]


def simpson_boundary_flux(xy, Z):
    """phi^T = closed-contour integral of F(Z^h).n_out, Simpson's rule on each edge.

    F is quadratic in Z and Z^h is linear along an edge, so Simpson is exact."""
    tot = np.zeros(4)
    for a, b in ((0, 1), (1, 2), (2, 0)):
        ex, ey = xy[b] - xy[a]
        nout = np.array([ey, -ex])  # outward for a counter-clockwise triangle, |n| = edge length
        fa = euler_flux_n(from_Z(Z[:, a]), *nout)
        fm = euler_flux_n(from_Z(0.5 * (Z[:, a] + Z[:, b])), *nout)
        fb = euler_flux_n(from_Z(Z[:, b]), *nout)
        tot += (fa + 4 * fm + fb) / 6.0
    return tot


def random_triangle_case(seed):
    rng = np.random.default_rng(seed)
    while True:
        x = rng.uniform(0, 1, 3)
        y = rng.uniform(0, 1, 3)
        A = 0.5 * ((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]))
        if abs(A) > 0.05:
            break
    if A < 0:
        x[[1, 2]] = x[[2, 1]]
        y[[1, 2]] = y[[2, 1]]
    rho = rng.uniform(0.5, 2.0, 3)
    u = rng.uniform(-1.5, 1.5, 3)
    v = rng.uniform(-1.5, 1.5, 3)
    p = rng.uniform(0.3, 2.0, 3)
    return one_triangle(x, y), inputs.conserved(rho, u, v, p)


@pytest.mark.parametrize("seed", range(12))
def test_cell_residual_is_boundary_flux_integral(seed):
    mesh, W = random_triangle_case(seed)
    t = oracle.triangle_terms(mesh, W)
    ref = simpson_boundary_flux(mesh.xy, to_Z(W))
    assert np.allclose(t["phiT"][0], ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("seed", range(12))
def test_distribution_invariants(seed):
    mesh, W = random_triangle_case(seed)
    t = oracle.triangle_terms(mesh, W, eps=1e-6)
    phiT = t["phiT"][0]
    sc = np.abs(t["phiN"][0]).max() + np.abs(phiT).max()
    # conservation of every distribution: sum_i phi_i = phi^T
    for key in ("phiN", "phiLDA", "phiB"):
        assert np.allclose(t[key][0].sum(axis=0), phiT, atol=1e-12 * sc), key
    # sum_i beta_i = I (Sec. 3.3.2)
    assert np.allclose(t["beta"][0].sum(axis=0), np.eye(4), atol=1e-11)
    # 0 <= Theta <= 1
    assert np.all(t["theta"][0] >= 0) and np.all(t["theta"][0] <= 1 + 1e-14)
    # K_i^+ + K_i^- = (1/2) dF.n_i/dW at the Roe state; K^+ eigenvalues >= 0, K^- <= 0
    Z = to_Z(W)
    Wroe = from_Z(Z.mean(axis=1))
    g = oracle.geometry(mesh)
    for i in range(3):
        n = g["normals"][0, i]
        J = 0.5 * flux_jacobian_cs(Wroe, n[0], n[1])
        Kp, Km = t["Kp"][0, i], t["Km"][0, i]
        assert np.allclose(Kp + Km, J, atol=1e-12 * np.abs(J).max())
        ep = np.linalg.eigvals(Kp).real
        em = np.linalg.eigvals(Km).real
        assert ep.min() > -1e-10 * np.abs(J).max()
        assert em.max() < 1e-10 * np.abs(J).max()


def test_one_target_supersonic():
    """Supersonic flow with one downstream node: N, LDA and B all send phi^T to it."""
    s3 = np.sqrt(3.0)
    mesh = one_triangle([0.0, 1.0, 0.5], [0.0, 0.0, s3 / 2])
    g = oracle.geometry(mesh)
    n1 = g["normals"][0, 0] / np.linalg.norm(g["normals"][0, 0])
    rng = np.random.default_rng(5)
    rho = 1.0 + 0.1 * rng.uniform(size=3)
    p = 1.0 + 0.1 * rng.uniform(size=3)
    speed = 3.0 * np.sqrt(1.4 * 1.2 / 0.9)   # Mach > 2 everywhere
    W = inputs.conserved(rho, speed * n1[0], speed * n1[1], p)
    t = oracle.triangle_terms(mesh, W)
    phiT = t["phiT"][0]
    for key in ("phiN", "phiLDA", "phiB"):
        sh = t[key][0]
        assert np.allclose(sh[0], phiT, rtol=1e-12, atol=1e-13 * np.abs(phiT).max()), key
        assert np.abs(sh[1:]).max() <= 1e-12 * np.abs(phiT).max(), key


@pytest.mark.parametrize("vel", [(0.0, 0.0), (0.7, -0.3), (3.0, 2.0)])
def test_uniform_state_has_zero_residual(vel):
    mesh = inputs.periodic_grid(6, 5, Lx=1.0, Ly=0.8, relabel_seed=1)
    W = inputs.uniform_state(mesh, rho=1.3, u=vel[0], v=vel[1], p=0.9)
    t = oracle.triangle_terms(mesh, W)
    scale = np.abs(W).max() / 6
    for key in ("phiT", "phiN", "phiLDA", "phiB"):
        assert np.abs(t[key]).max() < 1e-13 * scale, key
