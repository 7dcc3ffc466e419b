"""Kelvin-Helmholtz growth rate (Sec. 5.3, App. C).

The linear-stability solver that seeds the smoothed KHI is pinned first:
with App. C's closure it reproduces the growth rate the paper prints for
d = 0.25, k_x = 2 pi (s = 1.551); on a uniform background its spectrum is the
closed-form acoustic one; and with uniform entropy its two closures agree.
The oracle's B2 scheme is then pinned by the growth it produces: the vertical
kinetic energy grows at a rate that approaches the linear one under refinement
(Sec. 5.3: the schemes converge to the linear result at high resolution; at
32x32 the paper measures s = 1.4 for its second-order blended scheme and 1.3 for
a second-order Roe solver, averaged over 0 < t < 2).
"""
import numpy as np
import pytest

import oracle
from paper_1705_02028_gb300 import inputs

NTH = 4


def test_app_c_closure_reproduces_printed_growth_rate():
    s64, _ = inputs.khi_linear_mode(n=64, closure="adiabatic")
    s128, _ = inputs.khi_linear_mode(n=128, closure="adiabatic")
    assert abs(s128.real - 1.551) < 5e-4
    assert abs(s64 - s128) < 1e-4                       # spectral convergence in n


@pytest.mark.parametrize("closure", ["energy", "adiabatic"])
def test_uniform_background_has_the_acoustic_spectrum(closure):
    """U0 = 0, rho uniform: sigma = +-i c sqrt(kx^2 + (2 pi m)^2) and 0 (entropy/vorticity)."""
    n, kx, p0 = 32, 2.0 * np.pi, 2.5
    _, _ = inputs.khi_linear_mode(kx=kx, U0=0.0, rhoL=1.0, rhoH=1.0, p0=p0, n=n, closure=closure)
    # rebuild the spectrum directly to see every eigenvalue
    c = np.sqrt(1.4 * p0)
    m = np.fft.fftfreq(n, 1.0 / n)
    m[n // 2] = 0.0
    acoustic = c * np.sqrt(kx * kx + (2.0 * np.pi * m) ** 2)
    sig = _spectrum(kx, 0.0, 1.0, 1.0, p0, n, closure)
    assert np.abs(sig.real).max() < 1e-9
    pos = np.sort(sig.imag[sig.imag > 1e-6])
    assert np.allclose(pos, np.sort(acoustic), rtol=1e-10)


def _spectrum(kx, U0, rhoL, rhoH, p0, n, closure):
    # all eigenvalues of the same operator, by perturbing the mode solver's inputs:
    # sigma(U0) for uniform U0 is the U0 = 0 spectrum shifted by -i kx U0
    import numpy.linalg as la
    y = np.arange(n) / n
    u0, r0 = inputs.khi_smooth_profiles(y, 0.25, U0, rhoL, rhoH)
    k = 2.0 * np.pi * np.fft.fftfreq(n, 1.0 / n)
    k[n // 2] = 0.0
    D = np.real(np.fft.ifft(1j * k[:, None] * np.fft.fft(np.eye(n), axis=0), axis=0))
    I, Z = np.eye(n), np.zeros((n, n))
    U, R, Ri = np.diag(u0), np.diag(r0), np.diag(1.0 / r0)
    ik = 1j * kx
    if closure == "energy":
        M = np.block([[-ik * U, -ik * R, -D @ R, Z], [Z, -ik * U, -np.diag(D @ u0), -ik * Ri],
                      [Z, Z, -ik * U, -Ri @ D], [Z, -1.4 * p0 * ik * I, -1.4 * p0 * D, -ik * U]])
    else:
        C2 = np.diag(1.4 * p0 / r0)
        M = np.block([[-ik * U, -ik * R, -D @ R], [-ik * Ri @ C2, -ik * U, -np.diag(D @ u0)],
                      [-Ri @ D @ C2, Z, -ik * U]])
    return la.eigvals(M)


def test_closures_agree_for_uniform_entropy():
    """rho_0 uniform with p_0 constant: p_1 = c_0^2 rho_1 is exact, so both closures agree."""
    se, _ = inputs.khi_linear_mode(rhoL=1.0, rhoH=1.0, n=64, closure="energy")
    sa, _ = inputs.khi_linear_mode(rhoL=1.0, rhoH=1.0, n=64, closure="adiabatic")
    assert abs(se - sa) < 1e-9
    # the whole unstable spectrum agrees (the energy closure adds neutral entropy modes)
    ue = _spectrum(2.0 * np.pi, 0.5, 1.0, 1.0, 2.5, 48, "energy")
    ua = _spectrum(2.0 * np.pi, 0.5, 1.0, 1.0, 2.5, 48, "adiabatic")
    ue, ua = ue[ue.real > 1e-6], ua[ua.real > 1e-6]
    assert len(ue) == len(ua) > 0
    assert np.allclose(np.sort(ue.real), np.sort(ua.real), atol=1e-9)
    assert np.allclose(np.sort(ue.imag), np.sort(ua.imag), atol=1e-9)
    # with a density jump they part: the background entropy then varies with y
    s_e = inputs.khi_linear_mode(n=64, closure="energy")[0]
    s_a = inputs.khi_linear_mode(n=64, closure="adiabatic")[0]
    assert abs(s_e.real - s_a.real) > 0.01


def test_seeded_state_is_the_background_plus_the_mode():
    mesh = inputs.periodic_grid(32)
    W = inputs.khi_smooth_state(mesh, amp=1e-3)
    rho, u, v, p = inputs.primitives(W)
    u0, r0 = inputs.khi_smooth_profiles(mesh.xy[:, 1])
    assert np.abs(v).max() == pytest.approx(1e-3, rel=0.05)
    assert np.abs(rho - r0).max() < 1e-2 and np.abs(u - u0).max() < 1e-2
    assert np.abs(p - 2.5).max() < 1e-2


def measured_growth(mesh, scheme, T=2.0, chunk=0.1):
    """Average growth rate s = ln(E_v(T) / E_v(0)) / (2 T) of the oracle's run."""
    W = inputs.khi_smooth_state(mesh)
    V = oracle.geometry(mesh)["V"]
    E0 = inputs.vertical_kinetic_energy(V, W)
    for _ in range(int(round(T / chunk))):
        n = int(np.ceil(chunk / oracle.time_step(mesh, W)))
        W, _ = oracle.run(mesh, W, scheme, nsteps=n, dt_fixed=np.full(n, chunk / n), nthreads=NTH)
    return np.log(inputs.vertical_kinetic_energy(V, W) / E0) / (2.0 * T)


def test_b2_growth_rate_converges_to_linear_theory():
    s_lin = inputs.khi_linear_mode()[0].real
    s32 = measured_growth(inputs.periodic_grid(32), "B2")
    s64 = measured_growth(inputs.periodic_grid(64), "B2")
    print(f"B2 KHI growth: 32^2 {s32:.4f}, 64^2 {s64:.4f}, linear (energy closure) {s_lin:.4f}")
    assert 1.3 < s32 < 1.5
    assert s32 < s64 < s_lin
    assert s_lin - s64 < 0.08
