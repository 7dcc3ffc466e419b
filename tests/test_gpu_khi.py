"""Smoothed Kelvin-Helmholtz instability (Sec. 5.3) on the GPU path.

Parity: the seeded linear mode on a 64x64 mesh, B2, 100 steps, against the
oracle's long-double instantiation at 1e-12.  Physics: the vertical kinetic
energy E_v grows at 2 s; the GPU's average growth rate over 0 < t < 2 climbs
towards the linear rate s of the Euler equations as the mesh is refined
(128^2 -> 512^2), in FP64 and in FP32.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1705_02028_gb300 import inputs
from tests._gpu import rel_max_err, require_gpu

pytestmark = pytest.mark.gpu
NTH = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def rd():
    require_gpu()
    from paper_1705_02028_gb300 import binding
    return binding


def test_smooth_khi_parity_100_steps(rd):
    mesh = inputs.periodic_grid(64, relabel_seed=6)
    W0 = inputs.khi_smooth_state(mesh)
    m = rd.Mesh(mesh)
    s = rd.State(m, W0, scheme="B2")
    assert s.run(100) == 100
    Wld, _ = oracle.run(mesh, W0, "B2", nsteps=100, nthreads=NTH, long_double=True)
    assert rel_max_err(s.get(), Wld) < 1e-12


def gpu_growth(rd, N, precision, T=2.0, chunk=0.1):
    mesh = inputs.periodic_grid(N)
    W = inputs.khi_smooth_state(mesh)
    V = oracle.geometry(mesh)["V"]
    E0 = inputs.vertical_kinetic_energy(V, W)
    m = rd.Mesh(mesh)
    s = rd.State(m, W, scheme="B2", precision=precision)
    for k in range(1, int(round(T / chunk)) + 1):
        n = int(1.3 * chunk / oracle.time_step(mesh, W)) + 8
        s.run(n, t_end=k * chunk)
        W = s.get()
    t, _ = s.time()
    assert t == pytest.approx(T, rel=1e-12)
    s.close()
    return np.log(inputs.vertical_kinetic_energy(V, W) / E0) / (2.0 * T)


def test_growth_rate_converges_to_linear_theory(rd):
    s_lin = inputs.khi_linear_mode()[0].real
    s_app_c = inputs.khi_linear_mode(closure="adiabatic")[0].real
    g = {N: gpu_growth(rd, N, "fp64") for N in (128, 256, 512)}
    g32 = gpu_growth(rd, 512, "fp32")
    print(f"KHI growth (B2, FP64): {g}; FP32 512^2 {g32:.4f}; linear: energy closure {s_lin:.4f}, "
          f"App. C closure {s_app_c:.4f}")
    assert g[128] < g[256] < g[512] < s_lin + 2e-3
    assert s_lin - g[512] < 0.01
    assert abs(g32 - g[512]) < 2e-3
