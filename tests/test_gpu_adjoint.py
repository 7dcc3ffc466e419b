"""Discrete adjoint of a rollout (hand-written reverse kernels, checkpoints, branch masks)
against the oracle's forward-mode derivative and against central finite differences."""
import numpy as np
import pytest

import oracle
from paper_1705_02028_gb300 import inputs
from tests._gpu import rel_max_err, require_gpu

pytestmark = pytest.mark.gpu


def loss_seed(W, target, V):
    """L = 1/2 sum_i V_i (rho_i - rho_i^tgt)^2 and dL/dW."""
    d = W[0] - target[0]
    seed = np.zeros_like(W)
    seed[0] = V * d
    return 0.5 * float(np.sum(V * d * d)), seed


@pytest.fixture(scope="module")
def rd():
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    return torch, binding


@pytest.mark.parametrize("scheme,N,steps,ckpt", [("B2", 20, 30, 7), ("N1", 16, 25, 10), ("LDA2", 14, 12, 5),
                                                 ("B2", 48, 40, 20)])
def test_adjoint_matches_oracle_directional_derivatives(rd, scheme, N, steps, ckpt):
    torch, binding = rd
    mesh = inputs.periodic_grid(N, relabel_seed=7)
    W0 = inputs.smooth_density_state(mesh, seed=3)
    tgt = inputs.smooth_density_state(mesh, seed=4)
    V = oracle.geometry(mesh)["V"]
    m = binding.Mesh(mesh)
    s = binding.State(m, W0, scheme=scheme)
    dts = s.adjoint_forward(steps, ckpt)
    Wf = s.get()
    L, seed = loss_seed(Wf, tgt, V)
    g0 = s.adjoint_backward(seed)
    rng = np.random.default_rng(5)
    for _ in range(3):
        v = rng.normal(size=W0.shape)
        v /= np.linalg.norm(v)
        Wo, dWo = oracle.run_tangent(mesh, W0, v, dts, scheme=scheme)
        assert rel_max_err(Wf, Wo) < 1e-12
        ref = float(np.sum(seed * dWo))
        got = float(np.sum(g0 * v))
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-14 * np.abs(g0).sum()), (got, ref)


@pytest.mark.parametrize("scheme", ["N1", "LDA2", "B2"])
def test_adjoint_512_central_finite_differences(rd, scheme):
    """512x512 periodic mesh, FP64, 200 steps, checkpoints every 20, smooth density
    perturbation (amplitude 0.05); 16 random Gaussian directions (N(0,1) entries, so each
    vertex state moves by ~h), central FD with h = 1e-6 on the same map (the recorded dt
    sequence).  N1 and LDA2 are C^1 maps (the |lambda| regularisation is C^1): FD must
    agree to 1e-6.  B2 is only piecewise smooth: Theta = |t| / max(sum|N|, |t|) has kinks
    where a residual component changes sign, and +-h crosses some of them (the count of
    first-step branch-mask flips is printed); its derivative is checked exactly against
    the oracle's dual numbers above, and here only to 5e-2."""
    torch, binding = rd
    mesh = inputs.periodic_grid(512)
    W0 = inputs.smooth_density_state(mesh, seed=3)
    tgt = inputs.smooth_density_state(mesh, seed=4)
    V = oracle.geometry(mesh)["V"]
    m = binding.Mesh(mesh)
    s = binding.State(m, W0, scheme=scheme)
    base_masks = s.branch_masks()
    dts = s.adjoint_forward(200, 20)
    L0, seed = loss_seed(s.get(), tgt, V)
    g0 = s.adjoint_backward(seed)
    fd = binding.State(m, W0, scheme=scheme)
    rng = np.random.default_rng(5)
    h = 1e-6
    worst, flips = 0.0, 0
    for _ in range(16):
        v = rng.normal(size=W0.shape)
        Ls = []
        for sgn in (1.0, -1.0):
            fd.set(W0 + sgn * h * v)
            m1, m2 = fd.branch_masks()
            flips += int(np.count_nonzero(m1 != base_masks[0]) + np.count_nonzero(m2 != base_masks[1]))
            fd.run_fixed_dt(dts)
            Ls.append(loss_seed(fd.get(), tgt, V)[0])
        d_fd = (Ls[0] - Ls[1]) / (2 * h)
        d_adj = float(np.sum(g0 * v))
        worst = max(worst, abs(d_fd - d_adj) / max(abs(d_adj), 1e-30))
    print(f"adjoint vs central FD ({scheme}, 512^2, 200 steps, 16 Gaussian directions, h=1e-6): "
          f"worst rel diff {worst:.2e}; first-step branch-mask flips under +-h: {flips}")
    if scheme == "B2":
        assert worst < 5e-2
    else:
        assert worst < 1e-6


def test_autograd_function(rd):
    torch, binding = rd
    mesh = inputs.periodic_grid(24, relabel_seed=2)
    W0 = inputs.smooth_density_state(mesh, seed=3)
    tgt = inputs.smooth_density_state(mesh, seed=4)
    V = oracle.geometry(mesh)["V"]
    m = binding.Mesh(mesh)
    s = binding.State(m, W0, scheme="B2")
    w0 = torch.tensor(W0, dtype=torch.float64, requires_grad=True)
    Wf = binding.rollout(s, w0, 15, 4)
    L = 0.5 * torch.sum(torch.tensor(V) * (Wf[0] - torch.tensor(tgt[0])) ** 2)
    L.backward()
    v = np.random.default_rng(1).normal(size=W0.shape)
    # the autograd gradient equals the direct adjoint call on the same rollout
    s2 = binding.State(m, W0, scheme="B2")
    dts = s2.adjoint_forward(15, 4)
    _, seed = loss_seed(s2.get(), tgt, V)
    g = s2.adjoint_backward(seed)
    assert np.allclose(w0.grad.numpy(), g, rtol=1e-14, atol=0)
    Wo, dWo = oracle.run_tangent(mesh, W0, v, dts, "B2")
    assert float(np.sum(g * v)) == pytest.approx(float(np.sum(seed * dWo)), rel=1e-9)

