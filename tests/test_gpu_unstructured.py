"""GPU path vs the oracle on unstructured periodic meshes (jittered vertices,
Delaunay or random diagonals, valences 4 to 8, scrambled labels): the mesh
store's reorderings, the CSR gather with variable vertex degree, and the
batched form with mixed mesh kinds.  Same tolerance as the regular-grid
parity tests: 1e-12 relative in the max norm against the oracle's long-double
instantiation after 100 steps."""
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
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    return torch, binding


def _mesh(N, M=None, diagonal="delaunay", seed=6):
    M = N if M is None else M
    return inputs.jittered_grid(N, M, Lx=1.0, Ly=M / N, diagonal=diagonal, relabel_seed=seed)


def test_stage1_shares_on_unstructured_mesh(rd):
    _, binding = rd
    mesh = _mesh(29, 23, diagonal="random")
    W = inputs.khi_state(mesh)
    m = binding.Mesh(mesh)
    s = binding.State(m, W, scheme="B2")
    ref = oracle.triangle_terms_ld(mesh, W)
    scale = np.abs(ref["phiN"]).max()
    for which, key in (("N", "phiN"), ("LDA", "phiLDA"), ("B", "phiB")):
        out, _ = s.triangle_shares(which)
        assert np.abs(out - ref[key]).max() <= 1e-11 * scale, which


@pytest.mark.parametrize("reorder", ["none", "morton", "rcm"])
@pytest.mark.parametrize("scheme,state", [("N1", "vortex"), ("B2", "khi"), ("LDA2", "vortex")])
def test_unstructured_100_steps(rd, reorder, scheme, state):
    _, binding = rd
    mesh = _mesh(53, 41)
    W0 = {"vortex": inputs.vortex_state, "khi": inputs.khi_state}[state](mesh)
    m = binding.Mesh(mesh, reorder=reorder)
    s = binding.State(m, W0, scheme=scheme)
    assert s.run(100) == 100
    Wld, dto = oracle.run(mesh, W0, scheme, nsteps=100, nthreads=NTH, long_double=True)
    assert rel_max_err(s.get(), Wld) < TOL
    t, _ = s.time()
    assert t == pytest.approx(dto.sum(), rel=1e-13)


def test_unstructured_conservation_and_fp32(rd):
    _, binding = rd
    mesh = _mesh(64, diagonal="random", seed=9)
    W0 = inputs.vortex_state(mesh)
    m = binding.Mesh(mesh)
    s = binding.State(m, W0, scheme="B2")
    c0 = s.conserved()
    s.run(100)
    assert np.abs(s.conserved() - c0).max() <= 1e-13 * np.abs(c0).max()
    s32 = binding.State(m, W0, scheme="B2", precision="fp32")
    s32.run(100)
    Wo, _ = oracle.run(mesh, W0, "B2", nsteps=100, nthreads=NTH)
    l1 = exact.l1_error(oracle.geometry(mesh)["V"], s32.get()[0], Wo[0])
    print(f"FP32 L1 density error vs FP64 oracle (64^2 jittered vortex, B2, 100 steps): {l1:.3e}")
    assert l1 < 2e-6


def test_batch_with_mixed_mesh_kinds(rd):
    torch, binding = rd
    stream = torch.cuda.Stream()
    cases = []
    for k, (N, kind) in enumerate([(9, "grid"), (14, "jit"), (21, "jit"), (30, "grid"), (17, "jit")]):
        mesh = inputs.periodic_grid(N, relabel_seed=k) if kind == "grid" else _mesh(N, seed=k)
        W = inputs.khi_state(mesh, seed=k) if k % 2 else inputs.vortex_state(mesh)
        cases.append((mesh, W))
    meshes = [binding.Mesh(mesh, stream=stream) for mesh, _ in cases]
    b = binding.Batch(meshes, [W for _, W in cases], scheme="B2")
    b.run(30)
    for k, (mesh, W0) in enumerate(cases):
        Wo, _ = oracle.run(mesh, W0, "B2", nsteps=30, long_double=True)
        assert rel_max_err(b.get(k), Wo) < TOL, k
    b.close()
