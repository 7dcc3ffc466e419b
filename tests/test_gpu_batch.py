"""Batched form: many independent meshes (own sizes, states and dt) in one graph launch."""
import numpy as np
import pytest

import oracle
from paper_1705_02028_gb300 import inputs
from tests._gpu import rel_max_err, require_gpu

pytestmark = pytest.mark.gpu

CASES = [(8, "vortex"), (13, "khi"), (20, "sod"), (31, "smooth"), (40, "vortex"), (17, "khi")]


def make_case(N, kind, k):
    mesh = inputs.periodic_grid(N, relabel_seed=10 + k)
    W = {"vortex": inputs.vortex_state, "khi": lambda m: inputs.khi_state(m, seed=k),
         "sod": inputs.sod_like_state, "smooth": inputs.smooth_density_state}[kind](mesh)
    return mesh, W


@pytest.fixture(scope="module")
def rd():
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    return torch, binding


@pytest.mark.parametrize("scheme", ["B2", "N1"])
def test_batch_matches_oracle_and_plain_path(rd, scheme):
    torch, binding = rd
    stream = torch.cuda.Stream()
    cases = [make_case(N, kind, k) for k, (N, kind) in enumerate(CASES)]
    meshes = [binding.Mesh(m, stream=stream) for m, _ in cases]
    b = binding.Batch(meshes, [W for _, W in cases], scheme=scheme)
    steps = 20
    b.run(steps)
    t, n = b.time()
    assert np.all(n == steps)
    dts = b.dt()
    for k, (mesh, W0) in enumerate(cases):
        Wb = b.get(k)
        Wo, dto = oracle.run(mesh, W0, scheme, nsteps=steps, long_double=True)
        assert rel_max_err(Wb, Wo) < 1e-12, k
        assert t[k] == pytest.approx(dto.sum(), rel=1e-13)
        assert dts[k] == pytest.approx(dto[-1], rel=1e-13)
        # the batched kernels do the plain step's arithmetic in the same order: bitwise equal
        s = binding.State(meshes[k], W0, scheme=scheme)
        s.run(steps)
        assert np.array_equal(s.get(), Wb), k
        s.close()
    b.close()


def test_autotune_keeps_results_bitwise(rd):
    torch, binding = rd
    stream = torch.cuda.Stream()
    cases = [make_case(N, kind, k) for k, (N, kind) in enumerate(CASES[:4])]
    meshes = [binding.Mesh(m, stream=stream) for m, _ in cases]
    b1 = binding.Batch(meshes, [W for _, W in cases])
    b2 = binding.Batch(meshes, [W for _, W in cases])
    tb, vb = b2.autotune()
    assert tb in (64, 128, 192, 256) and vb in (128, 256, 512)
    b1.run(12)
    b2.run(5)
    b2.run(7)
    for k in range(len(cases)):
        assert np.array_equal(b1.get(k), b2.get(k))
    s = binding.State(meshes[0], cases[0][1])
    ref = binding.State(meshes[0], cases[0][1])
    s.autotune()
    s.run(9)
    ref.run(9)
    assert np.array_equal(s.get(), ref.get())


def test_batch_fp32_runs_close_to_fp64(rd):
    torch, binding = rd
    stream = torch.cuda.Stream()
    cases = [make_case(N, kind, k) for k, (N, kind) in enumerate(CASES[:3])]
    meshes = [binding.Mesh(m, stream=stream) for m, _ in cases]
    b64 = binding.Batch(meshes, [W for _, W in cases], precision="fp64")
    b32 = binding.Batch(meshes, [W for _, W in cases], precision="fp32")
    b64.run(10)
    b32.run(10)
    for k in range(len(cases)):
        assert rel_max_err(b32.get(k), b64.get(k)) < 1e-4
