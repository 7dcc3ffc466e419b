"""GPU path vs the oracle for the scheme variants of Sec. 3.3.3 and Sec. 3.4:
Bmax, Bmin, the Bx shock-sensor blend and selective lumping.  Tolerance as for
the B scheme: 1e-12 relative in the max norm against the oracle's long-double
instantiation (Sod-like runs over their first 20 steps, where the blended
schemes' round-off growth at the resting interface is still below it: 20
steps, 10 for Bmax, whose single max-weight amplifies round-off fastest -- the
oracle's own double and long-double runs part by 6.4e-12 after 20 Bmax steps
on the 48^2 Sod-like state and by 1.7e-13 after 10)."""
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


STATES = {"vortex": inputs.vortex_state, "khi": inputs.khi_state, "sod": inputs.sod_like_state,
          "khis": inputs.khi_smooth_state}


@pytest.mark.parametrize("scheme,state,N,mesh_kind,steps", [
    ("BMAX2", "sod", 48, "grid", 10), ("BMAX2", "khi", 48, "jit", 100),
    ("BMIN2", "vortex", 48, "jit", 100), ("BMIN2", "khis", 40, "grid", 100),
    ("BX2", "khi", 40, "jit", 100), ("BX2", "sod", 40, "grid", 20), ("BX2", "vortex", 32, "grid", 100),
    ("B2_SL", "vortex", 48, "jit", 100), ("LDA2_SL", "vortex", 40, "grid", 100),
    ("BX2_SL", "khi", 32, "grid", 100), ("BMAX2_SL", "sod", 40, "jit", 20)])
def test_variant_parity(rd, scheme, state, N, mesh_kind, steps):
    _, binding = rd
    mesh = inputs.periodic_grid(N, relabel_seed=6) if mesh_kind == "grid" else \
        inputs.jittered_grid(N, relabel_seed=6)
    W0 = STATES[state](mesh)
    m = binding.Mesh(mesh)
    s = binding.State(m, W0, scheme=scheme)
    assert s.run(steps) == steps
    Wld, dto = oracle.run(mesh, W0, scheme, nsteps=steps, nthreads=NTH, long_double=True)
    Wd, _ = oracle.run(mesh, W0, scheme, nsteps=steps, nthreads=NTH)
    err, floor = rel_max_err(s.get(), Wld), rel_max_err(Wd, Wld)
    print(f"{scheme} {state} {N}^2 {mesh_kind} {steps} steps: GPU vs oracle(ld) {err:.2e}, "
          f"oracle(double) vs oracle(ld) {floor:.2e}")
    assert err < TOL
    t, _ = s.time()
    assert t == pytest.approx(dto.sum(), rel=1e-13)


def test_bx_step_by_step_and_after_set(rd):
    """The Bx |v| range follows set() and survives a run stopped at t_end."""
    _, binding = rd
    mesh = inputs.periodic_grid(30, relabel_seed=2)
    W0 = inputs.khi_state(mesh)
    m = binding.Mesh(mesh)
    s = binding.State(m, W0, scheme="BX2")
    s.run(1000, t_end=0.01)
    _, n1 = s.time()
    s.run(7)
    # the t_end-clipped step has a shorter dt: compare against the oracle with that dt sequence
    _, dts = oracle.run(mesh, W0, "BX2", nsteps=n1, long_double=True)
    t1 = 0.01
    dts = np.concatenate([dts[:-1], [t1 - dts[:-1].sum()]])
    Wa, _ = oracle.run(mesh, W0, "BX2", nsteps=n1, dt_fixed=dts, long_double=True)
    Wb, _ = oracle.run(mesh, Wa, "BX2", nsteps=7, long_double=True)
    assert rel_max_err(s.get(), Wb) < TOL
    W1 = inputs.vortex_state(mesh)
    s.set(W1)
    s.run(5)
    Wc, _ = oracle.run(mesh, W1, "BX2", nsteps=5, long_double=True)
    assert rel_max_err(s.get(), Wc) < TOL


def test_variants_fp32(rd):
    _, binding = rd
    mesh = inputs.jittered_grid(64, relabel_seed=6)
    W0 = inputs.vortex_state(mesh)
    m = binding.Mesh(mesh)
    V = oracle.geometry(mesh)["V"]
    for scheme in ("BMAX2", "BMIN2", "BX2", "B2_SL"):
        s = binding.State(m, W0, scheme=scheme, precision="fp32")
        s.run(100)
        Wo, _ = oracle.run(mesh, W0, scheme, nsteps=100, nthreads=NTH)
        l1 = exact.l1_error(V, s.get()[0], Wo[0])
        print(f"FP32 {scheme} L1 density error vs FP64 oracle: {l1:.3e}")
        assert l1 < 2e-6, scheme
        s.close()


def test_batch_variants_and_limits(rd):
    torch, binding = rd
    stream = torch.cuda.Stream()
    cases = []
    for k, N in enumerate((11, 19, 26)):
        mesh = inputs.jittered_grid(N, relabel_seed=k) if k % 2 else inputs.periodic_grid(N, relabel_seed=k)
        cases.append((mesh, inputs.khi_state(mesh, seed=k)))
    meshes = [binding.Mesh(mesh, stream=stream) for mesh, _ in cases]
    for scheme in ("BMIN2_SL", "BMAX2"):
        b = binding.Batch(meshes, [W for _, W in cases], scheme=scheme)
        b.run(25)
        for k, (mesh, W0) in enumerate(cases):
            Wo, _ = oracle.run(mesh, W0, scheme, nsteps=25, long_double=True)
            assert rel_max_err(b.get(k), Wo) < TOL, (scheme, k)
        b.close()
    with pytest.raises(binding.RDError) as e:
        binding.Batch(meshes, [W for _, W in cases], scheme="BX2")
    assert e.value.status == binding.RD_ENOTSUP


def test_parameter_checks(rd):
    _, binding = rd
    mesh = inputs.periodic_grid(12)
    W0 = inputs.vortex_state(mesh)
    m = binding.Mesh(mesh)
    with pytest.raises(binding.RDError) as e:
        binding.State(m, W0, scheme="N1", lumping="selective")
    assert e.value.status == binding.RD_EINVAL
    s = binding.State(m, W0, scheme="BMIN2")
    with pytest.raises(binding.RDError) as e:
        s.adjoint_forward(4)
    assert e.value.status == binding.RD_ENOTSUP
