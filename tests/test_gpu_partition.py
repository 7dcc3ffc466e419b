"""Vertex-partitioned step on one GPU: P parts of one state, each with its own
owned and ghost vertices and local triangles, advanced with the library's
kernels; ghost states move between the parts' buffers by device copies and dt
is the minimum of the parts' dt.  The owned vertices of all parts together
must equal the single-part step bitwise (every precision and two-stage scheme
the partition offers), and the oracle at 1e-12."""
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


def _gather(parts, nv):
    W = np.full((4, nv), np.nan)
    for p in parts:
        W[:, p.local_vertices[:p.n_owned]] = p.owned()
    return W


@pytest.mark.parametrize("P", [2, 3, 4])
@pytest.mark.parametrize("scheme,precision", [("B2", "fp64"), ("N1", "fp64"), ("LDA2", "fp64"), ("B2", "fp32"),
                                              ("B2", "df64"), ("BMIN2_SL", "fp64")])
def test_parts_equal_single_part_bitwise(rd, P, scheme, precision):
    mesh = inputs.periodic_grid(48, 40, Lx=1.0, Ly=40 / 48, relabel_seed=6)
    W0 = inputs.khi_state(mesh)
    m = rd.Mesh(mesh, reorder="morton")
    steps = 12
    s = rd.State(m, W0, scheme=scheme, precision=precision)
    s.run(steps)
    ref = s.get()
    parts = [rd.Part(m, P, r, W0, scheme=scheme, precision=precision) for r in range(P)]
    assert sum(p.n_owned for p in parts) == mesh.nv
    rd.run_parts_local(parts, steps)
    got = _gather(parts, mesh.nv)
    assert np.array_equal(got, ref)
    for p in parts:
        t, n = p.status()
        assert n == steps
    if precision != "fp32":
        Wld, _ = oracle.run(mesh, W0, scheme, nsteps=steps, nthreads=NTH, long_double=True)
        assert rel_max_err(got, Wld) < 1e-12


def test_parts_on_an_unstructured_mesh_and_rcm_order(rd):
    mesh = inputs.jittered_grid(40, relabel_seed=6)
    W0 = inputs.vortex_state(mesh)
    for reorder in ("morton", "rcm"):
        m = rd.Mesh(mesh, reorder=reorder)
        s = rd.State(m, W0, scheme="B2")
        s.run(10)
        parts = [rd.Part(m, 3, r, W0, scheme="B2") for r in range(3)]
        rd.run_parts_local(parts, 10)
        assert np.array_equal(_gather(parts, mesh.nv), s.get()), reorder


def test_part_options_rejected(rd):
    mesh = inputs.periodic_grid(16)
    W0 = inputs.khi_state(mesh)
    m = rd.Mesh(mesh)
    with pytest.raises(rd.RDError) as e:
        rd.Part(m, 2, 0, W0, scheme="BX2")
    assert e.value.status == rd.RD_ENOTSUP
    with pytest.raises(rd.RDError) as e:
        rd.Part(m, 2, 2, W0)
    assert e.value.status == rd.RD_EINVAL
    box = inputs.bounded_grid(12, 12, periodic_x=True, bc_y="wall")
    mb = rd.Mesh(box)
    with pytest.raises(rd.RDError) as e:
        rd.Part(mb, 2, 0, inputs.khi_state(box))
    assert e.value.status == rd.RD_ENOTSUP
