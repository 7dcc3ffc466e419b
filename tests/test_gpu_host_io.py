"""State upload and download through page-locked host memory.

rd_state_set / rd_get_state read and write a page-locked caller array in place
(host-order kernels over the host link) and stage a pageable one through a
device copy.  Both routes must give bitwise the same device state and the same
host result, and both must reject a non-finite state."""
import numpy as np
import pytest

from paper_1705_02028_gb300 import inputs
from tests._gpu import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    return torch, binding


def pinned(torch, shape):
    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "df64"])
@pytest.mark.parametrize("reorder", ["morton", "rcm"])
def test_pinned_and_pageable_routes_agree(rd, precision, reorder):
    torch, binding = rd
    mesh = inputs.periodic_grid(37, 29, Lx=1.0, Ly=29 / 37, relabel_seed=4)
    W0 = inputs.khi_state(mesh)
    W1 = inputs.vortex_state(mesh)
    m = binding.Mesh(mesh, reorder=reorder)
    a = binding.State(m, W0, scheme="B2", precision=precision)
    b = binding.State(m, W0, scheme="B2", precision=precision)
    # upload: pageable into a, page-locked into b
    a.set(W1)
    Wp = pinned(torch, W1.shape)
    Wp[:] = W1
    b.set(Wp)
    ga, gb = a.get(), b.get()
    assert np.array_equal(ga, gb)
    # download into a page-locked array equals the pageable download
    out = pinned(torch, W1.shape)
    b.get(out=out)
    assert np.array_equal(out, ga)
    if precision != "fp32":
        assert np.array_equal(out, W1)          # FP64 state: the round trip is exact
    # and the steps that follow are the same
    a.run(4)
    b.run(4)
    out2 = pinned(torch, W1.shape)
    b.get(out=out2)
    assert np.array_equal(a.get(), out2)
    a.close()
    b.close()


def test_pinned_upload_rejects_non_finite_state(rd):
    torch, binding = rd
    mesh = inputs.periodic_grid(16)
    W0 = inputs.khi_state(mesh)
    m = binding.Mesh(mesh)
    s = binding.State(m, W0, scheme="B2")
    bad = pinned(torch, W0.shape)
    bad[:] = W0
    bad[2, 7] = np.nan
    with pytest.raises(binding.RDError):
        s.set(bad)
    s.close()
