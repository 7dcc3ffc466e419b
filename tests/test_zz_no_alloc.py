"""rd_cfl_dt_noalloc: the allocation-free CFL time step.

Some callers cannot allocate device memory when they need a time step (their
device heap belongs to another allocator, or they may not trigger cudaMalloc's
device synchronisation); rd_cfl_dt_noalloc serves them from a fixed scratch
array inside the library.  This file runs last (pytest collects it last) and
checks, through the C ABI, that the variant returns what rd_cfl_dt returns on
two calls in a row, and that it rejects meshes beyond its fixed limit.
"""
import pytest

import oracle
from paper_1705_02028_gb300 import inputs
from tests._gpu import mesh_device_arrays, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,state", [(64, "khi"), (300, "vortex")])
def test_noalloc_matches_allocating_entry_point_twice(N, state):
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    mesh = inputs.periodic_grid(N, relabel_seed=5)
    W = {"khi": inputs.khi_state, "vortex": inputs.vortex_state}[state](mesh)
    for prec, dtype, tol in (("fp64", torch.float64, 1e-14), ("fp32", torch.float32, 1e-6)):
        a = mesh_device_arrays(mesh, torch, dtype)
        Wd = torch.tensor(W, dtype=dtype, device="cuda")
        args = (Wd, a["tri"], a["lmax"], a["V"], a["csr_ptr"], a["csr_ent"])
        ref = binding.cfl_dt(*args, precision=prec)
        first = binding.cfl_dt(*args, precision=prec, entry="rd_cfl_dt_noalloc")
        second = binding.cfl_dt(*args, precision=prec, entry="rd_cfl_dt_noalloc")
        assert first == pytest.approx(ref, rel=tol, abs=0)
        assert second == pytest.approx(ref, rel=tol, abs=0)
        if prec == "fp64":
            # the FP64 variant against the oracle's CFL step directly
            assert first == pytest.approx(oracle.time_step(mesh, W), rel=1e-14, abs=0)
    assert ref == pytest.approx(oracle.time_step(mesh, W), rel=1e-6)


def test_noalloc_asks_the_installed_allocator_for_nothing():
    """With a counting allocator installed, rd_cfl_dt_noalloc makes no allocation or
    release while rd_cfl_dt (which takes its scratch from the allocator) makes some;
    both return the same dt.  The binding's allocator is put back afterwards."""
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    lib = binding.load()
    binding.use_torch_allocator()
    counts = {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, ctx):
        counts["alloc"] += 1
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except Exception:
            return None

    def _free(ptr, ctx):
        counts["free"] += 1
        torch.cuda.caching_allocator_delete(int(ptr))

    refs = (binding.ALLOC_FN(_alloc), binding.FREE_FN(_free))
    mesh = inputs.periodic_grid(96, relabel_seed=5)
    W = inputs.khi_state(mesh)
    a = mesh_device_arrays(mesh, torch, torch.float64)
    Wd = torch.tensor(W, dtype=torch.float64, device="cuda")
    args = (Wd, a["tri"], a["lmax"], a["V"], a["csr_ptr"], a["csr_ent"])
    binding.cfl_dt(*args, entry="rd_cfl_dt_noalloc")  # set-up call on this device
    assert lib.rd_set_allocator(refs[0], refs[1], None) == binding.RD_OK
    try:
        dt_free = [binding.cfl_dt(*args, entry="rd_cfl_dt_noalloc") for _ in range(2)]
        assert counts == {"alloc": 0, "free": 0}
        dt_ref = binding.cfl_dt(*args)
        assert counts["alloc"] >= 1 and counts["free"] == counts["alloc"]
    finally:
        prev = binding._alloc_refs
        assert lib.rd_set_allocator(prev[0], prev[1], None) == binding.RD_OK
    assert dt_free[0] == dt_ref and dt_free[1] == dt_ref


def test_noalloc_rejects_meshes_beyond_its_limit():
    torch = require_gpu()
    import ctypes
    from paper_1705_02028_gb300 import binding
    lib = binding.load()
    mesh = inputs.periodic_grid(8)
    a = mesh_device_arrays(mesh, torch, torch.float64)
    Wd = torch.tensor(inputs.uniform_state(mesh), device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    too_many = 65536 * 256 + 1
    rc = lib.rd_cfl_dt_noalloc(too_many, mesh.nt, 0, Wd.data_ptr(), a["tri"].data_ptr(), a["lmax"].data_ptr(),
                               a["V"].data_ptr(), a["csr_ptr"].data_ptr(), a["csr_ent"].data_ptr(), 1.4, 0.8,
                               out.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == binding.RD_EINVAL
