"""Tiled step (rd_state_set_tiling) against the untiled step and the oracle.

The tiled kernels compute every share with the same per-triangle code and sum
every vertex's corners in the same CSR order as the untiled step, so the two
states must be bitwise identical after any number of steps: that is checked
for every scheme, both precisions, structured and unstructured meshes, tile
sizes that leave a ragged last tile, and meshes with walls and ghost vertices
(where only stage 1 is tiled).  The tiled FP64 step is also held to the
oracle at 1e-12 (Sec. 3.4's B scheme, the KHI and vortex states)."""
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
    torch = require_gpu()
    from paper_1705_02028_gb300 import binding
    return torch, binding


def _pair(binding, mesh, W0, scheme, precision, tt, bt, reorder="morton", steps=20, use_run=True):
    m = binding.Mesh(mesh, reorder=reorder)
    a = binding.State(m, W0, scheme=scheme, precision=precision)
    b = binding.State(m, W0, scheme=scheme, precision=precision)
    b.set_tiling(tt, bt)
    assert b.tiling()[:2] == (tt, bt)
    if use_run:
        assert a.run(steps) == steps
        assert b.run(steps) == steps
    else:
        for _ in range(steps):
            a.step()
            b.step()
    Wa, Wb = a.get(), b.get()
    ta, tb = a.time(), b.time()
    nb = b.tiling()[2]
    for s in (a, b):
        s.close()
    m.close()
    return Wa, Wb, ta, tb, nb


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["B2", "N1", "LDA2", "BMAX2", "BMIN2", "B2_SL", "BX2"])
def test_tiled_equals_untiled_khi(rd, scheme, precision):
    _, binding = rd
    mesh = inputs.periodic_grid(72, relabel_seed=6)  # 10368 triangles: ragged last tile for every tt
    W0 = inputs.khi_state(mesh)
    Wa, Wb, ta, tb, nb = _pair(binding, mesh, W0, scheme, precision, 256, 128)
    assert nb > 0
    assert np.array_equal(Wa, Wb), f"max diff {np.abs(Wa - Wb).max():.3e}"
    assert ta == tb


@pytest.mark.parametrize("tt,bt", [(32, 32), (64, 64), (128, 128), (160, 64), (512, 256), (1024, 256),
                                   (2048, 128)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiled_tile_shapes_unstructured(rd, tt, bt, precision):
    _, binding = rd
    mesh = inputs.jittered_grid(90, 70, 1.0, 0.8, seed=6, diagonal="random", relabel_seed=6)
    W0 = inputs.khi_state(mesh)
    try:
        Wa, Wb, ta, tb, _ = _pair(binding, mesh, W0, "B2", precision, tt, bt, steps=15, use_run=False)
    except binding.RDError as e:  # a tile too large for the shared memory of one block
        assert e.status == binding.RD_ENOTSUP and tt >= 1024
        return
    assert np.array_equal(Wa, Wb)
    assert ta == tb


@pytest.mark.parametrize("reorder", ["morton", "rcm"])
def test_tiled_equals_untiled_reorders(rd, reorder):
    _, binding = rd
    mesh = inputs.jittered_grid(64, seed=3, relabel_seed=6)
    W0 = inputs.vortex_state(mesh)
    Wa, Wb, ta, tb, _ = _pair(binding, mesh, W0, "B2", "fp64", 128, 64, reorder=reorder, steps=25)
    assert np.array_equal(Wa, Wb)
    assert ta == tb


@pytest.mark.parametrize("scheme", ["B2", "N1", "BX2"])
def test_tiled_walls_and_ghosts(rd, scheme):
    """Stage 1 tiled, stage 2 per triangle (walls / ghost vertices)."""
    _, binding = rd
    for mesh in (inputs.bounded_grid(40, 24, Ly=0.6, periodic_x=True, bc_y="wall", relabel_seed=2),
                 inputs.bounded_grid(36, 30, bc_x="ghost", bc_y="wall", relabel_seed=3)):
        W0 = inputs.sod_like_state(mesh)
        Wa, Wb, ta, tb, _ = _pair(binding, mesh, W0, scheme, "fp64", 128, 128, steps=30)
        assert np.array_equal(Wa, Wb)
        assert ta == tb


def test_tiled_oracle_parity(rd):
    _, binding = rd
    mesh = inputs.periodic_grid(64, relabel_seed=6)
    W0 = inputs.khi_state(mesh)
    m = binding.Mesh(mesh)
    s = binding.State(m, W0, scheme="B2")
    s.set_tiling(128, 64)
    assert s.run(100) == 100
    Wo, dto = oracle.run(mesh, W0, "B2", nsteps=100, nthreads=NTH)
    err = rel_max_err(s.get(), Wo)
    print(f"tiled B2 FP64 64^2 KHI 100 steps: max rel err vs oracle {err:.2e}")
    assert err < 1e-12
    t, n = s.time()
    assert n == 100 and t == pytest.approx(dto.sum(), rel=1e-13)
    s.close()
    m.close()


def test_tiled_errors_and_switching(rd):
    _, binding = rd
    mesh = inputs.periodic_grid(40, relabel_seed=6)
    W0 = inputs.vortex_state(mesh)
    m0 = binding.Mesh(mesh, reorder="none")
    s0 = binding.State(m0, W0)
    with pytest.raises(binding.RDError) as e:  # triangles not sorted by smallest vertex
        s0.set_tiling(256, 128)
    assert e.value.status == binding.RD_ENOTSUP
    assert s0.tiling() == (0, 0, 0)
    for tt, bt in ((0 + 16, 32), (256, 48), (256, 512), (8192, 128), (-32, 32)):
        with pytest.raises(binding.RDError) as e:
            s0.set_tiling(tt, bt)
        assert e.value.status == binding.RD_EINVAL
    s0.close()
    m0.close()
    # switching tiling on and off between runs keeps the trajectory of the untiled step
    m = binding.Mesh(mesh)
    a = binding.State(m, W0)
    b = binding.State(m, W0)
    a.run(12)
    for k, (tt, bt) in enumerate(((128, 64), (0, 0), (256, 256), (64, 32))):
        b.set_tiling(tt, bt)
        b.run(3)
    assert np.array_equal(a.get(), b.get())
    a.close()
    b.close()
    m.close()


def test_tiled_nonphysical_and_autotune(rd):
    _, binding = rd
    # Noh with the B scheme is non-physical from the first step (the paper runs Noh with N)
    mesh = inputs.noh_quadrant(40, relabel_seed=1)
    W0 = inputs.noh_state(mesh)
    m = binding.Mesh(mesh)
    s = binding.State(m, W0, scheme="B2", gamma=5.0 / 3.0)
    s.set_tiling(128, 128)
    with pytest.raises(binding.RDError) as e:
        s.run(5)
    assert e.value.status == binding.RD_ENONPHYSICAL
    s.close()
    m.close()
    # the autotuner may keep or drop the tiling; the trajectory is the same either way
    mesh = inputs.periodic_grid(96, relabel_seed=6)
    W0 = inputs.khi_state(mesh)
    m = binding.Mesh(mesh)
    a = binding.State(m, W0, precision="fp32")
    b = binding.State(m, W0, precision="fp32")
    b.autotune()
    tt, bt, _ = b.tiling()
    print(f"autotune on 96^2 FP32: tiling {tt} x {bt}")
    a.run(10)
    b.run(10)
    assert np.array_equal(a.get(), b.get())
    for x in (a, b):
        x.close()
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["B2", "N1", "BMIN2", "B2_SL", "BX2"])
@pytest.mark.parametrize("tt,bt", [(256, 128), (512, 256), (96, 64)])
def test_staged_geometry_tiles_equal_untiled(rd, scheme, precision, tt, bt):
    """Tiles whose geometry is staged in shared memory (RD_TILE_STAGE_GEOMETRY) give
    the untiled step's states bitwise, on a mesh with a ragged last tile."""
    _, binding = rd
    mesh = inputs.periodic_grid(72, 61, Lx=1.0, Ly=61 / 72, relabel_seed=6)
    W0 = inputs.khi_state(mesh)
    m = binding.Mesh(mesh, reorder="morton")
    a = binding.State(m, W0, scheme=scheme, precision=precision)
    b = binding.State(m, W0, scheme=scheme, precision=precision)
    b.set_tiling(tt, bt, stage_geometry=True)
    assert b.tiling()[:2] == (tt, bt) and b.tiling_flags() == 1
    assert a.run(15) == 15 and b.run(15) == 15
    assert np.array_equal(a.get(), b.get())
