"""Tile plan of the tiled step, checked on the host (no GPU): the C++ checker
next to this file links the library's mesh store and plan builder and checks
every invariant the tiled kernels index with -- the tiles' vertex ranges
partition the vertices, every corner of an interior vertex lies in its own
tile's shared-memory records, every corner of a boundary vertex is flagged
for device memory, and every corner slot maps back to its vertex within the
slot bound -- on structured, jittered and walled meshes, for Morton and RCM
order and tile sizes that leave a ragged last tile."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from paper_1705_02028_gb300 import binding, build, inputs

HERE = os.path.dirname(os.path.abspath(__file__))
TILES = ["32", "64", "96", "128", "256", "512", "1024", "4096"]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    binding.load()
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("tile") / "tile_plan_check")
    lib_dir = os.path.dirname(build.LIB)
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", build.CSRC, os.path.join(HERE, "tile_plan_check.cpp"), "-o", out,
                    "-L", lib_dir, "-lrd", "-Wl,-rpath," + lib_dir], check=True)
    return out


def _dump(mesh, path):
    with open(path, "wb") as f:
        sh = mesh.shift
        f.write(struct.pack("<iiddi", mesh.nv, mesh.nt, float(mesh.Lx), float(mesh.Ly), 0 if sh is None else 1))
        f.write(np.ascontiguousarray(mesh.xy, dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(mesh.tri, dtype=np.int32).tobytes())
        if sh is not None:
            f.write(np.ascontiguousarray(sh, dtype=np.int8).tobytes())


def _run(checker, mesh, reorder, tmp_path):
    path = str(tmp_path / "mesh.bin")
    _dump(mesh, path)
    r = subprocess.run([checker, path, str(reorder)] + TILES, capture_output=True, text=True, check=True)
    rows = [ln.split() for ln in r.stdout.strip().splitlines()]
    return {int(w[1]): dict(zip(w[2::2], map(int, w[3::2]))) for w in rows}


MESHES = {
    "grid": lambda: inputs.periodic_grid(61, relabel_seed=6),
    "jittered": lambda: inputs.jittered_grid(70, 50, 1.0, 0.7, seed=6, diagonal="random", relabel_seed=6),
    "walled": lambda: inputs.bounded_grid(40, 24, Ly=0.6, periodic_x=True, bc_y="wall", relabel_seed=2),
}


@pytest.mark.parametrize("reorder", [1, 2])  # RD_ORDER_MORTON, RD_ORDER_RCM
@pytest.mark.parametrize("kind", sorted(MESHES))
def test_tile_plan_invariants(checker, kind, reorder, tmp_path):
    mesh = MESHES[kind]()
    res = _run(checker, mesh, reorder, tmp_path)
    assert set(res) == set(map(int, TILES))
    for tt, r in res.items():
        assert r["rc"] == 0 and r["bad"] == 0, (tt, r)
        assert r["tiles"] == -(-mesh.nt // tt)
        assert 0 <= r["boundary"] <= mesh.nv
    # larger tiles leave fewer boundary vertices; one tile has none
    assert res[4096]["boundary"] <= res[32]["boundary"]
    if mesh.nt <= 4096:
        assert res[4096]["boundary"] == 0


def test_tile_plan_needs_sorted_triangles(checker, tmp_path):
    res = _run(checker, inputs.periodic_grid(24, relabel_seed=6), 0, tmp_path)  # RD_ORDER_NONE
    assert all(r["rc"] == binding.RD_ENOTSUP for r in res.values())
