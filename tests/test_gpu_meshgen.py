"""GPU Delaunay refinement of a periodic domain (Sec. 2.3, 2.4, 4.1) checked
by the exact integer checker: the output is a valid periodic triangulation in
which every edge is locally Delaunay (so it is THE Delaunay triangulation of
its vertices) and every triangle meets the size and quality bounds; runs are
deterministic; the mesh feeds the solver, which matches the oracle on it."""
import os

import numpy as np
import pytest

import oracle
from oracle import meshcheck
from paper_1705_02028_gb300 import inputs
from tests._gpu import rel_max_err, require_gpu

pytestmark = pytest.mark.gpu
B = 2.0 ** 0.5


@pytest.fixture(scope="module")
def rd():
    require_gpu()
    from paper_1705_02028_gb300 import binding
    return binding


def _check(mesh, info, R):
    return meshcheck.check(info["xy_units"], info["Px"], info["Py"], mesh.tri, mesh.shift,
                           R_units=R / info["unit"], B=B)


@pytest.mark.parametrize("R,Ly,nx0", [(0.05, 1.0, 4), (0.02, 0.6, 3), (0.008, 1.0, 5)])
def test_refined_mesh_is_delaunay_and_meets_bounds(rd, R, Ly, nx0):
    mesh, info = rd.meshgen(R, Lx=1.0, Ly=Ly, nx0=nx0, ny0=nx0)
    assert info["status"] == 0
    r = _check(mesh, info, R)
    print(f"R={R} Ly={Ly}: {mesh.nv} vertices, {mesh.nt} triangles, {info['rounds']} rounds, "
          f"{info['flips']} flips; max beta {r['max_beta']:.3f}, min angle {r['min_angle_deg']:.1f} deg")
    for key in ("coords_in_box", "all_ccw", "area_tiles_box", "every_edge_has_twin", "euler_torus",
                "delaunay", "size_bound", "quality_bound"):
        assert r[key], key
    assert r["min_angle_deg"] > 20.7                    # beta <= sqrt 2
    assert mesh.Ly == pytest.approx(Ly, rel=1e-8)


def test_deterministic_and_seeded(rd):
    a, ia = rd.meshgen(0.02, seed=11)
    b, ib = rd.meshgen(0.02, seed=11)
    c, _ = rd.meshgen(0.02, seed=12)
    assert np.array_equal(ia["xy_units"], ib["xy_units"]) and np.array_equal(a.tri, b.tri)
    assert np.array_equal(a.shift, b.shift) and ia["rounds"] == ib["rounds"]
    assert a.nv != c.nv or not np.array_equal(a.xy, c.xy)


def test_capacity_limit_leaves_a_valid_delaunay_mesh(rd):
    mesh, info = rd.meshgen(0.01, max_vertices=600)
    assert info["status"] == rd.RD_ENOMEM and mesh.nv <= 600
    r = meshcheck.check(info["xy_units"], info["Px"], info["Py"], mesh.tri, mesh.shift)
    assert r["delaunay"] and r["every_edge_has_twin"] and r["area_tiles_box"]
    with pytest.raises(rd.RDError) as e:
        rd.meshgen(0.05, nx0=2)
    assert e.value.status == rd.RD_EINVAL


def test_generated_mesh_runs_the_solver(rd):
    """The paper's workflow: a refined unstructured mesh, then the hydrodynamics on it."""
    mesh, info = rd.meshgen(0.03, seed=3)
    W0 = inputs.vortex_state(mesh)
    m = rd.Mesh(mesh, reorder="morton")
    s = rd.State(m, W0, scheme="B2")
    assert s.run(60) == 60
    Wld, _ = oracle.run(mesh, W0, "B2", nsteps=60, nthreads=max(1, min(16, os.cpu_count() or 1)), long_double=True)
    assert rel_max_err(s.get(), Wld) < 1e-12


def test_benchmark_size_mesh_is_delaunay_and_meets_bounds(rd):
    """The mesh the benchmark generates (circumradius <= 7.3e-4, beta <= sqrt 2: about
    1.29 million vertices and 2.58 million triangles, the size of the paper's mesh
    generation test) passes every check of the exact checker."""
    R = 7.3e-4
    mesh, info = rd.meshgen(R)
    assert info["status"] == 0
    r = _check(mesh, info, R)
    print(f"R={R}: {mesh.nv} vertices, {mesh.nt} triangles, {info['rounds']} rounds, {info['flips']} flips; "
          f"max beta {r['max_beta']:.4f}, min angle {r['min_angle_deg']:.2f} deg, "
          f"cocircular edges {r['cocircular_edges']}")
    assert mesh.nv > 1_200_000
    for key in ("coords_in_box", "all_ccw", "area_tiles_box", "every_edge_has_twin", "euler_torus",
                "delaunay", "size_bound", "quality_bound"):
        assert r[key], key
