"""Pins of the exact mesh checker used for the GPU mesh generator (Sec. 2.3):
it must accept a valid periodic Delaunay triangulation, flag cocircular
(degenerate) edges, and reject a non-Delaunay edge, a clockwise triangle, a
hole and a non-periodic boundary -- each planted in the input, not in the checker."""
import numpy as np

from oracle import meshcheck
from paper_1705_02028_gb300 import inputs

P = 1 << 20


def units(mesh):
    return np.rint(mesh.xy / mesh.Lx * P).astype(np.int64) % P


def test_regular_grid_is_delaunay_with_cocircular_edges():
    m = inputs.periodic_grid(6)
    r = meshcheck.check(units(m), P, P, m.tri, m.shift)
    assert r["all_ccw"] and r["area_tiles_box"] and r["every_edge_has_twin"] and r["euler_torus"]
    assert r["delaunay"]
    assert r["cocircular_edges"] == 2 * 36            # every cell's diagonal, seen from both sides


def test_jittered_delaunay_cells_and_a_planted_flip():
    m = inputs.jittered_grid(8, jitter=0.05, diagonal="delaunay")
    u = units(m)
    r = meshcheck.check(u, P, P, m.tri, m.shift)
    assert r["every_edge_has_twin"] and r["area_tiles_box"] and r["delaunay"]
    # the other diagonal in one cell: the pair stays a valid triangulation but is not Delaunay
    tri, sh = m.tri.copy(), m.shift.copy()
    # cell 5 holds triangles 10 and 11; flip their shared edge (q, r) to (p, o)
    s10 = {int(v): tuple(x) for v, x in zip(tri[10], sh[10])}
    s11 = {int(v): tuple(x) for v, x in zip(tri[11], sh[11])}
    kp = next(k for k in range(3) if int(tri[10][k]) not in s11)
    p_, q_, r_ = (int(tri[10][(kp + i) % 3]) for i in range(3))
    o_ = next(int(v) for v in tri[11] if int(v) not in s10)
    # express the shifts of triangle 11's far vertex in triangle 10's frame via the shared vertex q
    d = np.subtract(s10[q_], s11[q_])
    so = tuple(np.add(s11[o_], d))
    tri[10], sh[10] = [p_, q_, o_], [s10[p_], s10[q_], so]
    tri[11], sh[11] = [p_, o_, r_], [s10[p_], so, s10[r_]]
    r2 = meshcheck.check(u, P, P, tri, sh)
    assert r2["all_ccw"] and r2["every_edge_has_twin"] and r2["area_tiles_box"]
    assert not r2["delaunay"]


def test_invalid_meshes_are_rejected():
    m = inputs.periodic_grid(5)
    u = units(m)
    tri, sh = m.tri.copy(), m.shift.copy()
    tri[3], sh[3] = tri[3][::-1], sh[3][::-1]          # clockwise
    assert not meshcheck.check(u, P, P, tri, sh)["all_ccw"]
    r = meshcheck.check(u, P, P, m.tri[1:], m.shift[1:])   # a hole
    assert not r["every_edge_has_twin"] and not r["area_tiles_box"]
    b = inputs.bounded_grid(5, 5)                      # not periodic: boundary edges have no twin
    ub = np.rint(b.xy / b.Lx * P).astype(np.int64)
    assert not meshcheck.check(ub, P, P, b.tri, b.shift)["every_edge_has_twin"]


def test_quality_measures():
    m = inputs.periodic_grid(4)
    r = meshcheck.check(units(m), P, P, m.tri, m.shift, R_units=P / 4 / np.sqrt(2) * 1.0001, B=1 / np.sqrt(2) * 1.0001)
    # right isosceles triangles with legs h: circumradius h / sqrt 2, beta = 1 / sqrt 2, min angle 45 deg
    assert r["size_bound"] and r["quality_bound"]
    assert abs(r["min_angle_deg"] - 45.0) < 1e-6
