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


def test_filtered_predicates_equal_the_integer_definitions():
    """The vectorised Orient2D / InCircle2D (int64, and a double-precision filter with
    an error bound) give the signs of the plain Python-integer determinants: on random
    points at the generator's coordinate scale (2^30 per period), on exactly
    cocircular quadruples (integer points on x^2 + y^2 = 5^2 13^2 17^2 scaled up) and
    on quadruples one unit off a circle, where the double evaluation alone is unsure."""
    rng = np.random.default_rng(3)
    n = 20000
    pts = rng.integers(-(1 << 30), 1 << 30, size=(4, n, 2), dtype=np.int64)
    assert np.array_equal(meshcheck.orient_sign(*pts[:3]), meshcheck._orient_sign_exact(*pts[:3]))
    assert np.array_equal(meshcheck.incircle_sign(*pts), meshcheck._incircle_sign_exact(*pts))
    # integer points on one circle of radius 1105 (many Pythagorean representations)
    r = 1105
    circ = [(x, y) for x in range(-r, r + 1) for y in (int(round((r * r - x * x) ** 0.5)),)
            if x * x + y * y == r * r]
    circ = np.array(circ + [(x, -y) for x, y in circ], dtype=np.int64)
    idx = rng.integers(0, len(circ), size=(4, 4000))
    scale = 1 << 17                                    # coordinates up to ~2^27, lifts up to ~2^55
    off = rng.integers(-(1 << 28), 1 << 28, size=(1, 4000, 2), dtype=np.int64)
    q = circ[idx] * scale + off
    # order a, b, c counter-clockwise where they are not collinear
    o = meshcheck._orient_sign_exact(q[0], q[1], q[2])
    q[1, o < 0], q[2, o < 0] = q[2, o < 0].copy(), q[1, o < 0].copy()
    exact = meshcheck._incircle_sign_exact(*q)
    assert np.array_equal(meshcheck.incircle_sign(*q), exact)
    assert np.sum(exact == 0) > 100                    # cocircular cases were exercised
    q2 = q.copy()
    q2[3, :, 0] += 1                                   # one unit off the circle
    assert np.array_equal(meshcheck.incircle_sign(*q2), meshcheck._incircle_sign_exact(*q2))


def test_edge_map_finds_twins_and_flags_duplicates():
    m = inputs.jittered_grid(7, jitter=0.1, diagonal="delaunay", relabel_seed=4)
    nbr, nc = meshcheck.edge_map(m.tri, m.shift)
    assert np.all(nbr >= 0)
    t = np.arange(m.nt)[:, None].repeat(3, 1)
    k = np.arange(3)[None, :].repeat(m.nt, 0)
    assert np.array_equal(nbr[nbr, nc], t) and np.array_equal(nc[nbr, nc], k)   # twin of twin
    # a triangle listed twice: its edges no longer have a unique twin
    tri = np.concatenate([m.tri, m.tri[:1]])
    sh = np.concatenate([m.shift, m.shift[:1]])
    nbr2, _ = meshcheck.edge_map(tri, sh)
    assert np.all(nbr2[0] < 0) and np.all(nbr2[-1] < 0)
