"""Checks of a periodic Delaunay refinement mesh (Sec. 2.3-2.4), in exact
integer arithmetic (Python ints), independent of the CUDA generator.

TEST INFRASTRUCTURE ONLY: used by tests/ and bench.py's baseline legs.

Input: integer vertex coordinates (units), periods Px, Py, triangles [nt][3]
counter-clockwise, per-corner image shifts [nt][3][2] (in periods), and
optionally the generator's adjacency (neighbour triangle and corner).

The Delaunay triangulation of points in general position is unique, so a
triangulation that is valid (a closed orientable surface of genus one that
tiles the periodic box once) and in which every edge is locally Delaunay
(Sec. 2.3.2) is THE Delaunay triangulation of its vertex set.
"""
from __future__ import annotations

import numpy as np


def positions(xy_units, tri, shift, Px, Py):
    """(nt, 3, 2) int64 corner positions in each triangle's frame."""
    P = xy_units[tri].astype(np.int64)
    P[..., 0] += shift[..., 0].astype(np.int64) * Px
    P[..., 1] += shift[..., 1].astype(np.int64) * Py
    return P


def orient_sign(a, b, c):
    """Exact sign of Orient2D (Eq. eqOrient) for int64 arrays of points (..., 2).

    With every coordinate difference below 2^31 in magnitude both products are
    below 2^62 and their difference below 2^63, so int64 arithmetic is exact;
    otherwise the determinant is formed with Python integers."""
    a, b, c = (np.asarray(q, dtype=np.int64) for q in (a, b, c))
    if a.size == 0:
        return np.zeros(a.shape[:-1], int)
    acx, acy = a[..., 0] - c[..., 0], a[..., 1] - c[..., 1]
    bcx, bcy = b[..., 0] - c[..., 0], b[..., 1] - c[..., 1]
    lim = (1 << 31) - 1
    if max(int(np.abs(q).max()) for q in (acx, acy, bcx, bcy)) <= lim:
        d = acx * bcy - acy * bcx
        return np.sign(d).astype(int)
    return _orient_sign_exact(a, b, c)


def _orient_sign_exact(a, b, c):
    """Orient2D with Python integers (any magnitude)."""
    ax, ay = a[..., 0].astype(object), a[..., 1].astype(object)
    bx, by = b[..., 0].astype(object), b[..., 1].astype(object)
    cx, cy = c[..., 0].astype(object), c[..., 1].astype(object)
    d = (ax - cx) * (by - cy) - (ay - cy) * (bx - cx)
    return np.array([(x > 0) - (x < 0) for x in np.ravel(d)], dtype=int).reshape(np.shape(d))


def _incircle_sign_exact(a, b, c, d):
    """InCircle2D with Python integers (any magnitude)."""
    o = lambda q: (q[..., 0].astype(object), q[..., 1].astype(object))
    (ax, ay), (bx, by), (cx, cy), (dx, dy) = o(a), o(b), o(c), o(d)
    adx, ady, bdx, bdy, cdx, cdy = ax - dx, ay - dy, bx - dx, by - dy, cx - dx, cy - dy
    det = ((adx * adx + ady * ady) * (bdx * cdy - cdx * bdy) - (bdx * bdx + bdy * bdy) * (adx * cdy - cdx * ady)
           + (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady))
    return np.array([(x > 0) - (x < 0) for x in np.ravel(det)], dtype=int).reshape(np.shape(det))


def incircle_sign(a, b, c, d):
    """Exact sign of InCircle2D (Eq. eqInCircle); > 0: d inside the circle of CCW a, b, c.

    Filtered: the determinant is first evaluated in double precision from the
    exact integer differences (each below 2^53, so exactly representable); where
    its magnitude exceeds a bound on the rounding error of that evaluation the
    sign is certain, and only the remaining cases are formed with Python
    integers.  The bound: every product and sum of the evaluation below rounds
    with relative error at most eps = 2^-53, there are at most 6 roundings on
    any path to the final sum, so |error| <= 6 eps (1 + eps)^6 * permanent,
    where the permanent is the same expression with every term replaced by its
    magnitude; 8 eps * permanent is used."""
    a, b, c, d = (np.asarray(q, dtype=np.int64) for q in (a, b, c, d))
    if a.size == 0:
        return np.zeros(a.shape[:-1], int)
    diffs = [a[..., 0] - d[..., 0], a[..., 1] - d[..., 1], b[..., 0] - d[..., 0], b[..., 1] - d[..., 1],
             c[..., 0] - d[..., 0], c[..., 1] - d[..., 1]]
    if max(int(np.abs(q).max()) for q in diffs) >= (1 << 53):
        return _incircle_sign_exact(a, b, c, d)
    adx, ady, bdx, bdy, cdx, cdy = (q.astype(np.float64) for q in diffs)
    alift = adx * adx + ady * ady
    blift = bdx * bdx + bdy * bdy
    clift = cdx * cdx + cdy * cdy
    bc = bdx * cdy - cdx * bdy
    ca = cdx * ady - adx * cdy
    ab = adx * bdy - bdx * ady
    det = alift * bc + blift * ca + clift * ab
    perm = (alift * (np.abs(bdx * cdy) + np.abs(cdx * bdy)) + blift * (np.abs(cdx * ady) + np.abs(adx * cdy)) +
            clift * (np.abs(adx * bdy) + np.abs(bdx * ady)))
    bound = 8.0 * 2.0 ** -53 * perm
    out = np.sign(det).astype(int)
    unsure = ~(np.abs(det) > bound)
    if np.any(unsure):
        out[unsure] = _incircle_sign_exact(a[unsure], b[unsure], c[unsure], d[unsure])
    return out


def edge_map(tri, shift):
    """Twin of every (triangle, corner) edge, found from vertex ids and relative shifts
    (not from any stored adjacency): returns (nbr, nbr_corner), -1 where unmatched
    or where a directed edge occurs more than once (an invalid triangulation).

    The directed edge of corner k of t runs from corner k+1 to corner k+2 with the
    relative image shift of its end; its twin is the directed edge with the ends
    swapped and the opposite relative shift.  Keys are packed into int64 and
    matched by sorting."""
    tri = np.asarray(tri, dtype=np.int64)
    shift = np.asarray(shift, dtype=np.int64)
    nt = len(tri)
    nv = int(tri.max()) + 1 if nt else 0
    rel_span = int(np.abs(shift).max()) * 2 + 1 if nt else 1
    R = 2 * rel_span + 1                      # relative shifts lie in [-rel_span, rel_span]
    if nt and nv * nv * R * R >= (1 << 62):
        raise ValueError("mesh too large for packed edge keys")
    t_idx = np.repeat(np.arange(nt, dtype=np.int64), 3)
    k_idx = np.tile(np.arange(3, dtype=np.int64), nt)
    a_c, b_c = (k_idx + 1) % 3, (k_idx + 2) % 3
    va, vb = tri[t_idx, a_c], tri[t_idx, b_c]
    rx = shift[t_idx, b_c, 0] - shift[t_idx, a_c, 0]
    ry = shift[t_idx, b_c, 1] - shift[t_idx, a_c, 1]

    def pack(u, v, x, y):
        return ((u * nv + v) * R + (x + rel_span)) * R + (y + rel_span)

    key = pack(va, vb, rx, ry)
    twin = pack(vb, va, -rx, -ry)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    dup = np.zeros(len(ks), dtype=bool)
    if len(ks) > 1:
        same = ks[1:] == ks[:-1]
        dup[1:] |= same
        dup[:-1] |= same
    pos = np.searchsorted(ks, twin)
    pos_c = np.minimum(pos, max(len(ks) - 1, 0))
    hit = (pos < len(ks)) & (ks[pos_c] == twin) & ~dup[pos_c]
    src = order[pos_c]
    nbr = np.where(hit, t_idx[src], -1).reshape(nt, 3)
    nc = np.where(hit, k_idx[src], -1).reshape(nt, 3)
    # a directed edge that occurs twice makes its own entries unmatched too
    own_dup = np.zeros(3 * nt, dtype=bool)
    own_dup[order] = dup
    nbr[own_dup.reshape(nt, 3)] = -1
    nc[own_dup.reshape(nt, 3)] = -1
    return nbr, nc


def _twice_area_sum(P):
    """Exact sum over triangles of twice the signed area (Python integer)."""
    e1 = P[:, 1] - P[:, 0]
    e2 = P[:, 2] - P[:, 0]
    lim = (1 << 31) - 1
    if len(P) == 0:
        return 0
    if max(int(np.abs(e1).max()), int(np.abs(e2).max())) > lim:
        return sum(int(x) * int(w) - int(y) * int(z) for x, w, y, z in
                   zip(e1[:, 0], e2[:, 1], e2[:, 0], e1[:, 1]))
    d = e1[:, 0] * e2[:, 1] - e2[:, 0] * e1[:, 1]          # |d| < 2^63, exact in int64
    # sum the low and high 32-bit halves separately so no partial sum can overflow
    lo = d & np.int64(0xFFFFFFFF)
    hi = d >> np.int64(32)
    return int(lo.sum(dtype=np.int64)) + (int(hi.sum(dtype=np.int64)) << 32)


def check(xy_units, Px, Py, tri, shift, R_units=None, B=None, adjacency=None):
    """Returns a dict of the checks' results (all True for a valid refined mesh)."""
    xy_units = np.asarray(xy_units, dtype=np.int64)
    tri = np.asarray(tri, dtype=np.int64)
    shift = np.asarray(shift, dtype=np.int64)
    nv, nt = len(xy_units), len(tri)
    out = {}
    out["coords_in_box"] = bool(np.all((xy_units[:, 0] >= 0) & (xy_units[:, 0] < Px) &
                                       (xy_units[:, 1] >= 0) & (xy_units[:, 1] < Py)))
    P = positions(xy_units, tri, shift, Px, Py)
    o = orient_sign(P[:, 0], P[:, 1], P[:, 2])
    out["all_ccw"] = bool(np.all(o > 0))
    # twice the areas tile twice the box exactly
    out["area_tiles_box"] = _twice_area_sum(P) == 2 * Px * Py
    nbr, nc = edge_map(tri, shift)
    out["every_edge_has_twin"] = bool(np.all(nbr >= 0))
    out["euler_torus"] = nv - (3 * nt) // 2 + nt == 0 and (3 * nt) % 2 == 0
    if adjacency is not None:
        tn, tc = (np.asarray(a, dtype=np.int64) for a in adjacency)
        out["adjacency_matches"] = bool(np.array_equal(tn, nbr) and np.array_equal(tc, nc))
    # local Delaunay property of every edge: far vertex of the twin outside t's circumcircle
    if out["every_edge_has_twin"]:
        t_idx, k_idx = np.nonzero(nbr >= 0)
        n_idx, j_idx = nbr[t_idx, k_idx], nc[t_idx, k_idx]
        a_c = (k_idx + 1) % 3
        # frame offset from the shared vertex (corner k+1 of t is corner j+2 of n)
        off = shift[n_idx, (j_idx + 2) % 3] - shift[t_idx, a_c]
        d = P[n_idx, j_idx] - off * np.array([Px, Py])
        s = incircle_sign(P[t_idx, 0], P[t_idx, 1], P[t_idx, 2], d)
        out["delaunay"] = bool(np.all(s <= 0))
        out["cocircular_edges"] = int(np.sum(s == 0))
    if R_units is not None or B is not None:
        e = np.stack([P[:, (k + 2) % 3] - P[:, (k + 1) % 3] for k in range(3)], axis=1).astype(float)
        l2 = (e ** 2).sum(axis=2)
        D = 2.0 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) -
                   (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1])).astype(float)
        r = np.sqrt(l2.prod(axis=1)) / D
        beta = r / np.sqrt(l2.min(axis=1))
        out["max_circumradius"] = float(r.max())
        out["max_beta"] = float(beta.max())
        out["min_angle_deg"] = float(np.degrees(np.arcsin(1.0 / (2.0 * beta.max()))))
        if R_units is not None:
            out["size_bound"] = bool(r.max() <= R_units * (1 + 1e-9))
        if B is not None:
            out["quality_bound"] = bool(beta.max() <= B * (1 + 1e-9))
    return out
