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
    """Exact sign of Orient2D (Eq. eqOrient) for int64 arrays of points (..., 2)."""
    ax, ay = a[..., 0].astype(object), a[..., 1].astype(object)
    bx, by = b[..., 0].astype(object), b[..., 1].astype(object)
    cx, cy = c[..., 0].astype(object), c[..., 1].astype(object)
    d = (ax - cx) * (by - cy) - (ay - cy) * (bx - cx)
    return np.sign(d.astype(float)).astype(int) if d.size else np.zeros(0, int)


def incircle_sign(a, b, c, d):
    """Exact sign of InCircle2D (Eq. eqInCircle); > 0: d inside the circle of CCW a, b, c."""
    o = lambda q: (q[..., 0].astype(object), q[..., 1].astype(object))
    (ax, ay), (bx, by), (cx, cy), (dx, dy) = o(a), o(b), o(c), o(d)
    adx, ady, bdx, bdy, cdx, cdy = ax - dx, ay - dy, bx - dx, by - dy, cx - dx, cy - dy
    det = ((adx * adx + ady * ady) * (bdx * cdy - cdx * bdy) - (bdx * bdx + bdy * bdy) * (adx * cdy - cdx * ady)
           + (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady))
    return np.array([(x > 0) - (x < 0) for x in det], dtype=int)


def edge_map(tri, shift):
    """Twin of every (triangle, corner) edge, found from vertex ids and relative shifts
    (not from any stored adjacency): returns (nbr, nbr_corner), -1 where unmatched."""
    nt = len(tri)
    key = {}
    for t in range(nt):
        for k in range(3):
            a, b = (k + 1) % 3, (k + 2) % 3
            va, vb = int(tri[t, a]), int(tri[t, b])
            rel = (int(shift[t, b, 0]) - int(shift[t, a, 0]), int(shift[t, b, 1]) - int(shift[t, a, 1]))
            key[(va, vb, rel)] = (t, k)
    nbr = -np.ones((nt, 3), dtype=np.int64)
    nc = -np.ones((nt, 3), dtype=np.int64)
    for t in range(nt):
        for k in range(3):
            a, b = (k + 1) % 3, (k + 2) % 3
            va, vb = int(tri[t, a]), int(tri[t, b])
            rel = (int(shift[t, a, 0]) - int(shift[t, b, 0]), int(shift[t, a, 1]) - int(shift[t, b, 1]))
            hit = key.get((vb, va, rel))
            if hit is not None:
                nbr[t, k], nc[t, k] = hit
    return nbr, nc


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
    two_area = sum(int((P[t, 1, 0] - P[t, 0, 0]) * (P[t, 2, 1] - P[t, 0, 1]) - (P[t, 2, 0] - P[t, 0, 0]) * (P[t, 1, 1] - P[t, 0, 1]))
                   for t in range(nt))
    out["area_tiles_box"] = two_area == 2 * Px * Py
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
