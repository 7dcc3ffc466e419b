"""Seeded synthetic inputs: periodic triangulations and initial states.

This module only builds inputs (meshes and conserved states).  It contains
none of the residual-distribution arithmetic, and both the CUDA library and the
CPU oracle are fed from it, so that the two sides see bit-identical inputs.

Meshes
------
``periodic_grid`` builds the structured triangulation of Sec. 2.1 (Eq. eqCart):
vertex (i, j) at (i Lx/Nx, j Ly/Ny), each cell a=(i,j), b=(i+1,j), c=(i+1,j+1),
d=(i,j+1) split along the diagonal a-c into the counter-clockwise triangles
(a,b,c) and (a,c,d).  Indices wrap periodically; a corner reached across the
periodic boundary carries an image shift (in periods) so that every triangle
has its true geometry (periodic boundaries "handled by the mesh", Sec. 3.5).
Every vertex has valence 6.  ``relabel_seed`` applies a seeded random
permutation to vertex and triangle labels, standing in for the unstructured
Delaunay meshes of Sec. 4.1 (whose locality has to be restored by reordering).

States
------
W is returned component-major, shape (4, nv): rho, rho u, rho v, e
(e = rho |v|^2 / 2 + p / (gamma - 1), Sec. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = 1.4


@dataclass
class Mesh:
    xy: np.ndarray        # (nv, 2) float64
    tri: np.ndarray       # (nt, 3) int32, counter-clockwise
    shift: np.ndarray     # (nt, 3, 2) int8, periodic image of each corner
    Lx: float
    Ly: float
    orig_vertex: np.ndarray  # (nv,) int64: structured id j*Nx+i of each vertex
    Nx: int = 0
    Ny: int = 0
    # boundary conditions (Sec. 3.5); None on fully periodic meshes
    ghost: np.ndarray | None = None   # (nv,) uint8: 1 = state held at its initial value
    walls: np.ndarray | None = None   # (n_wall, 2) int32: (triangle, corner) of the wall edge
    alpha: float = 0.75               # wall-correction split

    @property
    def nv(self) -> int:
        return int(self.xy.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tri.shape[0])


def periodic_grid(Nx: int, Ny: int | None = None, Lx: float = 1.0, Ly: float | None = None,
                  relabel_seed: int | None = None) -> Mesh:
    """Regular periodic triangulation with Nx*Ny vertices and 2*Nx*Ny triangles."""
    if Ny is None:
        Ny = Nx
    if Ly is None:
        Ly = Lx * Ny / Nx
    if Nx < 2 or Ny < 2:
        raise ValueError("periodic_grid needs at least 2 vertices per side")
    i = np.arange(Nx, dtype=np.int64)
    j = np.arange(Ny, dtype=np.int64)
    jj, ii = np.meshgrid(j, i, indexing="ij")           # (Ny, Nx)
    vid = (jj * Nx + ii).ravel()
    xy = np.stack([ii.ravel() * (Lx / Nx), jj.ravel() * (Ly / Ny)], axis=1).astype(np.float64)

    ip = (ii + 1) % Nx
    jp = (jj + 1) % Ny
    sx = (ii + 1 == Nx).astype(np.int8)
    sy = (jj + 1 == Ny).astype(np.int8)
    a = jj * Nx + ii
    b = jj * Nx + ip
    c = jp * Nx + ip
    d = jp * Nx + ii
    z = np.zeros_like(sx)
    t1 = np.stack([a, b, c], axis=-1).reshape(-1, 3)
    t2 = np.stack([a, c, d], axis=-1).reshape(-1, 3)
    s1 = np.stack([np.stack([z, z], -1), np.stack([sx, z], -1), np.stack([sx, sy], -1)], axis=-2).reshape(-1, 3, 2)
    s2 = np.stack([np.stack([z, z], -1), np.stack([sx, sy], -1), np.stack([z, sy], -1)], axis=-2).reshape(-1, 3, 2)
    tri = np.empty((2 * Nx * Ny, 3), dtype=np.int64)
    shift = np.empty((2 * Nx * Ny, 3, 2), dtype=np.int8)
    tri[0::2], tri[1::2] = t1, t2
    shift[0::2], shift[1::2] = s1, s2
    orig = vid.copy()

    mesh = Mesh(xy=np.ascontiguousarray(xy), tri=np.ascontiguousarray(tri.astype(np.int32)),
                shift=np.ascontiguousarray(shift), Lx=float(Lx), Ly=float(Ly),
                orig_vertex=orig, Nx=Nx, Ny=Ny)
    return relabel(mesh, relabel_seed) if relabel_seed is not None else mesh


def relabel(mesh: Mesh, seed: int) -> Mesh:
    """Seeded random permutation of vertex and triangle labels and a rotation of
    each triangle's corner order (orientation kept); boundary data follow."""
    rng = np.random.default_rng(seed)
    n = mesh.nv
    vperm = rng.permutation(n)          # new label of old vertex
    inv = np.empty_like(vperm)
    inv[vperm] = np.arange(n)
    xy = mesh.xy[inv]
    orig = mesh.orig_vertex[inv]
    tri = vperm[mesh.tri.astype(np.int64)]
    tperm = rng.permutation(tri.shape[0])   # old triangle of each new slot
    tri = tri[tperm]
    shift = mesh.shift[tperm]
    rot = rng.integers(0, 3, size=tri.shape[0])
    idx = (np.arange(3)[None, :] + rot[:, None]) % 3
    tri = np.take_along_axis(tri, idx, axis=1)
    shift = np.take_along_axis(shift, idx[:, :, None], axis=1)
    ghost = None if mesh.ghost is None else np.ascontiguousarray(mesh.ghost[inv])
    walls = None
    if mesh.walls is not None:
        tnew = np.empty_like(tperm)
        tnew[tperm] = np.arange(tperm.size)
        t_new = tnew[mesh.walls[:, 0]]
        c_new = (mesh.walls[:, 1] - rot[t_new]) % 3     # new corner k holds old corner (k + rot) % 3
        walls = np.ascontiguousarray(np.stack([t_new, c_new], axis=1).astype(np.int32))
    return Mesh(xy=np.ascontiguousarray(xy), tri=np.ascontiguousarray(tri.astype(np.int32)),
                shift=np.ascontiguousarray(shift), Lx=mesh.Lx, Ly=mesh.Ly, orig_vertex=orig,
                Nx=mesh.Nx, Ny=mesh.Ny, ghost=ghost, walls=walls, alpha=mesh.alpha)


def _incircle(ax, ay, bx, by, cx, cy, dx, dy):
    """> 0 when d lies inside the circle through the counter-clockwise a, b, c."""
    adx, ady = ax - dx, ay - dy
    bdx, bdy = bx - dx, by - dy
    cdx, cdy = cx - dx, cy - dy
    return ((adx * adx + ady * ady) * (bdx * cdy - cdx * bdy)
            - (bdx * bdx + bdy * bdy) * (adx * cdy - cdx * ady)
            + (cdx * cdx + cdy * cdy) * (adx * bdy - bdx * ady))


def jittered_grid(Nx: int, Ny: int | None = None, Lx: float = 1.0, Ly: float | None = None,
                  jitter: float = 0.2, seed: int = 6, diagonal: str = "delaunay",
                  relabel_seed: int | None = None) -> Mesh:
    """Unstructured periodic triangulation: the grid of ``periodic_grid`` with every
    vertex moved by a seeded offset of at most ``jitter`` cell widths per axis, and
    each (convex) cell split along the diagonal that the empty-circumcircle (Delaunay)
    test picks (``diagonal="delaunay"``) or along a seeded random one ("random").

    Vertex valences then range from 4 to 8 instead of being 6 everywhere, the edge
    lengths and angles vary from triangle to triangle, and the vertex and
    triangle labels can be scrambled with ``relabel_seed`` -- a stand-in for the
    unstructured Delaunay meshes of Sec. 4.1 that keeps the vertex count exact.
    Offsets come from SplitMix64(seed xor (2 id)) and SplitMix64(seed xor (2 id + 1))
    of the structured vertex id; stored coordinates are wrapped into [0, L).
    jitter <= 0.2 keeps every cell strictly convex, so both diagonals are valid.
    """
    if Ny is None:
        Ny = Nx
    if Ly is None:
        Ly = Lx * Ny / Nx
    if Nx < 3 or Ny < 3:
        raise ValueError("jittered_grid needs at least 3 vertices per side")
    if not (0.0 <= jitter <= 0.2):
        raise ValueError("jitter must lie in [0, 0.2]")
    if diagonal not in ("delaunay", "random"):
        raise ValueError("diagonal must be 'delaunay' or 'random'")
    hx, hy = Lx / Nx, Ly / Ny
    i = np.arange(Nx, dtype=np.int64)
    j = np.arange(Ny, dtype=np.int64)
    jj, ii = np.meshgrid(j, i, indexing="ij")           # (Ny, Nx)
    vid = (jj * Nx + ii).ravel()
    dx = jitter * (2.0 * uniform01(seed, 2 * vid) - 1.0)
    dy = jitter * (2.0 * uniform01(seed, 2 * vid + 1) - 1.0)
    bx = (ii.ravel() + dx) * hx                        # home positions, may leave [0, L)
    by = (jj.ravel() + dy) * hy
    kx = np.floor(bx / Lx).astype(np.int64)            # home image (periods), -1 or 0
    ky = np.floor(by / Ly).astype(np.int64)
    xy = np.stack([bx - kx * Lx, by - ky * Ly], axis=1)

    def corner(ci, cj):
        """vertex id and periodic shift of grid point (ci, cj), 0 <= ci <= Nx, 0 <= cj <= Ny."""
        v = (cj % Ny) * Nx + (ci % Nx)
        return v, kx[v] + ci // Nx, ky[v] + cj // Ny

    ci, cj = ii.ravel(), jj.ravel()
    a, b, c, d = corner(ci, cj), corner(ci + 1, cj), corner(ci + 1, cj + 1), corner(ci, cj + 1)
    pos = [(xy[q[0], 0] + q[1] * Lx, xy[q[0], 1] + q[2] * Ly) for q in (a, b, c, d)]
    if diagonal == "delaunay":
        # diagonal a-c unless d falls inside the circumcircle of (a, b, c)
        use_bd = _incircle(*pos[0], *pos[1], *pos[2], *pos[3]) > 0.0
    else:
        use_bd = uniform01(seed + 1, vid) < 0.5
    def pick(q_bd, q_ac):
        return tuple(np.where(use_bd, x, y) for x, y in zip(q_bd, q_ac))

    # diagonal a-c: (a, b, c) and (a, c, d);  diagonal b-d: (a, b, d) and (b, c, d)
    first = (a, b, pick(d, c))
    second = (pick(b, a), c, d)
    n = Nx * Ny
    tri = np.empty((2 * n, 3), dtype=np.int64)
    shift = np.empty((2 * n, 3, 2), dtype=np.int64)
    for slot, corners in ((0, first), (1, second)):
        for k, q in enumerate(corners):
            tri[slot::2, k] = q[0]
            shift[slot::2, k, 0] = q[1]
            shift[slot::2, k, 1] = q[2]
    # every triangle counter-clockwise with positive area
    P = xy[tri] + shift * np.array([Lx, Ly])
    area2 = ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
             - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))
    if not np.all(area2 > 0.0):
        raise AssertionError("jittered_grid produced a non-positive triangle")
    mesh = Mesh(xy=np.ascontiguousarray(xy), tri=np.ascontiguousarray(tri.astype(np.int32)),
                shift=np.ascontiguousarray(shift.astype(np.int8)), Lx=float(Lx), Ly=float(Ly),
                orig_vertex=vid.copy(), Nx=Nx, Ny=Ny)
    return relabel(mesh, relabel_seed) if relabel_seed is not None else mesh


def bounded_grid(Nx: int, Ny: int | None = None, Lx: float = 1.0, Ly: float | None = None,
                 periodic_x: bool = False, periodic_y: bool = False, bc_x: str = "wall", bc_y: str = "wall",
                 relabel_seed: int | None = None) -> Mesh:
    """Structured triangulation of [0, Lx] x [0, Ly] with Nx x Ny cells (split along
    the diagonal a-c as in ``periodic_grid``), periodic in the directions asked for
    and bounded in the others.  A bounded side is a reflecting wall ("wall": its
    edges are listed as (triangle, corner) pairs, Sec. 3.5) or a non-reflecting /
    inflow side ("ghost": its vertices are held at their initial state)."""
    if Ny is None:
        Ny = Nx
    if Ly is None:
        Ly = Lx * Ny / Nx
    for bc in (bc_x, bc_y):
        if bc not in ("wall", "ghost"):
            raise ValueError("bc must be 'wall' or 'ghost'")
    nxv = Nx if periodic_x else Nx + 1
    nyv = Ny if periodic_y else Ny + 1
    hx, hy = Lx / Nx, Ly / Ny
    jj, ii = np.meshgrid(np.arange(nyv), np.arange(nxv), indexing="ij")
    xy = np.stack([ii.ravel() * hx, jj.ravel() * hy], axis=1).astype(np.float64)
    ci, cj = np.meshgrid(np.arange(Nx), np.arange(Ny), indexing="xy")
    ci, cj = ci.ravel(), cj.ravel()

    def vid(i, j):
        return (j % nyv) * nxv + (i % nxv)

    def sh(i, j):
        sx = (i // nxv) if periodic_x else np.zeros_like(i)
        sy = (j // nyv) if periodic_y else np.zeros_like(j)
        return np.stack([sx, sy], axis=-1)

    A, B, C, D = (ci, cj), (ci + 1, cj), (ci + 1, cj + 1), (ci, cj + 1)
    n = Nx * Ny
    tri = np.empty((2 * n, 3), dtype=np.int64)
    shift = np.empty((2 * n, 3, 2), dtype=np.int64)
    for slot, corners in ((0, (A, B, C)), (1, (A, C, D))):
        for k, (i, j) in enumerate(corners):
            tri[slot::2, k] = vid(i, j)
            shift[slot::2, k] = sh(i, j)
    cell = cj * Nx + ci
    ghost = np.zeros(nxv * nyv, dtype=np.uint8)
    walls = []
    if not periodic_y:
        if bc_y == "ghost":
            ghost[(jj.ravel() == 0) | (jj.ravel() == Ny)] = 1
        else:
            bot, top = cell[cj == 0], cell[cj == Ny - 1]
            walls += [np.stack([2 * bot, np.full_like(bot, 2)], 1), np.stack([2 * top + 1, np.zeros_like(top)], 1)]
    if not periodic_x:
        if bc_x == "ghost":
            ghost[(ii.ravel() == 0) | (ii.ravel() == Nx)] = 1
        else:
            left, right = cell[ci == 0], cell[ci == Nx - 1]
            walls += [np.stack([2 * left + 1, np.ones_like(left)], 1), np.stack([2 * right, np.zeros_like(right)], 1)]
    mesh = Mesh(xy=np.ascontiguousarray(xy), tri=np.ascontiguousarray(tri.astype(np.int32)),
                shift=np.ascontiguousarray(shift.astype(np.int8)), Lx=float(Lx), Ly=float(Ly),
                orig_vertex=(jj * nxv + ii).ravel().astype(np.int64), Nx=nxv, Ny=nyv,
                ghost=ghost if ghost.any() else None,
                walls=np.ascontiguousarray(np.concatenate(walls).astype(np.int32)) if walls else None)
    return relabel(mesh, relabel_seed) if relabel_seed is not None else mesh


def noh_quadrant(N: int, relabel_seed: int | None = None) -> Mesh:
    """The quadrant [0, 1]^2 of the Noh problem (Sec. 5.2): reflecting walls on the
    symmetry lines x = 0 and y = 0, ghost vertices (held at the initial inflow
    state) on x = 1 and y = 1; N x N cells split along a-c."""
    m = bounded_grid(N, N, bc_x="wall", bc_y="wall")
    P = m.xy[m.tri] + m.shift * np.array([m.Lx, m.Ly])
    keep = [(t, c) for t, c in m.walls
            if (P[t, (c + 1) % 3, 0] == 0.0 and P[t, (c + 2) % 3, 0] == 0.0)
            or (P[t, (c + 1) % 3, 1] == 0.0 and P[t, (c + 2) % 3, 1] == 0.0)]
    m.walls = np.ascontiguousarray(np.array(keep, dtype=np.int32))
    x, y = m.xy[:, 0], m.xy[:, 1]
    m.ghost = ((x >= m.Lx * (1 - 1e-12)) | (y >= m.Ly * (1 - 1e-12))).astype(np.uint8)
    return relabel(m, relabel_seed) if relabel_seed is not None else m


# ---------------------------------------------------------------------------
# conserved state from primitives
# ---------------------------------------------------------------------------
def conserved(rho, u, v, p, gamma: float = GAMMA) -> np.ndarray:
    rho = np.asarray(rho, dtype=np.float64)
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), rho.shape)
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), rho.shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape)
    e = 0.5 * rho * (u * u + v * v) + p / (gamma - 1.0)
    return np.ascontiguousarray(np.stack([rho, rho * u, rho * v, e]))


def primitives(W: np.ndarray, gamma: float = GAMMA):
    rho = W[0]
    u = W[1] / rho
    v = W[2] / rho
    p = (gamma - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v))
    return rho, u, v, p


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea & Flood 2014) on uint64 counters."""
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """U[0,1) from the top 53 bits of SplitMix64(seed xor counter)."""
    z = splitmix64(np.uint64(seed) ^ np.asarray(counters, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ---------------------------------------------------------------------------
# initial states
# ---------------------------------------------------------------------------
def uniform_state(mesh: Mesh, rho=1.0, u=0.0, v=0.0, p=1.0, gamma=GAMMA) -> np.ndarray:
    one = np.ones(mesh.nv)
    return conserved(rho * one, u * one, v * one, p * one, gamma)


def noh_state(mesh: Mesh, p0: float = 1e-6, gamma: float = 5.0 / 3.0) -> np.ndarray:
    """Noh's implosion: rho = 1, velocity -r/|r| of unit magnitude towards the origin
    (zero at the origin), pressure p0; exact solution for gamma = 5/3 in 2-D: a shock
    at r = t/3 with rho = 16 behind it and rho = 1 + t/r ahead of it."""
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    r = np.hypot(x, y)
    rs = np.where(r > 0, r, 1.0)
    u = np.where(r > 0, -x / rs, 0.0)
    v = np.where(r > 0, -y / rs, 0.0)
    return conserved(np.ones(mesh.nv), u, v, np.full(mesh.nv, p0), gamma)


def vortex_primitives(x, y, t=0.0, beta=5.0, scale=10.0, u0=1.0, v0=1.0, Lx=1.0, Ly=1.0,
                      gamma=GAMMA, xc=0.5, yc=0.5):
    """Isentropic vortex of Sec. 5.2.1 translated by (u0, v0) t on a periodic box.

    The paper's setup (box [0,10]^2, beta=5, centre (5,5), p_inf=rho_inf=K=1) is
    mapped onto the box [0,Lx)x[0,Ly) by lengths/scale; velocities are unchanged.
    The nearest periodic image of the centre is used.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    cx = xc + u0 * t
    cy = yc + v0 * t
    dx = (x - cx) - Lx * np.round((x - cx) / Lx)
    dy = (y - cy) - Ly * np.round((y - cy) / Ly)
    dx = dx * scale
    dy = dy * scale
    r2 = dx * dx + dy * dy
    omega = beta * np.exp((1.0 - r2) / 2.0) / (2.0 * np.pi)
    T = 1.0 - (gamma - 1.0) / gamma * beta ** 2 / (8.0 * np.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    u = u0 - omega * dy
    v = v0 + omega * dx
    return rho, u, v, p


def vortex_state(mesh: Mesh, t=0.0, beta=5.0, u0=1.0, v0=1.0, gamma=GAMMA, scale=None) -> np.ndarray:
    if scale is None:
        scale = 10.0 / mesh.Lx
    rho, u, v, p = vortex_primitives(mesh.xy[:, 0], mesh.xy[:, 1], t=t, beta=beta, scale=scale,
                                     u0=u0, v0=v0, Lx=mesh.Lx, Ly=mesh.Ly, gamma=gamma,
                                     xc=0.5 * mesh.Lx, yc=0.5 * mesh.Ly)
    return conserved(rho, u, v, p, gamma)


def sod_like_state(mesh: Mesh, amp=0.01, gamma=GAMMA) -> np.ndarray:
    """Left (rho=1, p=1) where x < 0.5 + amp sin(2 pi y), right (0.125, 0.1) elsewhere; at rest."""
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    left = x < 0.5 + amp * np.sin(2.0 * np.pi * y)
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    return conserved(rho, 0.0, 0.0, p, gamma)


def sod_strip_state(mesh: Mesh, gamma=GAMMA) -> np.ndarray:
    """Sod tube on a periodic strip x in [0, 2): left state for x < 0.5 or x >= 1.5."""
    x = mesh.xy[:, 0]
    left = (x < 0.5) | (x >= 1.5)
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    return conserved(rho, 0.0, 0.0, p, gamma)


def khi_state(mesh: Mesh, seed=1, amp=0.01, gamma=GAMMA) -> np.ndarray:
    """Shear layer: rho=2, u=+0.5 for |y-0.5|<0.25; rho=1, u=-0.5 elsewhere; p=2.5;
    v = amp (2U-1), U from SplitMix64(seed xor structured vertex id)."""
    y = mesh.xy[:, 1]
    inner = np.abs(y - 0.5) < 0.25
    rho = np.where(inner, 2.0, 1.0)
    u = np.where(inner, 0.5, -0.5)
    U = uniform01(seed, mesh.orig_vertex)
    v = amp * (2.0 * U - 1.0)
    return conserved(rho, u, v, 2.5, gamma)


def _smooth_step(t):
    """g(t) = f(t) / (f(t) + f(1 - t)) with f(t) = exp(-1/t) for t > 0, else 0 (Sec. 5.3):
    a C-infinity transition from 0 (t <= 0) to 1 (t >= 1)."""
    t = np.asarray(t, dtype=np.float64)

    def f(z):
        out = np.zeros_like(z)
        pos = z > 0
        out[pos] = np.exp(-1.0 / z[pos])
        return out

    a, b = f(t), f(1.0 - t)
    return a / (a + b)


def khi_smooth_profiles(y, d=0.25, U0=0.5, rhoL=1.0, rhoH=2.0):
    """Smoothed shear layer of Sec. 5.3: u_0(y) and rho_0(y) go from the outer values
    (-U0, rhoL) to the inner ones (+U0, rhoH) over a width d around y = 1/4 and 3/4."""
    y = np.asarray(y, dtype=np.float64)
    G = _smooth_step(0.5 + (y - 0.25) / d) * _smooth_step(0.5 - (y - 0.75) / d)
    return 2.0 * U0 * G - U0, (rhoH - rhoL) * G + rhoL


def khi_linear_mode(kx=2.0 * np.pi, d=0.25, U0=0.5, rhoL=1.0, rhoH=2.0, p0=2.5, gamma=GAMMA,
                    n=128, closure="energy"):
    """Fastest-growing linear mode of the smoothed shear layer on the periodic unit box.

    Perturbations q(y) exp(i kx x + sigma t) of the Euler equations linearised about
    (rho_0(y), u_0(y), v = 0, p_0) are expanded in n Fourier modes in y (periodic
    collocation, spectral derivative), which turns App. C's eigenproblem into a
    dense n-block matrix eigenproblem.  ``closure`` picks the pressure perturbation:

    * "energy": p_1 from the linearised energy equation,
      d_t p_1 + u_0 d_x p_1 + gamma p_0 div v_1 = 0 (the Euler equations' own);
    * "adiabatic": p_1 = c_0(y)^2 rho_1, the closure App. C states.  With rho_0
      varying and p_0 constant the background entropy varies, so the two differ.

    Returns (sigma, q) with sigma the eigenvalue of largest real part (growth rate
    Re sigma) and q the eigenvector on y_j = j / n, rows (rho_1, u_1, v_1, p_1),
    scaled so that the v_1 entry of largest modulus is real and equal to 1.
    """
    y = np.arange(n) / n
    u0, r0 = khi_smooth_profiles(y, d, U0, rhoL, rhoH)
    k = 2.0 * np.pi * np.fft.fftfreq(n, 1.0 / n)
    if n % 2 == 0:
        k[n // 2] = 0.0                      # odd derivative of the Nyquist mode
    F = np.fft.fft(np.eye(n), axis=0)
    D = np.real(np.fft.ifft(1j * k[:, None] * F, axis=0))
    du0 = D @ u0
    I, Z = np.eye(n), np.zeros((n, n))
    U, R, Ri = np.diag(u0), np.diag(r0), np.diag(1.0 / r0)
    ik = 1j * kx
    if closure == "energy":
        M = np.block([[-ik * U, -ik * R, -D @ R, Z],
                      [Z, -ik * U, -np.diag(du0), -ik * Ri],
                      [Z, Z, -ik * U, -Ri @ D],
                      [Z, -gamma * p0 * ik * I, -gamma * p0 * D, -ik * U]])
    elif closure == "adiabatic":
        C2 = np.diag(gamma * p0 / r0)
        M = np.block([[-ik * U, -ik * R, -D @ R],
                      [-ik * Ri @ C2, -ik * U, -np.diag(du0)],
                      [-Ri @ D @ C2, Z, -ik * U]])
    else:
        raise ValueError("closure must be 'energy' or 'adiabatic'")
    ev, vec = np.linalg.eig(M)
    i = int(np.argmax(ev.real))
    q = vec[:, i].reshape(-1, n)
    if closure == "adiabatic":
        q = np.vstack([q, (gamma * p0 / r0) * q[0]])
    j = int(np.argmax(np.abs(q[2])))
    q = q / q[2, j]
    return complex(ev[i]), q


def khi_smooth_state(mesh: Mesh, amp=1e-3, kx=2.0 * np.pi, d=0.25, U0=0.5, rhoL=1.0, rhoH=2.0,
                     p0=2.5, gamma=GAMMA, n=128):
    """Smoothed KHI of Sec. 5.3 seeded with its fastest-growing linear mode
    (``khi_linear_mode``, energy closure) at vertical-velocity amplitude ``amp``:
    q(x, y) = background(y) + amp Re[q_hat(y) exp(i kx x)], q_hat interpolated to
    the vertex heights by its Fourier series."""
    _, q = khi_linear_mode(kx, d, U0, rhoL, rhoH, p0, gamma, n, "energy")
    c = np.fft.fft(q, axis=1) / n
    kk = np.fft.fftfreq(n, 1.0 / n)
    if n % 2 == 0:
        c[:, n // 2] = 0.0
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    yu, inv = np.unique(y, return_inverse=True)
    qy = (np.exp(2j * np.pi * np.outer(yu, kk)) @ c.T).T[:, inv]
    pert = amp * np.real(qy * np.exp(1j * kx * x))
    u0, r0 = khi_smooth_profiles(y, d, U0, rhoL, rhoH)
    return conserved(r0 + pert[0], u0 + pert[1], pert[2], p0 + pert[3], gamma)


def vertical_kinetic_energy(V, W):
    """E_v = sum_i V_i rho_i v_i^2 / 2, the diagnostic whose growth Sec. 5.3 tracks."""
    return float(np.sum(V * W[2] * W[2] / W[0]) * 0.5)


def smooth_density_state(mesh: Mesh, seed=3, amp=0.05, n_modes=16, kmax=4, gamma=GAMMA) -> np.ndarray:
    """rho = 1 + amp f / max|f|, f a sum of n_modes seeded Fourier modes with |k| <= kmax;
    p = 1, u = v = 1."""
    rng = np.random.default_rng(seed)
    ks = [(kx, ky) for kx in range(-kmax, kmax + 1) for ky in range(-kmax, kmax + 1)
          if 0 < kx * kx + ky * ky <= kmax * kmax]
    pick = rng.choice(len(ks), size=n_modes, replace=False)
    amps = rng.normal(size=n_modes)
    phases = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    x, y = mesh.xy[:, 0] / mesh.Lx, mesh.xy[:, 1] / mesh.Ly
    f = np.zeros(mesh.nv)
    for m, (a, ph) in enumerate(zip(amps, phases)):
        kx, ky = ks[pick[m]]
        f += a * np.cos(2.0 * np.pi * (kx * x + ky * y) + ph)
    rho = 1.0 + amp * f / np.max(np.abs(f))
    return conserved(rho, 1.0, 1.0, 1.0, gamma)


def sound_wave_state(mesh: Mesh, amp=1e-4, t=0.0, gamma=GAMMA) -> np.ndarray:
    """Right-moving linear sound wave in rho=1, v=0, c=1 (Sec. 5.1.1), wavelength Lx."""
    x = mesh.xy[:, 0]
    c = 1.0
    p0 = 1.0 / gamma
    d = amp * np.sin(2.0 * np.pi * (x - c * t) / mesh.Lx)
    return conserved(1.0 + d, c * d, 0.0, p0 + c * c * d, gamma)


def blast_state(mesh: Mesh, dim: int, gamma: float = 5.0 / 3.0, rho0: float = 1.0, p0: float = 1e-6,
                h: float | None = None) -> np.ndarray:
    """Strong blast waves (Secs. 5.1.3 and 5.2.3): gas at rest, rho0, p0, plus a
    Gaussian pressure pulse at the centre of the box.
    dim = 1 (planar, about the line x = Lx / 2):
        p1 = (gamma - 1) / (500 h sqrt(pi)) exp(-x^2 / (100 h^2)), total energy 1/50
        per unit length of the line;
    dim = 2 (cylindrical, about the centre point):
        p1 = (gamma - 1) (0.004 / h)^2 exp(-(x^2 + y^2) / (6.25 h^2)), total energy
        6.25 pi 0.004^2.
    h is the cell size (default: the x spacing of the mesh's vertex grid, Lx / Nx)."""
    if h is None:
        h = mesh.Lx / mesh.Nx
    x = mesh.xy[:, 0] - 0.5 * mesh.Lx
    y = mesh.xy[:, 1] - 0.5 * mesh.Ly
    if dim == 1:
        p1 = (gamma - 1.0) / (500.0 * h * np.sqrt(np.pi)) * np.exp(-x * x / (100.0 * h * h))
    elif dim == 2:
        p1 = (gamma - 1.0) * (0.004 / h) ** 2 * np.exp(-(x * x + y * y) / (6.25 * h * h))
    else:
        raise ValueError("dim must be 1 or 2")
    return conserved(np.full(mesh.nv, rho0), 0.0, 0.0, p0 + p1, gamma)


# four constant states of the two-dimensional Riemann problem (Sec. 5.2.4):
# (rho, u, v, p) in the quadrants x <= 0.8 / > 0.8 by y > 0.8 / <= 0.8
RIEMANN2D_STATES = {
    "UL": (0.5322581, 1.2060454, 0.0, 0.3),
    "UR": (1.5, 0.0, 0.0, 1.5),
    "LL": (0.1379928, 1.2060454, 1.2060454, 0.0290323),
    "LR": (0.5322581, 0.0, 1.2060454, 0.3),
}


def riemann2d_state(mesh: Mesh, gamma: float = GAMMA, xc: float = 0.8, yc: float = 0.8) -> np.ndarray:
    """Two-dimensional Riemann problem of Sec. 5.2.4 on [0, 1]^2: U1 for x <= 0.8 < y,
    U2 for x, y > 0.8, U3 for x, y <= 0.8, U4 for y <= 0.8 < x (primitive states)."""
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    q = np.empty((mesh.nv, 4))
    top, right = y > yc, x > xc
    for key, sel in (("UL", ~right & top), ("UR", right & top), ("LL", ~right & ~top), ("LR", right & ~top)):
        q[sel] = RIEMANN2D_STATES[key]
    return conserved(q[:, 0], q[:, 1], q[:, 2], q[:, 3], gamma)


def batch_workload(n_mesh=64, seed=2, smin=128, smax=1024, relabel_seed=None):
    """64 periodic meshes with sides ~ U{smin..smax}; each gets a vortex or shear state (50/50)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(smin, smax + 1, size=n_mesh)
    kinds = rng.integers(0, 2, size=n_mesh)
    out = []
    for m in range(n_mesh):
        mesh = periodic_grid(int(sides[m]), relabel_seed=relabel_seed)
        if kinds[m] == 0:
            W = vortex_state(mesh)
        else:
            W = khi_state(mesh, seed=seed * 1000 + m)
        out.append((mesh, W, "vortex" if kinds[m] == 0 else "shear"))
    return out
