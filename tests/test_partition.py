"""Vertex partition of the step (host plan, no GPU): the plan's invariants, and a
world-size-2 gloo run of the exchange logic (ghost states before each stage,
all-reduce min of dt) with a CPU stand-in for each rank's step, which must
equal the single-rank run bitwise.

The stand-in step computes each local triangle's shares with the oracle
(stage-1 shares and stage-2 total residuals of Sec. 3.3-3.4 on the part's
local mesh), gathers them per owned vertex in the plan's CSR order, takes the
CFL dt over the owned vertices (Sec. 3.2) and updates the owned states
(Eqs. eqRK1 / eqRK2): everything a rank does except run kernels, so a wrong
ghost list, send order or dt reduction changes the result."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1705_02028_gb300 import binding, inputs

GAMMA, CFL = 1.4, 0.8


def _mesh(kind):
    if kind == "grid":
        return inputs.periodic_grid(20, 17, Lx=1.0, Ly=17 / 20, relabel_seed=6)
    return inputs.jittered_grid(18, relabel_seed=6)


@pytest.mark.parametrize("kind", ["grid", "jittered"])
@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_plan_invariants(kind, P):
    mesh = _mesh(kind)
    plans = [binding.partition_plan(mesh, P, r) for r in range(P)]
    owned = np.concatenate([p["local_vertices"][:p["n_owned"]] for p in plans])
    assert np.array_equal(np.sort(owned), np.arange(mesh.nv))           # every vertex owned exactly once
    owner = np.empty(mesh.nv, np.int64)
    for r, p in enumerate(plans):
        owner[p["local_vertices"][:p["n_owned"]]] = r
    for r, p in enumerate(plans):
        lv, lt, n_own = p["local_vertices"], p["local_triangles"], p["n_owned"]
        # local triangles = exactly the triangles with an owned corner, ascending internal order
        has_owned = np.any(owner[mesh.tri] == r, axis=1)
        assert np.array_equal(np.sort(lt), np.flatnonzero(has_owned))
        # local corners name the same vertices as the caller's triangles
        assert np.array_equal(lv[p["local_corners"].T], mesh.tri[lt])
        # ghosts: the corners not owned, each once
        ghosts = lv[n_own:]
        assert len(set(ghosts.tolist())) == len(ghosts) and np.all(owner[ghosts] != r)
        assert set(ghosts.tolist()) == set(mesh.tri[lt].ravel().tolist()) - set(lv[:n_own].tolist())
        # the CSR lists every corner of each owned vertex, in ascending local triangle order
        for i in range(n_own):
            ent = p["csr_ent"][p["csr_ptr"][i]:p["csr_ptr"][i + 1]]
            assert np.all(np.diff(ent // 3) > 0)
            assert np.all(p["local_corners"][ent % 3, ent // 3] == i)
            assert len(ent) == int(np.sum(mesh.tri == lv[i]))
        # ghost slices by owner
        for q in range(P):
            sl = ghosts[p["recv_ptr"][q]:p["recv_ptr"][q + 1]]
            assert np.all(owner[sl] == q)
    # what r sends to q is exactly q's slice of ghosts owned by r, in q's order
    for r, p in enumerate(plans):
        for q, pq in enumerate(plans):
            sent = p["local_vertices"][p["send_idx"][p["send_ptr"][q]:p["send_ptr"][q + 1]]]
            ghosts_q = pq["local_vertices"][pq["n_owned"]:]
            want = ghosts_q[pq["recv_ptr"][r]:pq["recv_ptr"][r + 1]]
            assert np.array_equal(sent, want), (r, q)


# ---------------------------------------------------------------------------
# CPU stand-in of one rank's step
# ---------------------------------------------------------------------------
class Local:
    """A part's local mesh (its local vertices and triangles) for the oracle."""

    def __init__(self, mesh, plan):
        self.plan = plan
        self.nv = len(plan["local_vertices"])
        self.nt = plan["n_local_tri"]
        self.xy = mesh.xy[plan["local_vertices"]]
        self.tri = np.ascontiguousarray(plan["local_corners"].T)
        self.shift = mesh.shift[plan["local_triangles"]]
        self.Lx, self.Ly = mesh.Lx, mesh.Ly
        g = oracle.geometry(self)
        self.V = g["V"]
        self.lmax = g["lmax"]
        self.n_own = plan["n_owned"]
        ptr, ent = plan["csr_ptr"], plan["csr_ent"]
        deg = np.diff(ptr)
        self.maxdeg = int(deg.max()) if len(deg) else 0
        self.slots = [(np.flatnonzero(deg > k), ent[ptr[:-1][deg > k] + k]) for k in range(self.maxdeg)]

    def gather(self, per_corner):
        """Sum over each owned vertex's corners in CSR order; per_corner: (nt, 3, ...)."""
        flat = per_corner.reshape((3 * self.nt,) + per_corner.shape[2:])
        out = np.zeros((self.n_own,) + per_corner.shape[2:])
        for idx, e in self.slots:
            out[idx] = out[idx] + flat[(e // 3) * 3 + e % 3]
        return out


def _speed(W):
    rho, u, v, p = inputs.primitives(W)
    return np.hypot(u, v) + np.sqrt(GAMMA * p / rho)


def _stage1(loc, Wl):
    """Owned R1 and this part's min over owned vertices of 2 V / sigma."""
    sh = oracle.stage1_shares(loc, Wl, "B2")                      # (nt, 3, 4)
    s = _speed(Wl)
    cflT = loc.lmax * s[loc.tri].max(axis=1)
    R1 = loc.gather(sh)                                            # (n_own, 4)
    sig = loc.gather(np.repeat(cflT[:, None], 3, axis=1))
    return R1, float(np.min(2.0 * loc.V[:loc.n_own] / sig))


def _stage2(loc, Wn, Ws, dt):
    phi = oracle.stage2_terms(loc, Wn, Ws, dt, scheme="B2")["Phi"]
    return loc.gather(phi)


def _run_rank(mesh, plans, r, W0, steps, exchange, allmin):
    loc = Local(mesh, plans[r])
    lv = plans[r]["local_vertices"]
    Wl = np.ascontiguousarray(W0[:, lv])
    n = loc.n_own
    for _ in range(steps):
        exchange(Wl)
        R1, m = _stage1(loc, Wl)
        dt = CFL * allmin(m)
        Ws = Wl.copy()
        Ws[:, :n] = Wl[:, :n] - dt / loc.V[:n] * R1.T
        exchange(Ws)
        R2 = _stage2(loc, Wl, Ws, dt)
        Wl = Wl.copy()
        Wl[:, :n] = Ws[:, :n] - dt / loc.V[:n] * R2.T
    return Wl[:, :n]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, kind, steps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mesh = _mesh(kind)
    W0 = inputs.khi_state(mesh) if kind == "grid" else inputs.vortex_state(mesh)
    plans = [binding.partition_plan(mesh, ws, r) for r in range(ws)]
    p = plans[rank]
    n_own = p["n_owned"]

    def exchange(W):
        ops = []
        sendbufs = []
        for peer in range(ws):
            if peer == rank:
                continue
            a, b = p["send_ptr"][peer], p["send_ptr"][peer + 1]
            c, d = p["recv_ptr"][peer], p["recv_ptr"][peer + 1]
            if b > a:
                buf = torch.from_numpy(np.ascontiguousarray(W[:, p["send_idx"][a:b]].T))
                sendbufs.append(buf)
                ops.append(dist.P2POp(dist.isend, buf, peer))
            if d > c:
                rb = torch.empty((d - c, 4), dtype=torch.float64)
                ops.append(dist.P2POp(dist.irecv, rb, peer))
                sendbufs.append((rb, c, d))
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        for item in sendbufs:
            if isinstance(item, tuple):
                rb, c, d = item
                W[:, n_own + c:n_own + d] = rb.numpy().T

    def allmin(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        return float(t.item())

    out = _run_rank(mesh, plans, rank, W0, steps, exchange, allmin)
    q.put((rank, p["local_vertices"][:n_own].copy(), out))
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["grid", "jittered"])
def test_two_rank_gloo_exchange_equals_one_rank(kind):
    import torch.multiprocessing as mp
    steps = 3
    mesh = _mesh(kind)
    W0 = inputs.khi_state(mesh) if kind == "grid" else inputs.vortex_state(mesh)
    plan1 = [binding.partition_plan(mesh, 1, 0)]
    ref = _run_rank(mesh, plan1, 0, W0, steps, lambda W: None, lambda x: x)
    ref_full = np.empty_like(W0)
    ref_full[:, plan1[0]["local_vertices"]] = ref
    # the single-rank stand-in is the oracle's own B2 step (same dt sequence)
    Wo, _ = oracle.run(mesh, W0, "B2", nsteps=steps)
    assert np.abs(ref_full - Wo).max() <= 1e-13 * np.abs(Wo).max()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, kind, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.full_like(W0, np.nan)
    for _, ids, W in res:
        got[:, ids] = W
    assert np.array_equal(got, ref_full)
