"""bench.py's multi-rank path (replicas, barrier, max over ranks) with world size 2 on gloo."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist

    class A:
        pass
    w, r, local = bench.dist_setup(A())
    bench.barrier(w)
    mx = bench.max_over_ranks(float(rank + 1) * 1.5, w)
    q.put((r, w, mx))
    dist.destroy_process_group()


def test_two_rank_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r for r, _, _ in res] == [0, 1]
    assert all(w == 2 for _, w, _ in res)
    assert all(mx == pytest.approx(3.0) for _, _, mx in res)


def test_reference_arm_other_ranks_exit_without_work():
    import bench

    class A:
        workload = "khi4096_B2"
        steps = 1
        warmup = 0
    assert bench.reference(A(), 2, 1) is None
