"""The multi-GPU path's host logic (independent replicas, no data-path
collective) on two CPU ranks over gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_1701_08475_gb300 import replicas
    replicas.init("gloo")
    r, w, _ = replicas.rank_env()
    rows = replicas.replica_rows(1000, r)
    seconds = 0.5 + r              # this rank's time for its steps
    replicas.barrier()
    slowest = replicas.max_over_ranks(seconds)
    q.put((r, w, rows[:5].tolist(), sorted(rows.tolist()) == list(range(1000)), slowest,
           replicas.aggregate(1000, 3, slowest, w)))
    replicas.finish()


def test_two_ranks_draw_their_own_replica_and_time_by_the_slowest():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    (r0, w0, head0, perm0, slow0, agg0), (r1, w1, head1, perm1, slow1, agg1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert perm0 and perm1                     # each replica is all the rows
    assert head0 == [0, 1, 2, 3, 4] and head1 != head0
    assert slow0 == slow1 == 1.5               # the slowest rank sets the job's time
    assert agg0 == agg1 == 2 * 1000 * 3 / 1.5  # every rank's points over that time


def test_one_rank_needs_no_process_group():
    from paper_1701_08475_gb300 import replicas
    assert replicas.max_over_ranks(2.5) == 2.5
    assert replicas.aggregate(10, 2, 4.0, 1) == 5.0
    assert list(replicas.replica_rows(4, 0)) == [0, 1, 2, 3]
