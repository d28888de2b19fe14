"""Multi-rank host logic of the replica runs, on CPU with gloo (world size 2):
the barrier / max-over-ranks timing and the whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1606_03416_gb300 import replicas as R
    r, w, lr = R.rank_info()
    dist.barrier()
    mx = R.max_over_ranks([1.0 + rank, 10.0 - rank])
    thr = R.job_throughput(100.0, w, mx[0])
    q.put((r, w, lr, mx, thr))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, lr, mx, thr) in enumerate(res):
        assert (rank, world, lr) == (r, 2, r)
        assert mx == [2.0, 10.0]
        assert thr == pytest.approx(100.0 * 2 / 2.0)


def test_single_process_identity():
    from paper_1606_03416_gb300 import replicas as R
    assert R.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
