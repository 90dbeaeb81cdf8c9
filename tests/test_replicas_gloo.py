"""The N > 1 benchmark path (independent replicas) on CPU with gloo, world
size 2: every rank sees the slowest rank's time, and the whole-job rate is
the units of all ranks over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1906_11925_gb300 import replicas  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = replicas.rank_env()
    assert (r, lr, w) == (rank, rank, world)
    replicas.barrier(w)
    t = 1.0 + rank * 0.5          # rank 1 is the slowest replica
    tmax = replicas.max_over_ranks(t, w)
    rate = replicas.whole_job_rate(1000.0, w, tmax)
    out.put((rank, tmax, rate))
    dist.destroy_process_group()


def test_replicas_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for _, tmax, rate in res:
        assert tmax == 1.5
        assert rate == 2 * 1000.0 / 1.5


def test_single_rank_is_identity():
    assert replicas.max_over_ranks(3.25, 1) == 3.25
    assert replicas.whole_job_rate(10.0, 1, 2.0) == 5.0
