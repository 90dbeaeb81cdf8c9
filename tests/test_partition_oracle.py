"""Domain decomposition, emulated on the host with the FP64 oracle: k
contiguous Morton ranges, each stepping its own sites plus a halo refreshed
from the owning ranks after every step, reproduce the unpartitioned run bit
for bit (in one process for k = 1..4, and as two gloo ranks that exchange
their halos with send/recv)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1906_11925_gb300 import geometry as G
from paper_1906_11925_gb300 import partition as PT

torch = pytest.importorskip("torch")


def _case(q=15, seed=81):
    g = G.random_mask((9, 8, 7), p=0.65, seed=seed, n_iolets=2)
    nbr, link = oracle.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    rng = np.random.default_rng(seed)
    f0 = oracle.rest_state(q, g.n) * (1.0 + 0.01 * (2 * rng.random((q, g.n)) - 1))
    return g, nbr, link, f0


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_plan_covers_the_lattice(k):
    g, nbr, link, _ = _case()
    parts = PT.plan(g.xyz, nbr, link, k)
    own = np.concatenate([p.own for p in parts])
    assert np.array_equal(np.sort(own), np.arange(g.n))
    order = PT.morton_order(g.xyz)
    rank_in_order = np.empty(g.n, dtype=np.int64)
    rank_in_order[order] = np.arange(g.n)
    for p in parts:
        pos = np.sort(rank_in_order[p.own])
        assert np.all(np.diff(pos) == 1)  # a contiguous Morton range
        assert abs(p.n_own - g.n / k) <= 1
        assert not np.intersect1d(p.own, p.halo).size
        # every fluid link of an own site stays inside the local problem
        assert np.array_equal(p.link[:, : p.n_own], link[:, p.own])
        loc = p.nbr[:, : p.n_own]
        fl = p.link[:, : p.n_own] == 0
        assert np.array_equal(p.local[loc[fl]], nbr[:, p.own][fl])
    send = PT.exchange_lists(parts)
    for p in parts:
        got = np.concatenate([send[r][p.rank] for r in range(k) if r != p.rank] or [np.empty(0, int)])
        assert np.array_equal(np.sort(got), np.sort(p.halo))


@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("k", [2, 3, 4])
def test_partitioned_steps_are_bit_exact(q, k):
    g, nbr, link, f0 = _case(q)
    parts = PT.plan(g.xyz, nbr, link, k)
    tau, steps = 0.7, 12
    f = f0.copy()
    for t in range(steps):
        new = np.empty_like(f)
        for p in parts:
            fl = oracle.step(q, p.nbr, p.link, tau, f[:, p.local], t=t, geom=g)
            new[:, p.own] = fl[:, : p.n_own]
        f = new
    ref = oracle.run(q, nbr, link, tau, f0, steps, geom=g)
    assert np.array_equal(f, ref)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q, steps, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, nbr, link, f0 = _case(q)
    parts = PT.plan(g.xyz, nbr, link, world)
    send = PT.exchange_lists(parts)
    me = parts[rank]
    tau = 0.7
    f_own = f0[:, me.own].copy()  # this rank holds only its own sites' state
    own_pos = {int(x): i for i, x in enumerate(me.own)}
    for t in range(steps):
        # halo exchange: populations of the sites the other ranks need
        halo = np.empty((q, me.halo.shape[0]))
        reqs = []
        bufs = {}
        for r in range(world):
            if r == rank:
                continue
            idx = np.array([own_pos[int(x)] for x in send[rank][r]], dtype=np.int64)
            buf = torch.from_numpy(np.ascontiguousarray(f_own[:, idx])) if idx.size else torch.zeros(q, 0, dtype=torch.float64)
            reqs.append(dist.isend(buf, dst=r))
            rb = torch.empty(q, send[r][rank].shape[0], dtype=torch.float64)
            reqs.append(dist.irecv(rb, src=r))
            bufs[r] = rb
        for rq in reqs:
            rq.wait()
        for r, rb in bufs.items():
            sel = me.owner_of_halo == r
            halo[:, sel] = rb.numpy()  # send[r][rank] lists r's sites in my halo order
        f_local = np.concatenate([f_own, halo], axis=1)
        f_own = oracle.step(q, me.nbr, me.link, tau, f_local, t=t, geom=g)[:, : me.n_own]
    # gather on rank 0
    if rank == 0:
        full = np.empty((q, g.n))
        full[:, me.own] = f_own
        for r in range(1, world):
            rb = torch.empty(q, parts[r].n_own, dtype=torch.float64)
            dist.recv(rb, src=r)
            full[:, parts[r].own] = rb.numpy()
        ref = oracle.run(q, nbr, link, tau, f0, steps, geom=g)
        out.put(bool(np.array_equal(full, ref)))
    else:
        dist.send(torch.from_numpy(np.ascontiguousarray(f_own)), dst=0)
    dist.destroy_process_group()


def test_partitioned_gloo_world2_is_bit_exact():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, 19, 10, out)) for r in range(2)]
    for p in procs:
        p.start()
    ok = out.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert ok
