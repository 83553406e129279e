"""Host-side multi-process path of the benchmark, on CPU with gloo and two
ranks: the batch split covers every case once with balanced cells, and the
timing reduction returns the slowest rank's time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2304_00140_gb300 import replicas, workloads as wl


def test_lpt_partition_covers_and_balances():
    cases = wl.droplet_ensemble(ncases=200)
    w = [c.cells for c in cases]
    parts = replicas.lpt_partition(w, 2)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(cases)))
    loads = [sum(w[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(w)
    assert replicas.lpt_partition([3.0, 1.0], 4)[2:] == [[], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = replicas.max_over_ranks(1.5 + rank, dist)
    s = replicas.sum_over_ranks(10.0 * (rank + 1), dist)
    cases = wl.droplet_ensemble(ncases=64)
    mine = replicas.lpt_partition([c.cells for c in cases], world)[rank]
    n_all = replicas.sum_over_ranks(len(mine), dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, s, n_all))


def test_gloo_two_ranks_timing_and_split():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in ps)
    for rank, t, s, n_all in out:
        assert t == 2.5            # the slowest rank's time
        assert s == 30.0
        assert n_all == 64         # every case on exactly one rank
