"""Slab decomposition of one grid (the multi-GPU layout of the stage, Sec. 3.1:
the compact stencil needs two ghost planes from each neighbouring slab per
stage and one common dt per step), on CPU: the slab plan, the halo strips,
and a world-size-2 gloo run in which each rank advances its own slab with
the oracle, exchanging ghost planes before every stage and min-reducing dt,
and the gathered result equals the unsplit oracle step bit for bit."""
import dataclasses
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2304_00140_gb300 import slabs, workloads as wl


def test_plan_covers_the_grid_and_links_neighbours():
    for n, nb, per in ((20, 2, False), (21, 4, False), (9, 3, True), (8, 1, True), (7, 2, True)):
        p = slabs.plan(n, nb, periodic=per)
        assert sum(s["rows"] for s in p) == n
        assert [s["row0"] for s in p] == list(np.cumsum([0] + [s["rows"] for s in p[:-1]]))
        assert max(s["rows"] for s in p) - min(s["rows"] for s in p) <= 1
        for b, s in enumerate(p):
            if s["hi"] >= 0:
                assert p[s["hi"]]["lo"] == b
            if s["lo"] >= 0:
                assert p[s["lo"]]["hi"] == b
        assert (p[0]["lo"] >= 0) == per and (p[-1]["hi"] >= 0) == per
    with pytest.raises(ValueError):
        slabs.plan(10, 6)              # a slab would have fewer than two planes
    with pytest.raises(ValueError):
        slabs.plan(10, 2, rows=[3, 6])


def test_strips_pair_sends_with_receives():
    p = slabs.plan(17, 3, periodic=True)
    for b in range(3):
        st = slabs.strips(p, b)
        lo, hi = p[b]["lo"], p[b]["hi"]
        assert st["recv_lo"] == slabs.strips(p, lo)["send_hi"]
        assert st["recv_hi"] == slabs.strips(p, hi)["send_lo"]
        assert st["send_lo"][1] - st["send_lo"][0] == slabs.GHOST


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(periodic):
    bc_y = [wl.BC_PERIODIC] * 2 if periodic else [wl.BC_REFLECT, wl.BC_OUTFLOW]
    return wl.random_state(n=(14, 18), ncomp=3, iles=1, sigma=5.0,
                           bc=[[wl.BC_OUTFLOW, wl.BC_REFLECT], bc_y, [wl.BC_PERIODIC] * 2])


def _local(w, s, ax_d):
    """this slab with a neighbour's ghost planes as real cells on each shared
    side (zero-gradient beyond them: those cells' results are discarded)"""
    lo_g = slabs.GHOST if s["lo"] >= 0 else 0
    hi_g = slabs.GHOST if s["hi"] >= 0 else 0
    n = list(w.n)
    n[ax_d] = s["rows"] + lo_g + hi_g
    bc = [list(b) for b in w.bc]
    bc[ax_d] = [wl.BC_OUTFLOW if s["lo"] >= 0 else w.bc[ax_d][0],
                wl.BC_OUTFLOW if s["hi"] >= 0 else w.bc[ax_d][1]]
    return dataclasses.replace(w, n=n, bc=bc), lo_g, hi_g


def _worker(rank, world, port, periodic, q):
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _case(periodic)
        ax_d, ax = 1, 2                 # split y: array axis 2 of [nv, nz, ny, nx]
        p = slabs.plan(w.n[ax_d], world, periodic=periodic)
        s = p[rank]
        og = oracle.Oracle(w)
        q_all = og.prim_to_cons(w.primitives())
        wl_, lo_g, hi_g = _local(w, s, ax_d)
        ol = oracle.Oracle(wl_)
        ol.P.dx[ax_d] = og.P.dx[ax_d]    # the grid's own cell size, bit for bit
        # local arrays carry GHOST planes at both ends (unused where the side is the grid's)
        G = slabs.GHOST
        buf = torch.zeros((w.nvar, 1, s["rows"] + 2 * G, w.n[0]), dtype=torch.float64)
        buf[:, :, G:G + s["rows"]] = torch.from_numpy(q_all[:, :, s["row0"]:s["row0"] + s["rows"]])
        own = slice(G, G + s["rows"])
        used = slice(G - lo_g, G + s["rows"] + hi_g)

        def stage(k, dt, q0, prev):
            slabs.exchange(prev, p, rank, dist, axis=ax)
            out = ol.stage(k, dt, q0[:, :, used].numpy().copy(), prev[:, :, used].numpy().copy())
            res = prev.clone()
            res[:, :, used] = torch.from_numpy(out)
            return res
        wown = dataclasses.replace(w, n=[w.n[0], s["rows"], 1])
        oown = oracle.Oracle(wown)
        oown.P.dx[ax_d] = og.P.dx[ax_d]
        for _ in range(2):
            dt = slabs.min_dt(oown.dt(buf[:, :, own].numpy().copy(), w.cfl), dist)
            q0 = buf.clone()
            slabs.exchange(q0, p, rank, dist, axis=ax)
            prev = q0
            for k in (1, 2, 3, 4):
                prev = stage(k, dt, q0, prev)
            buf = prev
        mine = buf[:, :, own].contiguous()
        sizes = [pp["rows"] for pp in p]
        gathered = [torch.zeros((w.nvar, 1, r, w.n[0]), dtype=torch.float64) for r in sizes]
        if rank == 0:
            gathered[0].copy_(mine)
            for r in range(1, world):
                dist.recv(gathered[r], r)
            got = torch.cat(gathered, dim=ax).numpy()
            ref, _ = og.step(q_all, 2, w.cfl)
            q.put(("diff", float(np.abs(got - ref).max()), float(np.abs(ref - q_all).max())))
        else:
            dist.send(mine, 0)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("periodic", [False, True])
def test_gloo_two_slabs_equal_unsplit_oracle(periodic):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, periodic, q)) for r in range(2)]
    for p in ps:
        p.start()
    tag, diff, moved = q.get(timeout=300)
    for p in ps:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in ps)
    assert diff == 0.0, diff
    assert moved > 0.0
