"""Slab decomposition of one grid along its last dimension (y in 2D, z in
3D) and the halo exchange its stencil needs.

The stage of Sec. 3.1 reads two cells on each side of a face, so a slab that
owns planes [row0, row0 + rows) needs two ghost planes from each neighbouring
slab before every stage, and every slab must advance with the same dt (the
smallest over all slabs).  ``plan`` gives the slabs (the same rule the C ABI's
``fv_init_split`` uses when no row counts are passed); ``strips`` says which
planes a slab sends to and receives from each neighbour; ``exchange`` and
``min_dt`` carry them out between processes with ``torch.distributed`` on
host tensors laid out as ``[nv, planes + 4, ...]`` (two ghost planes at each
end of the split axis).  No scheme arithmetic lives here.
"""
from __future__ import annotations

from typing import Dict, List, Optional

GHOST = 2     # ghost planes per side (the stage's two-cell stencil reach)


def plan(n: int, nblocks: int, rows: Optional[List[int]] = None, periodic: bool = False) -> List[Dict]:
    """Slabs of a split dimension of n planes: row0, rows and the neighbouring
    slab across the low and high side (-1: the grid's own boundary)."""
    if nblocks < 1 or nblocks > n // GHOST:
        raise ValueError("nblocks must be 1 .. n/2")
    if rows is None:
        rows = [n // nblocks + (1 if b < n % nblocks else 0) for b in range(nblocks)]
    if len(rows) != nblocks or sum(rows) != n or min(rows) < GHOST:
        raise ValueError("slab rows must be >= 2 each and add up to n")
    out, r0 = [], 0
    for b, r in enumerate(rows):
        lo = b - 1 if b > 0 else (nblocks - 1 if periodic else -1)
        hi = b + 1 if b < nblocks - 1 else (0 if periodic else -1)
        out.append(dict(row0=r0, rows=r, lo=lo, hi=hi))
        r0 += r
    return out


def strips(p: List[Dict], b: int) -> Dict:
    """Planes (global indices, half-open) slab b sends towards each
    neighbour and receives into its ghost planes from it."""
    s = p[b]
    r0, r1 = s["row0"], s["row0"] + s["rows"]
    out = {}
    if s["lo"] >= 0:
        nb = p[s["lo"]]
        out["send_lo"] = (r0, r0 + GHOST)
        out["recv_lo"] = (nb["row0"] + nb["rows"] - GHOST, nb["row0"] + nb["rows"])
    if s["hi"] >= 0:
        nb = p[s["hi"]]
        out["send_hi"] = (r1 - GHOST, r1)
        out["recv_hi"] = (nb["row0"], nb["row0"] + GHOST)
    return out


def exchange(local, p: List[Dict], rank: int, dist, axis: int = 1) -> None:
    """Fill the ghost planes of this rank's slab ``local`` (a host tensor
    with GHOST extra planes at each end of ``axis``) from its neighbours'
    owned planes: every rank sends first-two / last-two owned planes and
    receives the matching planes of its neighbours."""
    s = p[rank]
    n = s["rows"]

    def planes(a, b):
        return local.narrow(axis, a, b - a)
    reqs, recvs = [], []
    for side, nb in (("lo", s["lo"]), ("hi", s["hi"])):
        if nb < 0:
            continue
        own = planes(GHOST, 2 * GHOST) if side == "lo" else planes(n, n + GHOST)
        ghost = planes(0, GHOST) if side == "lo" else planes(n + GHOST, n + 2 * GHOST)
        if nb == rank:      # a single periodic slab wraps onto itself
            other = planes(n, n + GHOST) if side == "lo" else planes(GHOST, 2 * GHOST)
            ghost.copy_(other)
            continue
        buf = ghost.contiguous().clone()
        reqs.append(dist.isend(own.contiguous(), nb, tag=0 if side == "lo" else 1))
        reqs.append(dist.irecv(buf, nb, tag=1 if side == "lo" else 0))
        recvs.append((ghost, buf))
    for r in reqs:
        r.wait()
    for ghost, buf in recvs:
        ghost.copy_(buf)


def min_dt(dt: float, dist) -> float:
    """The step's dt: the smallest over all slabs."""
    import torch
    t = torch.tensor([dt], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item())
