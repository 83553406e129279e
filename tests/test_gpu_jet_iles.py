"""FP64 parity of the App. D switch on the jet (the 3D primary break-up
configuration: three components, the inflow disc, CSF, Eq. D.3-D.6), with
the switch's branch flips counted.

The reference trajectory is the oracle's; the GPU is fed the oracle's own
states, one stage at a time, so a difference cannot propagate.  The App. D
flag of a cell may differ between the two only where its decision is not
fixed by the arithmetic: theta^D or theta^Gas within 1e-12 of its threshold
(Eq. D.4), or the Ducros ratio where the divergence and the curl are both
at rounding level (|div u| dx and |curl u| dx at most 1e-12 of the largest
local |u|: differences of velocities equal in all but their last digits).  Every stage result matches the oracle to 1e-10 per field in
every cell that no flipped flag touches (a face takes the larger flag of its
two cells, so a flip reaches the cell and its face neighbours)."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl
from tests.helpers import cell_rel_diff, gpu_stage

pytestmark = pytest.mark.gpu

def _explained(o, q, flip):
    """flip cells whose decision lies at a threshold or whose velocity
    derivatives are at rounding level: |div u| dx and |curl u| dx at most
    1e-12 of the largest |u| among the cell and its face neighbours (the
    differences of nearly equal velocities, whose leading digits cancel)"""
    a = o.sensor_args(q)
    s = o.w.scheme
    nd = o.w.ndim
    dx = min(o.w.dx[:nd])
    umag = np.sqrt((o.cons_to_prim(q)[:nd] ** 2).sum(0))
    pad = np.pad(umag, 1, mode="edge")
    uloc = umag.copy()
    for ax in range(umag.ndim):
        for sh in (0, 2):
            sl = tuple(slice(sh, sh + umag.shape[d]) if d == ax else slice(1, 1 + umag.shape[d])
                       for d in range(umag.ndim))
            uloc = np.maximum(uloc, pad[sl])
    near = (np.abs(a[0] - s["thr_ducros"]) <= 1e-12) | (np.abs(a[1] - s["thr_gas"]) <= 1e-12)
    rounding = (a[3] * dx <= 1e-12 * uloc) & (a[4] * dx <= 1e-12 * uloc)
    return (near | rounding)[flip], a, near[flip], rounding[flip]


def _touched(flip):
    """cells a flipped flag can reach: the cell and its six face neighbours"""
    t = flip.copy()
    for ax in range(flip.ndim):
        t[tuple(slice(1, None) if d == ax else slice(None) for d in range(flip.ndim))] |= \
            flip[tuple(slice(None, -1) if d == ax else slice(None) for d in range(flip.ndim))]
        t[tuple(slice(None, -1) if d == ax else slice(None) for d in range(flip.ndim))] |= \
            flip[tuple(slice(1, None) if d == ax else slice(None) for d in range(flip.ndim))]
    return t


def test_jet_iles_parity_with_flip_accounting():
    w = wl.jet3d(n=(48, 24, 24))           # App. D switch on, sigma = 0.025, uniform 300 m/s inflow
    assert w.scheme["iles"] == 1 and w.scheme["sigma"] > 0
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_FP64)
    flips_total, checked = 0, 0
    for step in range(21):
        if step % 10 == 0:
            # the four stages of one step, each from the oracle's inputs: the
            # sensor of the stage's input state cell by cell, then the stage
            dt = 0.3 * o.dt(q, 1.0)
            prev = q
            for k in (1, 2, 3, 4):
                s.set_state(prev)
                f_gpu = s.sensor_flags().astype(bool)
                f_ora = o.sensor(prev) > 0.5
                assert 0 < f_ora.sum() < f_ora.size            # both branches occur
                flip = f_gpu != f_ora
                ok, a, nr, rd = _explained(o, prev, flip)
                if flip.any():
                    print(f"step {step} stage {k}: {int(flip.sum())} flips, {int(nr.sum())} at a threshold, "
                          f"{int(rd.sum())} at rounding level; theta^D - thr {a[0][flip] - 0.95}, "
                          f"theta^Gas - thr {a[1][flip] - 0.4}, div dx {a[3][flip] * min(w.dx)}")
                assert ok.all(), (step, k, np.argwhere(flip)[~ok][:5], a[:, flip][:, ~ok][:, :5])
                flips_total += int(flip.sum())
                ref = o.stage(k, dt, q, prev)
                got = gpu_stage(w, fv.FV_FP64, k, dt, q, prev)
                d = cell_rel_diff(got, ref)
                touched = _touched(flip)
                assert np.all(d[~touched] <= 1e-10), (step, k, d[~touched].max())
                checked += int((~touched).sum())
                prev = ref
        q, _ = o.step(q, 1, w.cfl)
    print(f"jet App. D: {flips_total} flag flips, all at a threshold or at rounding level; "
          f"{checked} cell-stages compared at 1e-10")
