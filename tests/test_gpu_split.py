"""One grid split into slabs along its last dimension in one context
(fv_init_split: the decomposition a multi-GPU run distributes, Sec. 3.1's
two ghost layers copied device to device before every stage, dt
min-reduced over the slabs) equals the unsplit grid bit for bit, for every
stage kernel and scheme option the slabs can meet: walls, periodic wrap,
the inflow disc with a per-cell inflow array, App. D, CSF, viscous terms,
both precisions."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl

pytestmark = pytest.mark.gpu


def _run(w, precision, steps, split=None, inflow=None):
    s = fv.Solver(w, precision=precision, inflow_u=inflow, split=split)
    W = w.primitives()
    q = oracle.Oracle(w).prim_to_cons(W)
    if split:
        s.set_state_grid(q)
    else:
        s.set_state(q)
    s.step(steps, w.cfl)
    dts = [s.diag_scalar(fv.FV_DIAG_DT, case=c) for c in range(len(s.cases))]
    out = s.get_state_grid() if split else s.get_state()
    tile = s.tile()
    s.close()
    return out, dts, tile


def _jet():
    w = wl.jet3d(n=(40, 24, 24))
    return w, [wl.jet_inflow_velocity(w)]


CASES = {
    # name: (workload, inflow, precision, split (nblocks, rows), kernel environment)
    "shock_bubble_fused_mixed": (lambda: (wl.shock_bubble(nx=96, ny=48), None), fv.FV_MIXED, (2, None),
                                 dict(FV_FUSED="1")),
    "shock_bubble_tiled_fp64": (lambda: (wl.shock_bubble(nx=96, ny=48), None), fv.FV_FP64, (3, [20, 12, 16]),
                                dict(FV_TILE="0")),
    "droplet_csf_periodic_fused": (lambda: (wl.droplet(n=(64, 60), A=0.15), None), fv.FV_MIXED, (3, None),
                                   dict(FV_FUSED="1")),
    "random_iles_csf_periodic_tiled": (lambda: (wl.random_state(n=(40, 36), ncomp=3, iles=1, sigma=5.0), None),
                                       fv.FV_FP64, (2, None), dict(FV_TILE="1")),
    "rising_bubble_viscous_fused": (lambda: (wl.rising_bubble(1, n=(32, 64)), None), fv.FV_MIXED, (4, None),
                                    dict(FV_FUSED="1")),
    "jet3d_inflow_zmarch": (_jet, fv.FV_MIXED, (2, None), dict(FV_ZMARCH="1")),
    "jet3d_inflow_tiled_fp64": (_jet, fv.FV_FP64, (3, [8, 9, 7]), dict(FV_TILE="0")),
    "random3d_iles_csf_tiled": (lambda: (wl.random_state(n=(18, 14, 20), ndim=3, ncomp=3, iles=1, sigma=5.0,
                                                         bc=[[wl.BC_OUTFLOW] * 2, [wl.BC_PERIODIC] * 2,
                                                             [wl.BC_REFLECT, wl.BC_OUTFLOW]]), None),
                                fv.FV_MIXED, (2, [12, 8]), dict(FV_TILE="2", FV_ZMARCH="0")),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_split_equals_unsplit_bitwise(name, monkeypatch):
    make, precision, split, env = CASES[name]
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    w, inflow = make()
    # the random states are strong perturbations: the oracle itself turns
    # non-physical after four CFL steps of them
    steps = 3 if name.startswith("random") else 6
    ref, dref, tref = _run(w, precision, steps, inflow=inflow)
    got, dgot, tgot = _run(w, precision, steps, split=split, inflow=inflow)
    assert tref["fused"] == tgot["fused"] and tref["zmarch"] == tgot["zmarch"]
    assert all(d == dref[0] for d in dgot), (dgot, dref)
    assert np.array_equal(got, ref), np.abs(got - ref).max()
    assert np.abs(got - oracle.Oracle(w).prim_to_cons(w.primitives())).max() > 0


def test_split_argument_errors():
    w = wl.random_state(n=(16, 12))
    with pytest.raises(ValueError):
        fv.Solver(w, split=(7, None))          # a slab of fewer than two rows
    with pytest.raises(ValueError):
        fv.Solver(w, split=(2, [7, 6]))        # rows must add up to ny (the C ABI checks the same)
