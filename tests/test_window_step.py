"""The windowed oracle step that the full-size GPU parity tests and the
benchmark's CPU baseline use (no GPU): stage k evaluated on the window grown
by 2 (4 - k) cells gives, inside the window, exactly the full grid's step,
for walls, outflow and inflow sides, the App. D switch with CSF, viscous
terms with gravity, the capillary jump and 3D.  On periodic grids the
window keeps the growth's distance from the sides (the growth is clipped,
not wrapped)."""
import dataclasses
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl
from tests.helpers import oracle_step_dt, oracle_step_window

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _cases():
    sb = wl.shock_bubble(nx=48, ny=24)
    dr = wl.droplet(n=24, sigma=0.07, iles=1)
    rb = wl.rising_bubble(2, n=(16, 32))
    dj = wl.droplet(n=32, sigma=0.07)
    cj = dataclasses.replace(dj, scheme=dict(dj.scheme, st_model=1))
    jet = wl.jet3d(n=(16, 12, 12))
    return dict(shock_bubble=(sb, None), droplet_iles_csf=(dr, None), rising_bubble=(rb, None),
                capillary_jump=(cj, None), jet3d=(jet, wl.jet_inflow_velocity(jet)))


@pytest.mark.parametrize("name", list(_cases()))
def test_window_step_equals_the_full_step(name):
    w, u = _cases()[name]
    o = oracle.Oracle(w, inflow_u=u)
    q = o.prim_to_cons(w.primitives())
    dt = 0.3 * o.dt(q, 1.0)
    full = oracle_step_dt(o, q, dt)
    rng = np.random.default_rng(5)
    # the growth is clipped at the grid's sides: a window keeps the first
    # stage's growth (6 cells, 9 with the capillary jump) from a periodic side
    g1 = 9 if name == "capillary_jump" else 6
    m = [g1 if d < w.ndim and w.bc[d][0] == wl.BC_PERIODIC else 0 for d in range(3)]
    for _ in range(2):
        lo = [int(rng.integers(m[d], w.n[d] - m[d])) if d < w.ndim else 0 for d in range(3)]
        hi = [int(rng.integers(lo[d] + 1, w.n[d] - m[d] + 1)) if d < w.ndim else 1 for d in range(3)]
        lo[0] = 0 if name == "jet3d" else lo[0]                # the inflow side inside a window
        sl = (slice(None), slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        got = oracle_step_window(o, q, dt, lo, hi)
        assert np.array_equal(got[sl], full[sl]), name
        if name != "capillary_jump":
            assert np.array_equal(bench.oracle_window_step(o, q, dt, lo, hi)[sl], full[sl])
    assert np.abs(full - q).max() > 0
