"""GPU parity with the oracle for the Peng-Robinson closure (App. A.2.1):
FP64 Newton inversion warm-started from the previous temperature, cubic TDU
with the lowest-Gibbs root, and the FP32-mixed form's accuracy."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl
from tests.helpers import oracle_step_dt, rel_field_diff, rel_l1_vec

pytestmark = pytest.mark.gpu


def _mom(d, w, got, ref):
    mag = np.sqrt((ref[1:1 + w.ndim] ** 2).sum(0)).max()
    for a in range(w.ndim):
        d[1 + a] = np.abs(got[1 + a] - ref[1 + a]).max() / mag
    return d


def test_pr_random_state_parity():
    w = wl.random_state(n=(37, 23), pr=True)
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(q)
    dt = 0.3 * o.dt(q, 1.0)
    ref = q
    for _ in range(2):
        s.step_dt(dt)
        ref = oracle_step_dt(o, ref, dt)
    d = rel_field_diff(s.get_state(), ref)
    assert np.all(d < 1e-10), d
    # primitive read-back through the GPU's own Newton inversion
    Wg = s.get_state(fv.FV_PRIMITIVE)
    Wo = o.cons_to_prim(ref)
    assert np.abs(Wg[3] / Wo[3] - 1).max() < 1e-10          # temperature
    assert np.abs(Wg[2] / Wo[2] - 1).max() < 1e-8            # pressure


def test_pr_shock_droplet_small_fp64_and_mixed():
    w = wl.pr_shock_droplet(n=64)
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    ref, t_ref = o.step(q, 10, w.cfl)
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(q)
    t = s.step(10, w.cfl)
    got = s.get_state()
    d = _mom(rel_field_diff(got, ref), w, got, ref)
    assert np.all(d < 1e-9), d
    assert t == pytest.approx(t_ref, rel=1e-10, abs=0)
    m = fv.Solver(w, precision=fv.FV_MIXED)
    m.set_state(q)
    m.step(10, w.cfl)
    e = rel_l1_vec(m.get_state(), ref, w.ndim)
    assert np.all(e < 1e-3), e
