"""The fused 2D kernel's last stage also accumulates the CFL wave speeds of
the q^{n+1} it writes, so a step that follows a step of the same call takes
its dt from them and leaves out the CFL pass (Sec. 3.1: dt from the state at
the start of the step).  Several steps in one call (every step after the
first warm) must equal the same steps with the CFL pass in every step
(FV_FUSED_CFL=0), bit for bit, dt included; the launch counts show which
kind ran, and a state write makes the next step cold again."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl

pytestmark = pytest.mark.gpu

CASES = {
    "shock_bubble_plain": lambda: wl.shock_bubble(nx=160, ny=80),
    "shock_bubble_iles": lambda: wl.shock_bubble(nx=160, ny=80, iles=1),
    "droplet_csf": lambda: wl.droplet(n=64, A=0.15),
    "droplet_iles_csf": lambda: wl.droplet(n=96, A=0.15, iles=1),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_warm_steps_equal_cold_steps(name, monkeypatch):
    monkeypatch.setenv("FV_FUSED", "1")
    w = CASES[name]()
    q = oracle.Oracle(w).prim_to_cons(w.primitives())
    warm = fv.Solver(w, precision=fv.FV_MIXED)
    monkeypatch.setenv("FV_FUSED_CFL", "0")
    cold = fv.Solver(w, precision=fv.FV_MIXED)
    warm.set_state(q)
    cold.set_state(q)
    nsteps = 5
    l0, l1 = warm.launch_count(), cold.launch_count()
    warm.step(nsteps, w.cfl)
    cold.step(nsteps, w.cfl)
    assert warm.tile()["fused"] and cold.tile()["fused"]
    # a cold step: CFL pass, dt, four stages; a warm one leaves out the CFL pass
    assert warm.launch_count() - l0 == 6 + 5 * (nsteps - 1)
    assert cold.launch_count() - l1 == 6 * nsteps
    assert warm.diag_scalar(fv.FV_DIAG_DT) == cold.diag_scalar(fv.FV_DIAG_DT)
    a, b = warm.get_state(), cold.get_state()
    assert np.array_equal(a, b), np.abs(a - b).max()
    # the next call continues warm; after a state write it starts cold
    l0 = warm.launch_count()
    warm.step(1, w.cfl)
    assert warm.launch_count() - l0 == 5
    warm.set_state(a)
    l0 = warm.launch_count()
    warm.step(1, w.cfl)
    assert warm.launch_count() - l0 == 6
