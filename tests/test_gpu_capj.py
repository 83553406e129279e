"""GPU parity with the FP64 oracle for the capillary-jump surface tension
(the Sec. 3.5 alternative to the CSF force: [P] = sigma kappa [alpha] in the
Riemann solver), 2D and 3D, both curvature options, plain and App. D mode,
and the FP32-mixed form's accuracy; a static drop compares the parasitic
velocity of the two surface-tension models."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl
from tests.helpers import oracle_step_dt, rel_field_diff, rel_l1_vec

pytestmark = pytest.mark.gpu


def _rel(w, got, ref):
    d = rel_field_diff(got, ref)
    mag = np.sqrt((ref[1:1 + w.ndim] ** 2).sum(0)).max()
    for a in range(w.ndim):
        d[1 + a] = np.abs(got[1 + a] - ref[1 + a]).max() / mag
    return d


CASES = {
    "droplet_2d": lambda: wl.droplet(n=(48, 44), A=0.15, sigma=30.0, st_model=1),
    "droplet_2d_height_function": lambda: wl.droplet(n=(48, 44), A=0.15, sigma=30.0, st_model=1, curvature=1),
    "random_2d_iles_3comp": lambda: wl.random_state(n=(40, 33), ncomp=3, iles=1, sigma=5.0, st_model=1),
    "random_3d_iles_walls": lambda: wl.random_state(n=(18, 17, 21), ndim=3, ncomp=3, iles=1, sigma=5.0, st_model=1,
                                                    bc=[[wl.BC_REFLECT, wl.BC_OUTFLOW], [wl.BC_PERIODIC] * 2,
                                                        [wl.BC_OUTFLOW, wl.BC_REFLECT]]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_capillary_jump_parity_fp64(name):
    w = CASES[name]()
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(q)
    dt = 0.3 * o.dt(q, 1.0)
    ref = q
    for _ in range(3):
        s.step_dt(dt)
        ref = oracle_step_dt(o, ref, dt)
    assert not s.tile()["fused"] and not s.tile()["zmarch"]
    d = _rel(w, s.get_state(), ref)
    assert np.all(d < 1e-10), d
    # the jump model changes the result (against CSF)
    w0 = CASES[name]()
    w0.scheme = dict(w0.scheme, st_model=0)
    assert np.abs(oracle_step_dt(oracle.Oracle(w0), q, dt) - oracle_step_dt(o, q, dt)).max() > 0


def test_capillary_jump_mixed_accuracy_droplet():
    """FP32-mixed droplet with the jump model after 60 CFL steps: density,
    energy, mass fraction within 1e-4 relative L1 of the oracle"""
    w = wl.droplet(n=64, A=0.15, st_model=1)
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_MIXED)
    s.set_state(q)
    s.step(60, w.cfl)
    ref, _ = o.step(q, 60, w.cfl)
    e = rel_l1_vec(s.get_state(), ref, w.ndim)
    assert np.all(np.r_[e[:1], e[1 + w.ndim:]] < 1e-4), e


def test_static_drop_laplace_jump_both_models():
    """a drop at rest with the Laplace jump preset (sigma = 1 N/m, R = 25
    cells, FP64): the drop rings acoustically (the jump swings between about
    -0.4 and 2.6 sigma/R with a period near 1.2 us, in the oracle as on the
    GPU), so the jump is averaged over steps 1000 .. 8000, sampled every 50;
    that average is sigma/R within 25% for both surface-tension models, and
    the parasitic velocity stays bounded.  Reported for both models."""
    out = {}
    for model in (0, 1):
        n, L = 100, 1e-3
        R = 0.25 * L
        w = wl.droplet(n=n, A=0.0, sigma=1.0, dp=1.0 / R, st_model=model)
        s = fv.Solver(w, precision=fv.FV_FP64)
        s.set_state(w.primitives(), kind=fv.FV_PRIMITIVE)
        s.step(1000, w.cfl)
        jumps, umax = [], 0.0
        for _ in range(140):
            s.step(50, w.cfl)
            W = s.get_state(fv.FV_PRIMITIVE)
            p = W[2][0]
            jumps.append(p[n // 2 - 3:n // 2 + 3, n // 2 - 3:n // 2 + 3].mean() - p[:5, :5].mean())
            umax = np.sqrt(W[0] ** 2 + W[1] ** 2).max()
        out[model] = (float(np.mean(jumps)) * R, float(umax))
    print("static drop, jump * R / sigma averaged over steps 1000-8000 and max |u| (m/s) at step 8000: CSF",
          out[0], "capillary jump", out[1])
    for model, (j, u) in out.items():
        assert abs(j - 1.0) < 0.25 and u < 10.0, (model, j, u)
