"""GPU parity with the oracle for the CSF source, the App. D switch, 3D grids,
three components, the inflow disc, batches of droplets and the FP32-mixed
form's accuracy."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl
from tests.helpers import oracle_step_dt, rel_field_diff, rel_l1_vec

pytestmark = pytest.mark.gpu


def _run_pair(w, steps_dt=1, dt_frac=0.3, inflow_u=None, precision=fv.FV_FP64):
    o = oracle.Oracle(w, inflow_u=inflow_u)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=precision, inflow_u=[inflow_u] if inflow_u is not None else None)
    s.set_state(q)
    dt = dt_frac * o.dt(q, 1.0)
    ref = q
    for _ in range(steps_dt):
        s.step_dt(dt)
        ref = oracle_step_dt(o, ref, dt)
    return o, q, s.get_state(), ref


def _scale_momentum(d, w, got, ref):
    """momentum components measured against the momentum vector's scale"""
    nd = w.ndim
    mag = np.sqrt((ref[1:1 + nd] ** 2).sum(0)).max()
    for a in range(nd):
        d[1 + a] = np.abs(got[1 + a] - ref[1 + a]).max() / mag
    return d


# 2D cases run both stage kernels: tiled after a primitive pass (FV_FUSED=0)
# and fused (FV_FUSED=1)
FUSED = pytest.mark.parametrize("fused", ["0", "1"])


@FUSED
def test_csf_droplet_parity(fused, monkeypatch):
    monkeypatch.setenv("FV_FUSED", fused)
    w = wl.droplet(n=(40, 36), A=0.15, sigma=30.0)
    o, q, got, ref = _run_pair(w, steps_dt=3)
    S = o.csf_source(q)
    assert np.abs(S).max() > 0.0
    d = _scale_momentum(rel_field_diff(got, ref), w, got, ref)
    assert np.all(d < 1e-11), d


@FUSED
def test_iles_switch_parity_2d(fused, monkeypatch):
    monkeypatch.setenv("FV_FUSED", fused)
    w = wl.random_state(n=(40, 33), iles=1)
    o = oracle.Oracle(w)
    f = o.sensor(o.prim_to_cons(w.primitives()))
    assert 0.05 < f.mean() < 0.95          # both branches of Eq. D.3 are exercised
    o, q, got, ref = _run_pair(w, steps_dt=2)
    d = rel_field_diff(got, ref)
    assert np.all(d < 1e-11), d


@FUSED
@pytest.mark.parametrize("ncomp", [2, 3])
def test_iles_csf_2d_parity(ncomp, fused, monkeypatch):
    """App. D switch and CSF together in 2D, two or three components, mixed
    boundary kinds."""
    monkeypatch.setenv("FV_FUSED", fused)
    w = wl.random_state(n=(45, 31), ncomp=ncomp, iles=1, sigma=5.0,
                        bc=[[wl.BC_OUTFLOW, wl.BC_REFLECT], [wl.BC_PERIODIC] * 2, [0, 0]])
    o, q, got, ref = _run_pair(w, steps_dt=2)
    d = _scale_momentum(rel_field_diff(got, ref), w, got, ref)
    assert np.all(d < 1e-11), d


# the tiled kernel's halo tiles: TMA bulk tensor copies (FV_TMA=1) or
# per-element cp.async (FV_TMA=0)
TMA = pytest.mark.parametrize("tma", ["1", "0"])


@TMA
@pytest.mark.parametrize("ncomp", [2, 3])
def test_plain_3d_parity(ncomp, tma, monkeypatch):
    monkeypatch.setenv("FV_TMA", tma)
    w = wl.random_state(n=(20, 14, 11), ndim=3, ncomp=ncomp)
    o, q, got, ref = _run_pair(w)
    d = rel_field_diff(got, ref)
    assert np.all(d < 1e-12), d


@TMA
def test_iles_csf_3d_three_components_parity(tma, monkeypatch):
    monkeypatch.setenv("FV_TMA", tma)
    w = wl.random_state(n=(18, 12, 10), ndim=3, ncomp=3, iles=1, sigma=5.0,
                        bc=[[wl.BC_OUTFLOW, wl.BC_REFLECT], [wl.BC_PERIODIC] * 2, [wl.BC_REFLECT, wl.BC_OUTFLOW]])
    o, q, got, ref = _run_pair(w, steps_dt=2)
    d = _scale_momentum(rel_field_diff(got, ref), w, got, ref)
    assert np.all(d < 1e-11), d


def test_jet_inflow_parity():
    """Inflow disc, three components and CSF in 3D.  Plain mode: in the
    quiescent gas ahead of an impulsive jet the App. D Ducros ratio is formed
    from rounding-level velocities, so its decisions there follow rounding
    noise (a 1e-15 perturbation of the oracle's own input flips hundreds of
    them) and FP64 parity is only defined away from that; the switch itself is
    checked on states with O(10 m/s) velocities above."""
    w = wl.jet3d(n=(24, 16, 16), iles=0)
    w.inflow["radius"] = 4.5 * w.dx[1]
    u = wl.jet_inflow_velocity(w)
    o, q, got, ref = _run_pair(w, steps_dt=4, inflow_u=u)
    # the liquid has entered
    assert (ref[2 + w.ndim, :, :, 0] / ref[0, :, :, 0]).min() < 0.5
    d = _scale_momentum(rel_field_diff(got, ref), w, got, ref)
    assert np.all(d < 1e-11), d


@FUSED
def test_droplet_batch_matches_single_and_oracle(fused, monkeypatch):
    monkeypatch.setenv("FV_FUSED", fused)
    cases = [wl.droplet(n=n, A=a, sigma=20.0) for n, a in ((24, 0.1), (40, 0.2), (33, 0.05), (16, 0.15))]
    qs = [oracle.Oracle(c).prim_to_cons(c.primitives()) for c in cases]
    b = fv.Solver(cases)
    for i, q in enumerate(qs):
        b.set_state(q, case=i)
    b.step(4, 0.4)
    for i, c in enumerate(cases):
        s = fv.Solver(c)
        s.set_state(qs[i])
        s.step(4, 0.4)
        assert np.array_equal(s.get_state(), b.get_state(case=i))
    ref, _ = oracle.Oracle(cases[1]).step(qs[1], 4, 0.4)
    got = b.get_state(case=1)
    d = _scale_momentum(rel_field_diff(got, ref), cases[1], got, ref)
    assert np.all(d < 1e-11), d


def test_mixed_form_accuracy_advection():
    """FP32-mixed 128^2 advection run (200 steps) against the FP64 oracle:
    relative L1 per conserved field below 1e-5."""
    w = wl.advection(n=128, steps=200)
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_MIXED)
    s.set_state(q)
    s.step(w.steps, w.cfl)
    ref, _ = o.step(q, w.steps, w.cfl)
    e = rel_l1_vec(s.get_state(), ref, w.ndim)
    assert np.all(e < 1e-5), e
    W = s.get_state(fv.FV_PRIMITIVE)
    # the low-Mach pressure survives the p + pinf cancellation in FP32
    assert np.abs(W[2] / 1e5 - 1).max() < 1e-3


def test_mixed_form_accuracy_droplets():
    """FP32-mixed oscillating droplets (CSF on) against the FP64 oracle after
    60 steps.  Density, energy and mass fraction: relative L1 below 1e-4.
    Momentum starts at zero and is the small residual of the pressure jump
    against the CSF force, so it is ill-conditioned: in the FP64 oracle itself
    a relative perturbation of the initial state of 1e-9 (well under FP32
    rounding) already moves it by 2e-4 to 3e-4 in L1.  Its bound is therefore
    the oracle's own spread under a 1e-8 relative input perturbation."""
    cases = [wl.droplet(n=64, A=0.15), wl.droplet(n=96, A=0.08)]
    m = fv.Solver(cases, precision=fv.FV_MIXED)
    refs, spread = [], []
    rng = np.random.default_rng(20230401)
    for i, c in enumerate(cases):
        o = oracle.Oracle(c)
        q = o.prim_to_cons(c.primitives())
        m.set_state(q, case=i)
        ref = o.step(q, 60, c.cfl)[0]
        pert = o.step(q * (1 + 1e-8 * rng.standard_normal(q.shape)), 60, c.cfl)[0]
        refs.append(ref)
        spread.append(rel_l1_vec(pert, ref, c.ndim))
    m.step(60, 0.4)
    for i, c in enumerate(cases):
        e = rel_l1_vec(m.get_state(case=i), refs[i], c.ndim)
        mom = slice(1, 1 + c.ndim)
        other = np.r_[e[:1], e[1 + c.ndim:]]
        assert np.all(other < 1e-4), (i, e)
        assert np.all(e[mom] < spread[i][mom]), (i, e, spread[i])
        # the spread is a conditioning figure, not a loose bound
        assert np.all(spread[i][mom] < 1e-2), spread[i]
