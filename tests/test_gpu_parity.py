"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the FP64 form must match the oracle to 1e-10 relative per
conserved field (max |gpu - oracle| / max |oracle|) after the 128^2, 200-step
advection run, and to 1e-12 after single steps (different but equivalent
rounding order: division-free limiters, closed-form closure inverse)."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl
from tests.helpers import oracle_step_dt, oracle_step_window, rel_field_diff

pytestmark = pytest.mark.gpu


def _pair(w, precision=fv.FV_FP64, inflow_u=None):
    o = oracle.Oracle(w, inflow_u=inflow_u)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=precision, inflow_u=[inflow_u] if inflow_u is not None else None)
    s.set_state(q)
    return o, q, s


# 2D plain-mode parity runs both stage kernels: the tiled one after a
# primitive pass (FV_FUSED=0) and the fused one (FV_FUSED=1)
FUSED = pytest.mark.parametrize("fused", ["0", "1"])


def _check_kernel(s, fused):
    assert s.tile()["fused"] == (fused == "1")


@pytest.mark.parametrize("n,bc", [
    ((24, 20), None),
    ((37, 23), None),                                            # ragged tiles in x and y
    ((5, 3), None),                                              # smaller than one tile
    ((70, 9), [[wl.BC_OUTFLOW, wl.BC_OUTFLOW], [wl.BC_REFLECT, wl.BC_REFLECT], [0, 0]]),
    ((33, 17), [[wl.BC_REFLECT, wl.BC_OUTFLOW], [wl.BC_OUTFLOW, wl.BC_REFLECT], [0, 0]]),
    ((40, 1), None),                                             # one cell wide (1D through the 2D path)
])
@FUSED
def test_step_parity_random_state(n, bc, fused, monkeypatch):
    monkeypatch.setenv("FV_FUSED", fused)
    w = wl.random_state(n=n, bc=bc)
    o, q, s = _pair(w)
    dt = 0.3 * o.dt(q, 1.0)
    s.step_dt(dt)
    ref = oracle_step_dt(o, q, dt)
    got = s.get_state()
    _check_kernel(s, fused)
    assert np.all(rel_field_diff(got, ref) < 1e-12), rel_field_diff(got, ref)


@FUSED
def test_step_parity_inflow_disc_2d(fused, monkeypatch):
    """x-low inflow boundary in 2D (Dirichlet u, T, Y inside the disc, a slip
    wall outside it), with a per-cell inflow velocity profile."""
    monkeypatch.setenv("FV_FUSED", fused)
    w = wl.random_state(n=(41, 30), bc=[[wl.BC_INFLOW, wl.BC_OUTFLOW], [wl.BC_REFLECT, wl.BC_REFLECT], [0, 0]])
    ly = w.n[1] * w.dx[1]
    w.inflow = dict(yc=w.lo[1] + 0.4 * ly, zc=0.0, radius=0.3 * ly, T=310.0, Y=[0.7], u0=(40.0, 0.0, 0.0))
    u = np.zeros((3, 1, w.n[1]))
    u[0, 0] = 40.0 + 5.0 * np.sin(np.arange(w.n[1]))
    u[1, 0] = 3.0 * np.cos(np.arange(w.n[1]))
    o, q, s = _pair(w, inflow_u=u)
    dt = 0.3 * o.dt(q, 1.0)
    for _ in range(2):
        s.step_dt(dt)
    ref = oracle_step_dt(o, oracle_step_dt(o, q, dt), dt)
    got = s.get_state()
    _check_kernel(s, fused)
    assert np.all(rel_field_diff(got, ref) < 1e-12), rel_field_diff(got, ref)


@pytest.mark.parametrize("lims", [
    (wl.LIM_VANLEER, wl.LIM_VANALBADA),
    (wl.LIM_MC, wl.LIM_SUPERBEE),
    (wl.LIM_CHAKRAVARTHY, wl.LIM_KOREN),
    (wl.LIM_MINMOD, wl.LIM_MINMOD),
])
@FUSED
def test_step_parity_other_limiter_pairs(lims, fused, monkeypatch):
    """Table 4.2's other limiters (the stage kernels' run-time limiter
    variants; Koren/Minmod has compile-time kernels of its own)."""
    monkeypatch.setenv("FV_FUSED", fused)
    w = wl.random_state(n=(37, 23), lim_vel=lims[0], lim_scalar=lims[1])
    o, q, s = _pair(w)
    dt = 0.3 * o.dt(q, 1.0)
    s.step_dt(dt)
    ref = oracle_step_dt(o, q, dt)
    d = rel_field_diff(s.get_state(), ref)
    _check_kernel(s, fused)
    assert np.all(d < 1e-12), d


def test_cfl_dt_matches_oracle():
    w = wl.random_state(n=(50, 31))
    o, q, s = _pair(w)
    t = s.step(1, 0.4)
    assert t == pytest.approx(o.dt(q, 0.4), rel=1e-13, abs=0)
    ref, _ = o.step(q, 1, 0.4)
    assert np.all(rel_field_diff(s.get_state(), ref) < 1e-12)


@FUSED
def test_advection_128_full_run_fp64(fused, monkeypatch):
    """128^2 water column in air, 200 steps at CFL 0.4 (the full run)."""
    monkeypatch.setenv("FV_FUSED", fused)
    w = wl.advection(n=128, steps=200)
    o, q, s = _pair(w)
    t_gpu = s.step(w.steps, w.cfl)
    ref, t_ref = o.step(q, w.steps, w.cfl)
    got = s.get_state()
    _check_kernel(s, fused)
    d = rel_field_diff(got, ref)
    assert np.all(d < 1e-10), d
    assert t_gpu == pytest.approx(t_ref, rel=1e-12, abs=0)


def test_conservation_and_uniform_pressure_gpu():
    w = wl.random_state(n=(48, 40))
    o, q, s = _pair(w)
    t0 = s.totals()
    s.step(10, 0.4)
    t1 = s.totals()
    scale = np.abs(q).reshape(q.shape[0], -1).sum(axis=1)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale)
    w = wl.advection(n=40)
    o, q, s = _pair(w)
    s.step(40, 0.4)
    W = s.get_state(fv.FV_PRIMITIVE)
    assert np.abs(W[2] / 1e5 - 1).max() < 1e-10
    assert np.abs(W[0] / 50 - 1).max() < 1e-10


def test_batch_case_equals_single_run():
    cases = [wl.random_state(n=(40, 24), seed=1), wl.random_state(n=(17, 33), seed=2),
             wl.random_state(n=(64, 64), seed=3)]
    qs = [oracle.Oracle(c).prim_to_cons(c.primitives()) for c in cases]
    b = fv.Solver(cases)
    for i, q in enumerate(qs):
        b.set_state(q, case=i)
    b.step(3, 0.4)
    for i, c in enumerate(cases):
        s = fv.Solver(c)
        s.set_state(qs[i])
        s.step(3, 0.4)
        assert np.array_equal(s.get_state(), b.get_state(case=i))


def test_shock_bubble_full_size_windows():
    """2048 x 1024 shock-bubble in the launch configuration the benchmark
    times: one GPU step against the oracle on sampled windows (shock front,
    bubble interface, reflective and outflow boundaries, corner)."""
    w = wl.shock_bubble()
    W = w.primitives()
    o = oracle.Oracle(w)
    q = o.prim_to_cons(W)
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(q)
    dt = 0.3 * o.dt(q, 1.0)        # a full-size step (CFL 0.3)
    s.step_dt(dt)
    got = s.get_state()
    nx, ny = w.n[0], w.n[1]
    xs = int(0.3e-3 / w.dx[0])
    xb = int(0.4e-3 / w.dx[0])
    wins = [((xs - 6, 500, 0), (xs + 6, 512, 1)),
            ((xb - 4, ny // 2 - 8, 0), (xb + 12, ny // 2 + 8, 1)),
            ((0, 0, 0), (10, 6, 1)),
            ((nx - 7, ny - 9, 0), (nx, ny, 1)),
            ((1000, 0, 0), (1010, 4, 1))]
    # differences relative to each field's scale over the whole domain
    # (momentum components share the scale of the momentum vector)
    scale = np.abs(q).reshape(q.shape[0], -1).max(axis=1)
    scale[1:3] = np.sqrt(q[1] ** 2 + q[2] ** 2).max()
    moved = []
    for lo, hi in wins:
        ref = oracle_step_window(o, q, dt, lo, hi)
        sl = (slice(None), 0, slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        d = np.abs(got[sl] - ref[sl]).reshape(q.shape[0], -1).max(axis=1) / scale
        assert np.all(d < 1e-10), (lo, d)
        moved.append((np.abs(ref[sl] - q[sl]).reshape(q.shape[0], -1).max(axis=1) / scale).max())
    # the step moved the shock window by far more than the tolerance
    assert moved[0] > 1e-4, moved


def test_nonphysical_state_reported_not_trapped():
    w = wl.random_state(n=(16, 16))
    o, q, s = _pair(w)
    bad = q.copy()
    bad[0, 0, 5, 5] = -1.0
    s.set_state(bad)
    with pytest.raises(fv.FVError) as e:
        s.step(1, 0.4)
    assert e.value.status == fv.FV_ERR_NONPHYSICAL
    # the context stays usable
    s.set_state(q)
    s.step(1, 0.4)
