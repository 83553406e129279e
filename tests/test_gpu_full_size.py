"""FP64 parity at the full sizes of the workloads the benchmark times, on
outputs the oracle computes window by window (or case by case): the
1024^2 Peng-Robinson shock/droplet, the 1024-case droplet ensemble in one
context, and the 512 x 256^2 jet with its per-cell inflow velocities, App.
D switch and CSF.  (The 2048 x 1024 shock-bubble, the 1000^2 vapour
collapse and the 1024 x 2048 rising bubble have theirs beside their other
parity tests.)  One step from the initial state with the oracle's CFL dt
(scaled by 0.3 where the step size is given).

Tolerance: 1e-10 of each field's scale (the larger of its largest value
before and after the step; the momentum components share the momentum
vector's), plus, for momentum, 1e-13 of (dt / dx_min) max|rho E|.  A state
at rest gains its first momentum as a difference of two face pressures in
one step; the pressure recovered from rho E carries a rounding error of a
few ulp of rho E (of p_inf for the stiffened-gas liquid), so the momentum
of such cells is only defined to about eps (dt / dx) max|rho E| in FP64
(measured: 2e-15 of that figure on the droplet ensemble, against 5e-9 of
the momentum's own 7e-3 kg/m^2 s scale)."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl
from tests.helpers import oracle_step_window

pytestmark = pytest.mark.gpu


def _scale(qs, ndim):
    """per field, the largest |value| over the arrays qs (the momentum
    components: the largest momentum magnitude)"""
    s = np.zeros(qs[0].shape[0])
    for q in qs:
        t = np.abs(q).reshape(q.shape[0], -1).max(axis=1)
        t[1:1 + ndim] = np.sqrt((q[1:1 + ndim] ** 2).sum(0)).max()
        s = np.maximum(s, t)
    return s


def _allowed(w, q, ref, dt, tol=1e-10):
    """the absolute difference each field may show (module docstring)"""
    nd = w.ndim
    a = tol * _scale([q, ref], nd)
    a[1:1 + nd] += 1e-13 * dt / min(w.dx[:nd]) * max(np.abs(q[1 + nd]).max(), np.abs(ref[1 + nd]).max())
    return a


def _windows_match(o, q, got, dt, wins):
    nd = o.w.ndim
    refs, moved = [], []
    for lo, hi in wins:
        ref = oracle_step_window(o, q, dt, lo, hi)
        sl = (slice(None), slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        refs.append((sl, ref[sl].copy()))
    allowed = _allowed(o.w, q, np.concatenate([r.reshape(r.shape[0], -1) for _, r in refs], axis=1)[:, :, None, None], dt)
    scale = _scale([q] + [r for _, r in refs], nd)
    for (lo, _), (sl, ref) in zip(wins, refs):
        d = np.abs(got[sl] - ref).reshape(q.shape[0], -1).max(axis=1)
        assert np.all(d <= allowed), (lo, d / allowed)
        moved.append((np.abs(ref - q[sl]).reshape(q.shape[0], -1).max(axis=1) / scale).max())
    return moved


def test_pr_shock_droplet_full_size_windows():
    w = wl.pr_shock_droplet(n=1024)
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(q)
    dt = 0.3 * o.dt(q, 1.0)
    s.step_dt(dt)
    got = s.get_state()
    n = 1024
    xs = n // 4                                  # the shock
    xd = n // 2 - 128                            # the droplet's left edge
    wins = [((xs - 6, n // 2 - 6, 0), (xs + 6, n // 2 + 6, 1)),
            ((xd - 6, n // 2 - 6, 0), (xd + 6, n // 2 + 6, 1)),
            ((n // 2 - 6, n // 2 + 128 - 6, 0), (n // 2 + 6, n // 2 + 128 + 6, 1)),
            ((n - 6, n - 6, 0), (n, n, 1))]
    moved = _windows_match(o, q, got, dt, wins)
    assert moved[0] > 1e-6, moved


def test_droplet_ensemble_full_size_sampled_cases():
    """all 1024 cases in one context, one CFL step each (per-case dt); the
    first case of every drop size and the last case checked whole against
    the oracle"""
    cases = wl.droplet_ensemble()
    s = fv.Solver(cases, precision=fv.FV_FP64)
    q0 = [oracle.Oracle(c).prim_to_cons(c.primitives()) for c in cases]
    s.set_state_all(np.concatenate([q.ravel() for q in q0]))
    s.step(1, cases[0].cfl)
    sides = [c.n[0] for c in cases]
    pick = sorted({sides.index(side) for side in set(sides)} | {len(cases) - 1})
    for i in pick:
        o = oracle.Oracle(cases[i])
        ref, t = o.step(q0[i], 1, cases[i].cfl)
        assert abs(s.diag_scalar(fv.FV_DIAG_DT, case=i) / t - 1.0) < 1e-12
        got = s.get_state(case=i)
        d = np.abs(got - ref).reshape(ref.shape[0], -1).max(axis=1)
        allowed = _allowed(cases[i], q0[i], ref, t)
        assert np.all(d <= allowed), (i, sides[i], d / allowed)


def test_jet_full_size_windows():
    w = wl.jet3d()                               # 512 x 256 x 256
    inflow = wl.jet_inflow_velocity(w)
    o = oracle.Oracle(w, inflow_u=inflow)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_FP64, inflow_u=[inflow])
    s.set_state(q)
    dt = 0.3 * o.dt(q, 1.0)
    s.step_dt(dt)
    got = s.get_state()
    nx, ny, nz = w.n
    c = ny // 2
    r = int(16 * ny / 256)
    wins = [((0, c - r - 3, c - 4), (6, c + r + 3, c + 4)),          # the nozzle, across the disc edge
            ((0, c + r - 3, c + r - 3), (4, c + r + 3, c + r + 3)),    # the disc rim off the axes
            ((nx // 2 - 4, c - 4, c - 4), (nx // 2 + 4, c + 4, c + 4)),  # gas at rest
            ((nx - 5, ny - 5, nz - 5), (nx, ny, nz))]                 # outflow corner
    moved = _windows_match(o, q, got, dt, wins)
    assert moved[0] > 1e-6, moved
