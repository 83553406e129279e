"""GPU parity with the FP64 oracle for the barotropic cavitation closure
(Sec. 2.2, Eq. 2-3 ... 2-7) and the liquid-vapour density THINC (Sec. 3.4
Remarks 1-2): gas and vapour bubble collapse near a wall (Sec. 4.9) on
coarse grids, and sheared gas / vapour pockets at uniform pressure in
plain and App. D mode; step size, state I/O of the passive energy slot and
the FP32-mixed form's accuracy.  Tolerance 1e-10 relative per conserved
field (momentum against the momentum vector's scale), the parity bound;
collapses that start at rest are also run as they are, an ill-conditioned
case with its own bound."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl
from tests.helpers import oracle_step_dt, rel_field_diff, rel_l1_vec

pytestmark = pytest.mark.gpu


def _rel(w, got, ref):
    d = rel_field_diff(got, ref)
    mag = np.sqrt((ref[1:1 + w.ndim] ** 2).sum(0)).max()
    if mag > 0:
        for a in range(w.ndim):
            d[1 + a] = np.abs(got[1 + a] - ref[1 + a]).max() / mag
    return d


def _sheared(kind, iles, n=(36, 30)):
    """a gas bubble at the liquid's pressure (kind 'gas') or a collapsing
    vapour pocket (kind 'vapour'), liquid at 2e5 Pa, with shearing
    velocities, periodic.  (Liquid held at the saturation pressure itself is
    avoided: there the branch of Eq. 2-3 / 2-4, and with it the sound speed,
    switches on the last bit of p, which the oracle's bisection and the
    kernels' closed-form root need not share.)"""
    w = wl.bubble_collapse(kind, n=n, p_inf=2e5, iles=iles)
    w.bc = [[wl.BC_PERIODIC] * 2] * 3
    W = w.primitives()
    x, y, _ = w.centres()
    Y, X = np.meshgrid(y, x, indexing="ij")
    W[0] = 3.0 * np.sin(2 * np.pi * Y[None] / (w.hi[1] - w.lo[1]))
    W[1] = 2.0 * np.cos(2 * np.pi * X[None] / (w.hi[0] - w.lo[0]))
    W[3] = 1e3 * np.sin(2 * np.pi * X[None] / (w.hi[0] - w.lo[0]))     # passive internal energy
    if kind == "gas":
        W[2] = 2e5
    return w, W


CASES = {
    "gas_collapse": lambda: (lambda w: (w, w.primitives()))(wl.bubble_collapse("gas", n=(40, 36))),
    "vapour_collapse": lambda: (lambda w: (w, w.primitives()))(wl.bubble_collapse("vapour", n=(37, 41))),
    "gas_sheared_plain": lambda: _sheared("gas", 0),
    "gas_sheared_iles": lambda: _sheared("gas", 1),
    "vapour_sheared_plain": lambda: _sheared("vapour", 0),
    "vapour_sheared_iles": lambda: _sheared("vapour", 1),
    "vapour_other_limiters": lambda: (lambda w: (w, w.primitives()))(
        wl.bubble_collapse("vapour", n=(33, 29), lim_vel=wl.LIM_VANLEER, lim_scalar=wl.LIM_MC)),
    "gas_collapse_3d": lambda: (lambda w: (w, w.primitives()))(wl.bubble_collapse3d("gas", n=(20, 18, 16))),
    "two_gases_collapse_3d": lambda: (lambda w: (w, w.primitives()))(
        wl.bubble_collapse3d("gas", n=(21, 17, 18), gases=2)),
    "vapour_collapse_3d": lambda: (lambda w: (w, w.primitives()))(
        wl.bubble_collapse3d("vapour", n=(20, 18, 16), p_inf=2e5)),
    "gas_collapse_3d_iles": lambda: (lambda w: (w, w.primitives()))(
        wl.bubble_collapse3d("gas", n=(20, 18, 16), p_inf=2e4, iles=1)),
}


def _with_flow(w, W, amp=3.0):
    """the same state with a smooth O(3 m/s) velocity field added, so that
    the momentum is no longer the small residual of balanced pressure
    forces"""
    W = W.copy()
    X, Y = np.meshgrid(*w.centres()[:2], indexing="xy")
    Lx, Ly = w.hi[0] - w.lo[0], w.hi[1] - w.lo[1]
    if w.ndim == 2:
        W[0] += amp * np.sin(2 * np.pi * Y / Ly)[None]
        W[1] += 0.8 * amp * np.cos(2 * np.pi * X / Lx)[None]
    else:
        W[0] += amp * np.sin(2 * np.pi * Y / Ly)[None]
        W[1] += 0.8 * amp * np.cos(2 * np.pi * X / Lx)[None]
        W[2] += 0.6 * amp
    return W


AT_REST = [n for n in sorted(CASES) if "collapse" in n]


def _parity(w, W):
    o = oracle.Oracle(w)
    q = o.prim_to_cons(W)
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(q)
    dt = 0.3 * o.dt(q, 1.0)
    ref = q
    pert = q * (1 + 1e-16 * np.random.default_rng(20230401).standard_normal(q.shape))
    for _ in range(3):
        s.step_dt(dt)
        ref = oracle_step_dt(o, ref, dt)
        pert = oracle_step_dt(o, pert, dt)
    assert not s.tile()["fused"]
    return _rel(w, s.get_state(), ref), _rel(w, pert, ref)


@pytest.mark.parametrize("name", sorted(CASES))
def test_baro_parity_fp64(name):
    """well-conditioned states (sheared pockets, and the collapses with an
    O(3 m/s) flow added): 1e-10 per conserved field after three steps"""
    w, W = CASES[name]()
    if name in AT_REST:
        W = _with_flow(w, W)
    d, spread = _parity(w, W)
    print(name, "max rel diff", d.max(), "oracle spread under 1e-16 input noise", spread.max())
    assert np.all(d < 1e-10), (d, spread)


@pytest.mark.parametrize("name", AT_REST)
def test_baro_parity_fp64_collapse_at_rest(name):
    """the ill-conditioned case beside the test above: a collapse that
    starts at rest, whose momentum is the small residual of large pressure
    forces; bound 1e-10, or three times the oracle's own spread under a
    1e-16 relative perturbation of its input where that is larger"""
    w, W = CASES[name]()
    d, spread = _parity(w, W)
    assert np.all(spread < 1e-8), spread
    assert np.all(d < np.maximum(1e-10, 3 * spread)), (d, spread)


def test_baro_cfl_steps_and_time():
    w = wl.bubble_collapse("vapour", n=(48, 48))
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(q)
    s.step(1, w.cfl)
    assert abs(s.diag_scalar(fv.FV_DIAG_DT) / o.dt(q, w.cfl) - 1.0) < 1e-12
    s.step(5, w.cfl)
    ref, t = o.step(q, 6, w.cfl)
    assert abs(s.diag_scalar(fv.FV_DIAG_TIME) / t - 1.0) < 1e-12
    d = _rel(w, s.get_state(), ref)
    assert np.all(d < 1e-11), d


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_baro_primitive_io(precision):
    """primitive input (u, p, e, Y) -> conserved -> primitive: p from the
    barotropic inverse, the energy slot passed through"""
    w, W = _sheared("vapour", 0)
    s = fv.Solver(w, precision=precision)
    s.set_state(W, kind=fv.FV_PRIMITIVE)
    back = s.get_state(fv.FV_PRIMITIVE)
    tol = 1e-12 if precision == fv.FV_FP64 else 1e-7
    # p comes back through rho: one rounding of rho (~1000 kg/m^3) times c_L^2
    p_abs = 4 * wl.WATER_BARO["cl"] ** 2 * 1000.0 * 2.2e-16
    for v in range(W.shape[0]):
        bound = tol * max(np.abs(W[v]).max(), 1.0) + (p_abs if v == w.ndim else 0.0)
        assert np.abs(back[v] - W[v]).max() <= bound, v
    ref = oracle.Oracle(w).prim_to_cons(W)
    assert np.all(rel_field_diff(s.get_state(), ref) < 1e-13)


def test_baro_mixed_accuracy_gas_collapse():
    """FP32-mixed gas bubble collapse against the FP64 oracle after 30 CFL
    steps: relative L1 per conserved field"""
    w = wl.bubble_collapse("gas", n=(64, 64))
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_MIXED)
    s.set_state(q)
    s.step(30, w.cfl)
    ref, _ = o.step(q, 30, w.cfl)
    e = rel_l1_vec(s.get_state(), ref, w.ndim)
    print("mixed gas collapse L1", e)
    assert np.all(e < 1e-5), e


def test_baro_rejections():
    w = wl.bubble_collapse("gas", n=(16, 16))
    for bad in (wl.with_transport(w, mu=[1e-5, 1e-3]), w.__class__(**dict(w.__dict__, scheme=dict(w.scheme, sigma=0.07)))):
        with pytest.raises(fv.FVError) as ei:
            fv.Solver(bad, precision=fv.FV_FP64)
        assert ei.value.status == fv.FV_ERR_ARG


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_vapour_collapse_long_run(precision):
    """the 1000 x 1000 vapour collapse (4 um cells) runs 500 CFL steps in
    both forms without a non-physical state (the liquid-vapour THINC stays
    off where the density is not monotone, reading of Remark 1); mass is
    conserved up to the outflow through the open sides"""
    w = wl.bubble_collapse("vapour", n=(1000, 1000))
    s = fv.Solver(w, precision=precision)
    s.set_state(w.primitives(), kind=fv.FV_PRIMITIVE)
    s.step(500, w.cfl)
    q = s.get_state()
    assert np.all(np.isfinite(q)) and q[0].min() > 0


def test_vapour_collapse_full_size_windows():
    """the 1000 x 1000 vapour collapse in the configuration the benchmark
    times: one GPU step (FP64) against the oracle on windows at the top and
    the bottom of the bubble, at the wall and at an outflow corner"""
    from tests.helpers import oracle_step_window
    w = wl.bubble_collapse("vapour", n=(1000, 1000))
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_FP64)
    s.set_state(q)
    dt = 0.4 * 4e-6 / (2 * 1460.0)
    s.step_dt(dt)
    got = s.get_state()
    nx, ny = w.n[0], w.n[1]
    jt = int((440e-6 + 400e-6) / w.dx[1])           # top of the bubble
    jb = int((440e-6 - 400e-6) / w.dx[1])           # bottom, 10 cells above the wall
    wins = [((nx // 2 - 8, jt - 8, 0), (nx // 2 + 8, jt + 8, 1)),
            ((nx // 2 - 8, max(jb - 6, 0), 0), (nx // 2 + 8, jb + 8, 1)),
            ((nx // 2 + 60, 0, 0), (nx // 2 + 76, 6, 1)),
            ((nx - 7, ny - 9, 0), (nx, ny, 1))]
    scale = np.abs(got).reshape(q.shape[0], -1).max(axis=1)
    scale[1:3] = np.sqrt(got[1] ** 2 + got[2] ** 2).max()
    scale[4] = 1.0                                   # no gas anywhere
    tol = np.full(q.shape[0], 1e-11)
    for lo, hi in wins:
        ref = oracle_step_window(o, q, dt, lo, hi)
        sl = (slice(None), 0, slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        d = np.abs(got[sl] - ref[sl]).reshape(q.shape[0], -1).max(axis=1) / scale
        assert np.all(d < tol), (lo, d)


PLAIN_2D = ["gas_collapse", "vapour_collapse", "gas_sheared_plain", "vapour_sheared_plain", "vapour_other_limiters"]


@pytest.mark.parametrize("name", PLAIN_2D)
def test_baro_fused_matches_tiled_mixed(name, monkeypatch):
    """the fused 2D kernel's barotropic mode (FP32-mixed form) against the
    tiled kernel after its primitive pass: the same formulas in the same
    order, so both agree to rounding over three CFL steps"""
    w, W = CASES[name]()
    q = oracle.Oracle(w).prim_to_cons(W)
    out = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("FV_FUSED", fused)
        s = fv.Solver(w, precision=fv.FV_MIXED)
        s.set_state(q)
        s.step(3, w.cfl)
        assert s.tile()["fused"] == (fused == "1")
        out[fused] = s.get_state()
    d = _rel(w, out["1"], out["0"])
    assert np.all(d < 1e-6), d
