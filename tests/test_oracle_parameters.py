"""Pins that the oracle's scheme parameters reach the arithmetic (no GPU):
each is set away from its default and its closed-form effect checked: the
THINC steepness beta (Eq. 3-3/3-4) and eligibility epsilon, the limiter
pair (Table 4.2), the Ducros threshold and epsilon (Eq. D.4) and the CSF
normal's cut-off."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl


def _one_dim(**scheme):
    return wl.Workload(name="1d", ndim=1, n=[4, 1, 1], lo=[0.0, 0, 0], hi=[1.0, 1, 1],
                       bc=[[wl.BC_OUTFLOW] * 2, [0, 0], [0, 0]], comps=[wl.AIR, wl.WATER], liquid=1,
                       scheme=wl.default_scheme(**scheme), steps=1, cfl=0.4, init="random")


def _face_Y(o, xi4, u=40.0):
    F = o.face_flux(0, np.array([[u, 1.3e5, 310.0, x] for x in xi4]))
    return F[3] / F[0]


def test_thinc_steepness_beta():
    """beta = 2.5 in place of 1.6: the face value is Eq. 3-3's with 2.5"""
    xi4 = (0.05, 0.3, 0.8, 0.9)
    o = oracle.Oracle(_one_dim(beta=2.5))
    want = oracle.thinc(2.5, 1e-20, *xi4)[0]
    assert abs(want - oracle.thinc(1.6, 1e-20, *xi4)[0]) > 1e-3
    assert _face_Y(o, xi4) == pytest.approx(want, rel=1e-12, abs=0)


def test_thinc_eligibility_epsilon():
    """eps = 0.05: a centre value of 0.03 is not eligible (Minmod), 0.07 is"""
    o = oracle.Oracle(_one_dim(thinc_eps=0.05))
    for x2, eligible in ((0.03, False), (0.07, True)):
        xi4 = (0.0, x2, 0.6, 0.9)
        th, mm = oracle.thinc(1.6, 1e-20, *xi4)[0], oracle.muscl(wl.LIM_MINMOD, *xi4)[0]
        assert abs(th - mm) > 1e-4
        assert _face_Y(o, xi4) == pytest.approx(th if eligible else mm, rel=1e-12, abs=0)


def test_limiter_pair():
    """van Leer for the velocity and MC for p, T, Y (Table 4.2) in place of
    Koren and Minmod: the face pressure and velocity follow those two"""
    o = oracle.Oracle(_one_dim(thinc=0, lim_vel=wl.LIM_VANLEER, lim_scalar=wl.LIM_MC))
    pv = (1.0e5, 1.3e5, 1.45e5, 2.1e5)
    F = o.face_flux(0, np.array([[0.0, p, 300.0, 0.4] for p in pv]))
    mc = oracle.muscl(wl.LIM_MC, *pv)
    assert abs(sum(mc) - sum(oracle.muscl(wl.LIM_MINMOD, *pv))) > 1.0
    assert F[1] == pytest.approx(0.5 * sum(mc), rel=1e-14, abs=0)
    uv = (3.0, 10.0, 12.0, 30.0)
    F = o.face_flux(0, np.array([[u, 2e5, 300.0, 0.4] for u in uv]))
    rho = o.forward(2e5, 300.0, [0.4])[0]
    vl = oracle.muscl(wl.LIM_VANLEER, *uv)
    assert abs(sum(vl) - sum(oracle.muscl(wl.LIM_KOREN, *uv))) > 0.05
    assert F[0] / rho == pytest.approx(0.5 * sum(vl), rel=1e-13, abs=0)


def _linear_field(w, A):
    x = [(np.arange(w.n[d]) + 0.5) * w.dx[d] for d in range(2)]
    Yc, X = np.meshgrid(x[1], x[0], indexing="ij")
    W = np.zeros((w.nvar, 1) + X.shape)
    W[0, 0], W[1, 0] = A[0][0] * X + A[0][1] * Yc, A[1][0] * X + A[1][1] * Yc
    W[2], W[3], W[4] = 2e5, 300.0, 1.0
    return W


def _grid2(**scheme):
    return wl.Workload(name="g", ndim=2, n=[8, 7, 1], lo=[0, 0, 0], hi=[1e-3, 0.9e-3, 1.0],
                       bc=[[wl.BC_OUTFLOW] * 2] * 3, comps=[wl.AIR, wl.WATER], liquid=1,
                       scheme=wl.default_scheme(iles=1, **scheme), steps=1, cfl=0.4, init="random")


def test_ducros_threshold():
    """u = A x with (tr A)^2 / ((tr A)^2 + curl^2) = 0.6: no interior cell is
    flagged at the default threshold 0.95 or at 0.7, every one at 0.5"""
    # tr A = 2e4; the antisymmetric part gives curl^2 = (4e8/0.6 - 4e8)
    b = np.sqrt(4e8 / 0.6 - 4e8) / 2
    A = [[1e4, -b], [b, 1e4]]
    for thr, flagged in ((0.95, False), (0.7, False), (0.5, True)):
        w = _grid2(thr_ducros=thr)
        o = oracle.Oracle(w)
        q = o.prim_to_cons(_linear_field(w, A))
        s = o.sensor_args(q)[0, 0, 1:-1, 1:-1]
        assert np.allclose(s, 0.6, rtol=1e-9, atol=0)
        f = o.sensor(q)[0, 1:-1, 1:-1]
        assert np.all(f == (1.0 if flagged else 0.0)), thr


def test_ducros_epsilon():
    """eps = 1e-6 1/s^2 in place of 1e-20: at gradients of 1e-3 1/s theta^D
    is (tr A)^2/((tr A)^2 + curl^2 + 1e-6)"""
    A = [[1e-3, -2e-3], [1e-3, 0.5e-3]]
    div, curl = 1.5e-3, 3e-3
    for eps in (1e-6, 1e-20):
        w = _grid2(eps_ducros=eps)
        o = oracle.Oracle(w)
        s = o.sensor_args(o.prim_to_cons(_linear_field(w, A)))[0, 0, 1:-1, 1:-1]
        assert np.allclose(s, div * div / (div * div + curl * curl + eps), rtol=1e-6, atol=0)


def test_normal_cut_off():
    """the CSF normal's cut-off |grad alpha~| dx < grad_eps: with grad_eps
    above the largest |grad alpha~| dx of a drop (about 1/(4 width)) every
    normal is cut and the curvature is zero; with the default it is not"""
    w = wl.droplet(n=24, sigma=0.07)
    q = oracle.Oracle(w).prim_to_cons(w.primitives())
    assert np.abs(oracle.Oracle(w).curvature(q)).max() > 0
    w2 = wl.droplet(n=24, sigma=0.07, grad_eps=0.5)
    assert np.all(oracle.Oracle(w2).curvature(q) == 0.0)
