"""Pins of the oracle's App. D switch (Eq. D.1, D.4, D.5, D.6)."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl


def _w(ndim=2, n=(12, 12, 1), **kw):
    return wl.Workload(name="iles", ndim=ndim, n=list(n), lo=[0, 0, 0], hi=[1e-3, 1e-3 * n[1] / n[0], 1e-3],
                       bc=[[0, 0]] * 3, comps=[wl.AIR, wl.WATER], liquid=1,
                       scheme=wl.default_scheme(iles=1, **kw), steps=1, cfl=0.4, init="random")


def _uniform_prims(w, u=(0.0, 0.0, 0.0), p=1e6, T=300.0, Y=1.0):
    shape = (w.n[2], w.n[1], w.n[0])
    W = np.zeros((w.nvar,) + shape)
    for d in range(w.ndim):
        W[d] = u[d]
    W[w.ndim], W[w.ndim + 1], W[w.ndim + 2] = p, T, Y
    return W


def test_ducros_sensor_dilatation_vs_rotation():
    """theta^D = (div u)^2 / ((div u)^2 + |curl u|^2 + eps): 1 for pure
    dilatation, 0 for pure rotation and for uniform flow (Eq. D.4)."""
    w = _w(n=(16, 16, 1))
    o = oracle.Oracle(w)
    x = (np.arange(16) + 0.5) / 16 - 0.5
    Y, X = np.meshgrid(x, x, indexing="ij")
    for (ux, uy, expect) in ((X, Y, 1.0), (-Y, X, 0.0), (0 * X + 3.0, 0 * X, 0.0)):
        W = _uniform_prims(w)
        W[0, 0], W[1, 0] = 40 * ux, 40 * uy
        f = o.sensor(o.prim_to_cons(W))
        assert np.all(f[0, 3:-3, 3:-3] == expect)


def test_gas_variation_sensor():
    """theta^Gas > 0.4 at a sharp gas/liquid step (Eq. D.4)."""
    w = _w(n=(16, 8, 1))
    o = oracle.Oracle(w)
    W = _uniform_prims(w)
    W[2 + 2, 0, :, 8:] = 0.0           # liquid on the right half
    f = o.sensor(o.prim_to_cons(W))
    assert np.all(f[0, :, 7:9] == 1.0) and np.all(f[0, :, 2:5] == 0.0)


def test_central_face_value_fourth_order():
    """Eq. D.1: (7(u_i + u_{i+1}) - u_{i-1} - u_{i+2})/12 is exact for cell
    averages of cubics; with uniform p the smooth-branch u* is that value."""
    w = _w()
    o = oracle.Oracle(w)
    rng = np.random.default_rng(2)
    for _ in range(20):
        poly = rng.normal(size=4) * 10
        P = np.polyint(poly)
        avg = [(np.polyval(P, i + 1) - np.polyval(P, i)) for i in range(4)]
        W4 = np.array([[avg[c], 0.0, 1e6, 300.0, 1.0] for c in range(4)])
        rho, e, c, al = o.forward(1e6, 300.0, [1.0])
        F = o.face_flux(0, W4, rho4=np.full(4, rho), c4=np.full(4, c), f=0)
        assert F[0] / rho == pytest.approx(np.polyval(poly, 2.0), abs=1e-11 * (1 + abs(np.polyval(poly, 2.0))))


def test_smooth_branch_pressure_term_damps_odd_even_mode():
    """READING of Eq. D.5's Delta^3 p sign: for a sawtooth pressure the
    smooth-branch correction has the sign of the upwind branch's p_L - p_R
    term (flow from high to low pressure)."""
    w = _w()
    o = oracle.Oracle(w)
    rho, e, c, al = o.forward(1e6, 300.0, [1.0])
    for s in (1.0, -1.0):
        ps = [1e6 - s * 1e3, 1e6 + s * 1e3, 1e6 - s * 1e3, 1e6 + s * 1e3]
        W4 = np.array([[0.0, 0.0, ps[k], 300.0, 1.0] for k in range(4)])
        F0 = o.face_flux(0, W4, rho4=np.full(4, rho), c4=np.full(4, c), f=0)
        F1 = o.face_flux(0, W4, rho4=np.full(4, rho), c4=np.full(4, c), f=1)
        assert np.sign(F0[0]) == np.sign(F1[0]) == s
