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


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("coef", [0.5, 1.0])
def test_odd_even_pressure_mode_follows_linear_theory(ndim, coef):
    """App. D smooth branch (Eq. D.5): in a liquid at rest the pressure mode
    (-1)^(i+j+k) has zero central face pressure and velocity, so it evolves
    only through the Delta^3 p term of u*: each face carries
    u* = 4 coef p'/(rho c) and the pressure equation gives dp'/dt = lambda p'
    with lambda = -8 ndim coef c / dx.  One step of the four-stage scheme
    multiplies the mode by 1 + z + z^2/2 + z^3/6 + z^4/24, z = lambda dt (the
    linear-theory factor the oracle must reproduce).  At CFL 0.4 z = -3.2
    coef: coef = 1 gives a factor 1.83 per step (the explicit step is
    unstable, beyond z = -2.785), coef = 1/2 damps the mode by 0.27."""
    import dataclasses
    n = 8
    w = wl.random_state(n=(n,) * ndim if ndim == 3 else (n, n), ndim=ndim, ncomp=3, iles=1, d3p_coef=coef)
    w = dataclasses.replace(w, comps=[wl.N2_IG, wl.CH4_IG, wl.DODECANE_SG], liquid=2)
    o = oracle.Oracle(w)
    shape = (n,) * 3 if ndim == 3 else (1, n, n)
    sgn = (-1.0) ** np.indices(shape).sum(0)
    W = np.zeros((w.nvar,) + shape)
    W[ndim] = 6e6 + 1.0 * sgn                  # a 1 Pa mode on 6 MPa: linear
    W[ndim + 1] = 363.0                         # pure liquid (tracked gas fractions 0)
    q = o.prim_to_cons(W)
    assert o.sensor(q).max() == 0.0             # the smooth branch everywhere
    dt = o.dt(q, 0.4)
    c = o.forward(6e6, 363.0, [0.0, 0.0])[2]
    z = -8.0 * ndim * coef * c * dt / w.dx[0]
    factor = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    q1, _ = o.step(q, 1, 0.4)
    g = ((o.cons_to_prim(q1)[ndim] - 6e6) * sgn).mean() / (W[ndim] - 6e6)[0].flat[0]
    assert abs(z - (-3.2 * coef)) < 1e-9
    assert abs(g / factor - 1.0) < 1e-5, (g, factor)
