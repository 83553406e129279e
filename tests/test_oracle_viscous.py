"""Pins of the oracle's viscous stress, heat conduction and gravity terms
(Eq. 2-2; mixture viscosity Eq. 2-8) against what the mathematics fixes:

* the residual the viscous terms add (the stage with them on minus the stage
  with them off, on the same state) converges at second order to the
  continuum div(tau), div(u . tau) and div(k_c grad T) of smooth periodic
  fields, differentiated symbolically here (2D and 3D);
* a small-amplitude shear wave decays as exp(-nu k^2 t);
* a uniform state under gravity gains exactly rho g dt of momentum and
  rho |g dt|^2 / 2 of energy in one step (the four stages integrate a
  constant force exactly);
* the step-size rule keeps a diffusion-dominated run stable;
* the mixture properties equal a pure component's wherever only that
  component is present.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl

L = 1e-3
K = 2.0 * math.pi / L
P0, T0 = 1e5, 300.0


def _air_box(ndim, n, mu, kc, mu2=None, kc2=None):
    """periodic box of air and a second ideal gas with air's gamma and cv
    (so at equal p and T its volume fraction equals its mass fraction) but
    its own viscosity mu2 and conductivity kc2"""
    w = wl.Workload(name="visc", ndim=ndim, n=[n, n, n if ndim == 3 else 1], lo=[0, 0, 0],
                    hi=[L, L, L if ndim == 3 else 1.0], bc=[[0, 0]] * 3, comps=[wl.AIR, dict(wl.AIR)],
                    liquid=1, scheme=wl.default_scheme(), steps=1, cfl=0.4, init="random")
    return wl.with_transport(w, mu=[mu, mu if mu2 is None else mu2], kc=[kc, kc if kc2 is None else kc2])


def _fields(ndim, mixed):
    """smooth periodic u, v (, w), T and air mass fraction Y as sympy
    expressions of x, y (, z)"""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    k = sp.Float(K)
    U, dT = 2.0, 5.0
    if ndim == 2:
        u = U * (sp.sin(k * x) * sp.cos(k * y) + 0.5 * sp.sin(k * y))
        v = U * (0.7 * sp.cos(k * x) * sp.sin(k * y) + 0.4 * sp.sin(k * x))
        T = T0 + dT * sp.sin(k * x + k * y)
        Y = 0.5 + 0.4 * sp.cos(k * x - k * y) if mixed else sp.Float(1.0)
        return sp, (x, y), [u, v], T, Y
    u = U * (sp.sin(k * x) * sp.cos(k * z) + 0.5 * sp.sin(k * y))
    v = U * (0.7 * sp.cos(k * x) * sp.sin(k * y) + 0.4 * sp.sin(k * z))
    ww = U * (0.6 * sp.sin(k * y) * sp.cos(k * z) + 0.3 * sp.cos(k * x))
    T = T0 + dT * sp.sin(k * x + k * y + k * z)
    Y = 0.5 + 0.4 * sp.sin(k * x + k * z) * sp.cos(k * y) if mixed else sp.Float(1.0)
    return sp, (x, y, z), [u, v, ww], T, Y


def _continuum_residual(ndim, mu1, kc1, mu2, kc2):
    """symbolic div(tau) (momentum) and div(u . tau + k_c grad T) (energy),
    with the Eq. 2-8 mixture mu = Y mu1 + (1 - Y) mu2 (volume fraction =
    mass fraction here) and k_c mixed the same way"""
    sp, X, u, T, Y = _fields(ndim, mixed=(mu2, kc2) != (mu1, kc1))
    mu = Y * mu1 + (1 - Y) * mu2
    kc = Y * kc1 + (1 - Y) * kc2
    g = [[sp.diff(u[a], X[b]) for b in range(ndim)] for a in range(ndim)]
    div = sum(g[a][a] for a in range(ndim))
    tau = [[mu * (g[a][b] + g[b][a]) - (sp.Rational(2, 3) * mu * div if a == b else 0)
            for b in range(ndim)] for a in range(ndim)]
    mom = [sum(sp.diff(tau[a][b], X[b]) for b in range(ndim)) for a in range(ndim)]
    en = sum(sp.diff(sum(u[a] * tau[a][b] for a in range(ndim)) + kc * sp.diff(T, X[b]), X[b])
             for b in range(ndim))
    f = sp.lambdify(X, mom + [en], "numpy")
    fu = sp.lambdify(X, u + [T, Y], "numpy")
    return f, fu


def _grid(ndim, n):
    c = (np.arange(n) + 0.5) * (L / n)
    if ndim == 2:
        Y, Xg = np.meshgrid(c, c, indexing="ij")
        return (Xg[None], Y[None])
    Z, Y, Xg = np.meshgrid(c, c, c, indexing="ij")
    return (Xg, Y, Z)


def _viscous_residual(ndim, n, mu, kc, mu2=None, kc2=None):
    """(stage residual with viscous terms) - (without), and the continuum one"""
    mu2 = mu if mu2 is None else mu2
    kc2 = kc if kc2 is None else kc2
    f, fu = _continuum_residual(ndim, mu, kc, mu2, kc2)
    G = _grid(ndim, n)
    vals = [np.broadcast_to(np.asarray(a, dtype=float), G[0].shape) for a in fu(*G)]
    w_on = _air_box(ndim, n, mu, kc, mu2, kc2)
    w_off = _air_box(ndim, n, 0.0, 0.0)
    W = np.zeros((w_on.nvar,) + G[0].shape)
    for a in range(ndim):
        W[a] = vals[a]
    W[ndim] = P0
    W[ndim + 1] = vals[ndim]
    W[ndim + 2] = vals[ndim + 1]                       # air mass fraction
    o_on, o_off = oracle.Oracle(w_on), oracle.Oracle(w_off)
    q = o_on.prim_to_cons(W)
    # stage 4 (a = 1) with dt = 1 returns q + R(q)
    R_on = o_on.stage(4, 1.0, q, q) - q
    R_off = o_off.stage(4, 1.0, q, q) - q
    got = R_on - R_off
    exact = [np.broadcast_to(np.asarray(a, dtype=float), G[0].shape) for a in f(*G)]
    return got, exact


def _errors(ndim, n, mu, kc, mu2=None, kc2=None):
    got, exact = _viscous_residual(ndim, n, mu, kc, mu2, kc2)
    # mass and the tracked mass fraction get nothing from these terms
    assert np.abs(got[0]).max() == 0.0 and np.abs(got[ndim + 2:]).max() == 0.0
    errs = []
    for v in range(ndim + 1):
        ex = exact[v]
        scale = np.abs(ex).max()
        errs.append(np.abs(got[1 + v] - ex).max() / scale if scale > 0 else np.abs(got[1 + v]).max())
    return np.array(errs)


@pytest.mark.parametrize("mu,kc", [(2e-3, 0.0), (0.0, 0.5), (2e-3, 0.5)], ids=["stress", "heat", "both"])
def test_viscous_residual_converges_2d(mu, kc):
    e32 = _errors(2, 32, mu, kc)
    e64 = _errors(2, 64, mu, kc)
    live = [0, 1, 2] if mu else [2]                      # heat conduction alone drives no momentum
    assert np.all(e64[live] < 0.01), e64
    assert np.all(e32[live] / e64[live] > 3.5), (e32, e64)   # second order
    if not mu:
        got, _ = _viscous_residual(2, 32, mu, kc)
        assert np.abs(got[1:3]).max() == 0.0


def test_viscous_residual_converges_2d_variable_properties():
    """mu and k_c varying with the composition (Eq. 2-8): face values are
    the two cells' mean, so the residual stays second order"""
    e32 = _errors(2, 32, 2e-3, 0.5, 6e-3, 0.1)
    e64 = _errors(2, 64, 2e-3, 0.5, 6e-3, 0.1)
    assert np.all(e64 < 0.01), e64
    assert np.all(e32 / e64 > 3.5), (e32, e64)


def test_viscous_residual_converges_3d():
    e12 = _errors(3, 12, 2e-3, 0.5, 6e-3, 0.1)
    e24 = _errors(3, 24, 2e-3, 0.5, 6e-3, 0.1)
    assert np.all(e24 < 0.03), e24
    assert np.all(e12 / e24 > 3.5), (e12, e24)


def _shear(mu, n=32, U=1e-3, waves=1):
    w = wl.Workload(name="shear", ndim=2, n=[4, n, 1], lo=[0, 0, 0], hi=[L / 8, L, 1.0],
                    bc=[[0, 0]] * 3, comps=[wl.AIR, wl.WATER], liquid=1, scheme=wl.default_scheme(),
                    steps=1, cfl=0.4, init="random")
    w = wl.with_transport(w, mu=[mu, 1e-3])
    y = (np.arange(n) + 0.5) * (L / n)
    W = np.zeros((w.nvar, 1, n, 4))
    W[0] = (U * np.sin(waves * K * y))[None, :, None]
    W[2], W[3], W[4] = P0, T0, 1.0
    o = oracle.Oracle(w)
    return o, o.prim_to_cons(W), np.sin(waves * K * y)


def test_shear_wave_decay():
    """u = U sin(k y): the amplitude decays as exp(-nu k^2 t) (the inviscid
    flux of this state has zero divergence)"""
    mu = 2e-3
    o, q, s = _shear(mu)
    q1, t = o.step(q, 200, 0.4)
    rho = q[0].mean()
    amp = ((q1[1] / q1[0])[0] * s[:, None]).mean() * 2.0
    expected = 1e-3 * math.exp(-mu / rho * K * K * t)
    assert 1e-3 * 0.85 > amp                             # it decays visibly
    assert abs(amp / expected - 1.0) < 0.003, (amp, expected)


def test_step_size_rule_keeps_diffusion_stable():
    """a viscosity for which the acoustic step alone would be unstable
    (diffusion number ~ 16): the step-size rule keeps every step stable"""
    o, q, s = _shear(0.5)
    amps = []
    for _ in range(10):
        q, _ = o.step(q, 5, 0.4)
        amps.append(np.abs(q[1] / q[0]).max())
    assert np.all(np.isfinite(amps)) and np.all(np.diff(amps) < 0) and amps[-1] < 1e-3


def test_gravity_one_step_exact():
    """uniform mixture at rest under a constant body force: one step adds
    rho g dt of momentum and rho |g dt|^2 / 2 of energy"""
    g = (0.3, -9.81, 0.0)
    w = wl.with_transport(wl.random_state(n=(8, 6)), mu=[0.0, 0.0], gravity=g)
    W = np.zeros((w.nvar, 1, 6, 8))
    W[2], W[3], W[4] = 2e6, 320.0, 0.4
    o = oracle.Oracle(w)
    q = o.prim_to_cons(W)
    dt = 0.1
    from tests.helpers import oracle_step_dt
    q1 = oracle_step_dt(o, q, dt)
    rho = q[0]
    assert np.array_equal(q1[0], q[0]) and np.array_equal(q1[4], q[4])
    for a in range(2):
        np.testing.assert_allclose(q1[1 + a], rho * g[a] * dt, rtol=1e-12)
    dE = q1[3] - q[3]
    np.testing.assert_allclose(dE, 0.5 * rho * (g[0] ** 2 + g[1] ** 2) * dt * dt, rtol=1e-8)


def test_gravity_residual_of_stage_one():
    """the first stage's residual of a moving uniform state is rho g and
    rho u . g"""
    g = (0.0, -0.98, 0.0)
    w = wl.with_transport(wl.random_state(n=(8, 6)), mu=[0.0, 0.0], gravity=g)
    W = np.zeros((w.nvar, 1, 6, 8))
    W[0], W[1] = 3.0, -4.0
    W[2], W[3], W[4] = 2e6, 320.0, 0.4
    o = oracle.Oracle(w)
    q = o.prim_to_cons(W)
    R = (o.stage(4, 1.0, q, q) - q)
    np.testing.assert_allclose(R[2], q[0] * g[1], rtol=1e-9)
    np.testing.assert_allclose(R[3], q[0] * (-4.0) * g[1], rtol=1e-9)
    assert np.abs(R[1]).max() < 1e-9 * np.abs(q[1]).max()


def test_mixture_transport_pure_components():
    """Eq. 2-8: pure air cells carry the air values, pure water cells the
    water values, interface cells lie between them"""
    w = wl.with_transport(wl.droplet(n=32), mu=[1.8e-5, 1e-3], kc=[0.026, 0.6])
    o = oracle.Oracle(w)
    W = w.primitives()
    W[4] = np.where(W[4] < 1e-3, 0.0, np.where(W[4] > 1 - 1e-3, 1.0, W[4]))
    q = o.prim_to_cons(W)
    tr = o.transport(q)
    pure_air, pure_water = W[4] == 1.0, W[4] == 0.0
    assert pure_air.any() and pure_water.any()
    np.testing.assert_allclose(tr[0][pure_air], 1.8e-5, rtol=1e-12)
    np.testing.assert_allclose(tr[0][pure_water], 1e-3, rtol=1e-12)
    np.testing.assert_allclose(tr[1][pure_water], 0.6, rtol=1e-12)
    assert tr[0].min() >= 1.8e-5 * (1 - 1e-12) and tr[0].max() <= 1e-3 * (1 + 1e-12)


def test_lsrk_amplifies_a_linear_mode_by_the_degree_4_taylor_polynomial():
    """Sec. 3.1's explicit four-stage low-storage scheme (coefficients
    1/4, 1/3, 1/2, 1): on a linear mode with R = lambda q one step multiplies
    the mode by 1 + z + z^2/2 + z^3/6 + z^4/24, z = lambda dt (a different
    order of the coefficients gives another polynomial).  The mode is a small
    shear wave, for which the residual is linear (no convective flux, heating
    of order U^2), four cells per wavelength, so that no other mode of the
    grid has more than twice its decay rate and rounding noise in them stays
    damped at these step sizes."""
    o, q, s = _shear(0.5, U=1e-7, waves=8)
    ku = 2                                            # a row where sin(k y) is near its peak
    R = o.stage(4, 1.0, q, q) - q
    lam = R[1][0, ku, 0] / q[1][0, ku, 0]
    assert lam < 0
    for z in (-0.4, -0.9, -1.3):
        dt = z / lam
        from tests.helpers import oracle_step_dt
        q1 = oracle_step_dt(o, q, dt)
        G = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
        assert abs(q1[1][0, ku, 0] / q[1][0, ku, 0] - G) < 1e-9, (z, q1[1][0, ku, 0] / q[1][0, ku, 0], G)


def _aniso_errors(nx, ny, mu, kc):
    """the 2D residual error on an nx x ny grid of the same periodic box
    (unequal spacings)"""
    f, fu = _continuum_residual(2, mu, kc, mu, kc)
    cx, cy = (np.arange(nx) + 0.5) * (L / nx), (np.arange(ny) + 0.5) * (L / ny)
    Y, Xg = np.meshgrid(cy, cx, indexing="ij")
    G = (Xg[None], Y[None])
    vals = [np.broadcast_to(np.asarray(a, dtype=float), G[0].shape) for a in fu(*G)]
    mk = lambda m, k: wl.with_transport(wl.Workload(
        name="visc", ndim=2, n=[nx, ny, 1], lo=[0, 0, 0], hi=[L, L, 1.0], bc=[[0, 0]] * 3,
        comps=[wl.AIR, dict(wl.AIR)], liquid=1, scheme=wl.default_scheme(), steps=1, cfl=0.4, init="random"),
        mu=[m, m], kc=[k, k])
    w_on, w_off = mk(mu, kc), mk(0.0, 0.0)
    W = np.zeros((w_on.nvar,) + G[0].shape)
    W[0], W[1], W[2], W[3], W[4] = vals[0], vals[1], P0, vals[2], vals[3]
    o_on, o_off = oracle.Oracle(w_on), oracle.Oracle(w_off)
    q = o_on.prim_to_cons(W)
    got = (o_on.stage(4, 1.0, q, q) - q) - (o_off.stage(4, 1.0, q, q) - q)
    exact = [np.broadcast_to(np.asarray(a, dtype=float), G[0].shape) for a in f(*G)]
    return np.array([np.abs(got[1 + v] - exact[v]).max() / max(np.abs(exact[v]).max(), 1e-300) for v in range(3)])


@pytest.mark.parametrize("mu,kc", [(2e-3, 0.0), (0.0, 0.5)], ids=["stress", "heat"])
def test_viscous_residual_converges_on_an_anisotropic_grid(mu, kc):
    """the same second-order convergence with dy = 2 dx: every derivative
    divides by its own direction's spacing"""
    e1 = _aniso_errors(32, 16, mu, kc)
    e2 = _aniso_errors(64, 32, mu, kc)
    live = [0, 1, 2] if mu else [2]
    assert np.all(e2[live] < 0.02), e2
    assert np.all(e1[live] / e2[live] > 3.5), (e1, e2)
