"""Pins of the oracle's barotropic closure (Sec. 2.2, Eq. 2-3 ... 2-7) and of
the liquid-vapour density THINC (Sec. 3.4 Remarks 1-2, Eq. 3-7/3-8):

* single-phase limits reduce to the textbook laws: the linear liquid law of
  Eq. 2-3, the mixture law of Eq. 2-4 with c_M^2 = p_sat / rho_sat,liq, the
  isothermal ideal gas of Eq. 2-5;
* a gas-liquid state satisfies the coupled relation the paper writes after
  Eq. 2-6, rho = sum alpha_k rho_k and sum alpha_k = 1;
* the sound speed equals dp/drho at fixed mass fractions (finite
  differences of the inverse);
* the vapour fraction of Eq. 2-7 at its end points and its cap;
* a periodic run conserves every conserved field;
* the App. D vapour sensor flags a vapour interface at rest and the
  liquid-vapour THINC changes a face only where the vapour fraction is
  eligible.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl

LIQ = wl.WATER_BARO
RT = wl.AIR_BARO["rt"]


def _o(n=(8, 6), **scheme):
    w = wl.bubble_collapse("gas", n=n, **scheme)
    return oracle.Oracle(w), w


def test_pure_liquid_is_the_linear_law():
    o, _ = _o()
    c2 = LIQ["cl"] ** 2
    for rho in (999.7001, 1000.0, 1004.5, 1020.0):
        p, e = o.inverse(rho, 0.0, np.array([0.0]))
        assert e == 0.0
        # tolerance: the rounding of rho - rho_sat,liq, amplified by c_L^2
        assert abs(p - (LIQ["psat"] + c2 * (rho - LIQ["rho_sl"]))) <= 1e-12 * p + 4 * c2 * rho * 2.2e-16
        r, _, c, al = o.forward(p, 0.0, np.array([0.0]))
        assert abs(r / rho - 1) < 1e-14 and abs(c / LIQ["cl"] - 1) < 1e-12 and al[1] == pytest.approx(1.0)


def test_pure_mixture_below_saturation():
    o, _ = _o()
    for rho in (5.0, 100.0, 700.0, 999.0):
        p, _ = o.inverse(rho, 0.0, np.array([0.0]))
        assert abs(p / (LIQ["psat"] * rho / LIQ["rho_sl"]) - 1) < 1e-13
        _, _, c, _ = o.forward(p, 0.0, np.array([0.0]))
        assert abs(c * c / (LIQ["psat"] / LIQ["rho_sl"]) - 1) < 1e-12


def test_pure_gas_is_isothermal_ideal_gas():
    o, _ = _o()
    for rho in (0.01, 0.0357, 1.2, 50.0):
        p, _ = o.inverse(rho, 0.0, np.array([1.0]))
        assert abs(p / (rho * RT) - 1) < 1e-14
        _, _, c, al = o.forward(p, 0.0, np.array([1.0]))
        assert abs(c * c / RT - 1) < 1e-12 and al[0] == pytest.approx(1.0)


@pytest.mark.parametrize("rho,xg", [(500.0, 1e-5), (900.0, 1e-6), (50.0, 1e-5), (1003.0, 1e-7), (2.0, 0.2)])
def test_gas_liquid_state_obeys_the_coupled_relation(rho, xg):
    """the relation after Eq. 2-6: (1 - rho xi_g R T / p)(rho_sat + (p - p_sat)/c^2)
    = (1 - xi_g) rho, with c = c_L above p_sat and c_M below"""
    o, _ = _o()
    p, _ = o.inverse(rho, 0.0, np.array([xg]))
    c2 = LIQ["cl"] ** 2 if p >= LIQ["psat"] else LIQ["psat"] / LIQ["rho_sl"]
    lhs = (1 - rho * xg * RT / p) * (LIQ["rho_sl"] + (p - LIQ["psat"]) / c2)
    assert abs(lhs - (1 - xg) * rho) < 1e-11 * rho
    r, _, _, al = o.forward(p, 0.0, np.array([xg]))
    rho_g = p / RT
    rho_lm = LIQ["rho_sl"] + (p - LIQ["psat"]) / c2
    assert abs(al.sum() - 1) < 1e-13
    assert abs(al[0] * rho_g + al[1] * rho_lm - r) < 1e-12 * r


@pytest.mark.parametrize("rho,xg", [(1002.0, 0.0), (300.0, 0.0), (800.0, 1e-6), (1002.0, 1e-7), (1.0, 0.5)])
def test_sound_speed_is_dp_drho(rho, xg):
    o, _ = _o()
    h = 1e-6 * rho
    pp, _ = o.inverse(rho + h, 0.0, np.array([xg]))
    pm, _ = o.inverse(rho - h, 0.0, np.array([xg]))
    p, _ = o.inverse(rho, 0.0, np.array([xg]))
    _, _, c, _ = o.forward(p, 0.0, np.array([xg]))
    assert abs((pp - pm) / (2 * h) / (c * c) - 1) < 1e-6


def test_density_continuous_at_saturation():
    o, _ = _o()
    ps = LIQ["psat"]
    lo = o.forward(ps * (1 - 1e-12), 0.0, np.array([1e-6]))[0]
    hi = o.forward(ps * (1 + 1e-12), 0.0, np.array([1e-6]))[0]
    assert abs(hi - lo) < 1e-8 * hi


def test_vapour_fraction_eq_2_7():
    o, _ = _o()
    ps, rl, rv = LIQ["psat"], LIQ["rho_sl"], LIQ["rho_sv"]
    assert o.vapour(2 * ps, [0.0, 1.0]) == 0.0
    assert o.vapour(ps, [0.0, 1.0]) == 0.0
    # half-way density of the mixture branch rho_M = rho_sl p / p_sat
    pm = ps * 0.5 * (rl + rv) / rl
    assert abs(o.vapour(pm, [0.2, 0.8]) - 0.8 * 0.5) < 1e-12
    # the 99.5% cap of the vapour share of the liquid-vapour phase
    assert abs(o.vapour(1e-6, [0.0, 1.0]) - 0.995) < 1e-15
    assert abs(o.vapour(1e-6, [0.3, 0.7]) - 0.7 * 0.995) < 1e-15


@pytest.mark.parametrize("iles", [0, 1])
def test_periodic_run_conserves(iles):
    """a gas bubble in liquid at uniform pressure with shearing velocities,
    periodic box, plain mode and App. D switch: every conserved total is
    constant"""
    w = wl.bubble_collapse("gas", n=(24, 20), p_inf=2e5, iles=iles)
    w.bc = [[wl.BC_PERIODIC] * 2] * 3
    W = w.primitives()
    W[2] = 2e5
    x, y, _ = w.centres()
    Y, X = np.meshgrid(y, x, indexing="ij")
    W[0] = 3.0 * np.sin(2 * np.pi * Y[None] / (w.hi[1] - w.lo[1]))
    W[1] = 2.0 * np.cos(2 * np.pi * X[None] / (w.hi[0] - w.lo[0]))
    o = oracle.Oracle(w)
    q = o.prim_to_cons(W)
    t0 = o.totals(q)
    q1, _ = o.step(q, 10, 0.4)
    t1 = o.totals(q1)
    scale = np.abs(q).reshape(q.shape[0], -1).sum(1)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale


def _vapour_pocket(thr_vap):
    """a vapour pocket at rest in liquid at saturation pressure"""
    w = wl.bubble_collapse("vapour", n=(20, 20), p_inf=1342.0, iles=1, thr_vap=thr_vap)
    w.bc = [[wl.BC_PERIODIC] * 2] * 3
    W = w.primitives()
    W[0] = W[1] = 0.0
    return oracle.Oracle(w), W


def test_vapour_sensor():
    o, W = _vapour_pocket(0.4)
    q = o.prim_to_cons(W)
    f = o.sensor(q)
    assert 0 < f.sum() < f.size                         # the interface cells only
    o2, W2 = _vapour_pocket(1e9)
    assert o2.sensor(o2.prim_to_cons(W2)).sum() == 0   # nothing else fires at rest


def test_liquid_vapour_density_thinc_only_where_eligible():
    o, _ = _o()
    ps, rl = LIQ["psat"], LIQ["rho_sl"]
    # four cells across a liquid-vapour interface: mixture densities and the
    # matching barotropic pressures, at rest
    rho4 = np.array([20.0, 150.0, 700.0, 980.0])
    p4 = ps * rho4 / rl
    W4 = np.zeros((4, 5))
    W4[:, 2] = p4
    W4[:, 3] = 1.0e3
    av4 = np.array([o.vapour(p, [0.0, 1.0]) for p in p4])
    c4 = np.array([o.forward(p, 0.0, np.array([0.0]))[2] for p in p4])
    F_plain = o.face_flux(0, W4, rho4, c4, f=1)
    F_thinc = o.face_flux(0, W4, rho4, c4, f=1, av4=av4)
    assert np.abs(F_thinc - F_plain).max() > 0          # eligible: the face density changes
    av_bad = av4.copy()
    av_bad[1] = av_bad[0]                                # not monotone at cell i or i+1
    av_bad[2] = av_bad[3]
    F_bad = o.face_flux(0, W4, rho4, c4, f=1, av4=av_bad)
    assert np.array_equal(F_bad, F_plain)


def test_liquid_vapour_density_thinc_per_side():
    """the left face state takes the THINC density when cell i (with its
    neighbours i-1, i+1) is eligible, the right one when cell i+1 is"""
    o, _ = _o()
    ps, rl = LIQ["psat"], LIQ["rho_sl"]
    rho4 = np.array([20.0, 150.0, 700.0, 980.0])
    p4 = ps * rho4 / rl
    W4 = np.zeros((4, 5))
    W4[:, 2] = p4
    c4 = np.array([o.forward(p, 0.0, np.array([0.0]))[2] for p in p4])
    av = np.array([o.vapour(p, [0.0, 1.0]) for p in p4])
    F_plain = o.face_flux(0, W4, rho4, c4, f=1)
    left_only = np.array([av[0], av[1], av[2], av[2] + 0.5])   # cell i+1 not monotone
    right_only = np.array([av[2] + 0.5, av[1], av[2], av[3]])              # cell i not monotone
    F_left = o.face_flux(0, W4, rho4, c4, f=1, av4=left_only)
    F_right = o.face_flux(0, W4, rho4, c4, f=1, av4=right_only)
    F_both = o.face_flux(0, W4, rho4, c4, f=1, av4=av)
    assert not np.array_equal(F_left, F_plain) and not np.array_equal(F_right, F_plain)
    assert not np.array_equal(F_left, F_right)
    assert not np.array_equal(F_left, F_both) and not np.array_equal(F_right, F_both)


def test_smooth_branch_internal_energy_is_second_order_central():
    """App. D smooth faces: 4th-order central (Eq. D.1) for u and p, the
    2nd-order mean for the internal energy (the text after Eq. D.4)"""
    w = wl.bubble_collapse("gas", n=(8, 6), iles=1)
    o = oracle.Oracle(w)
    W4 = np.zeros((4, 5))
    W4[:, 0] = 2.0
    W4[:, 2] = 2e6
    W4[:, 3] = np.array([0.0, 1.0, 4.0, 9.0]) * 1e3           # e quadratic along the stencil
    rho = o.forward(2e6, 0.0, np.array([0.0]))[0]
    _, _, c, _ = o.forward(2e6, 0.0, np.array([0.0]))
    F = o.face_flux(0, W4, np.full(4, rho), np.full(4, c), f=0)
    es = (F[3] - 2e6 * 2.0) / F[0] - 0.5 * 2.0 ** 2
    assert abs(es - 2.5e3) < 1e-9 * 2.5e3


def test_density_thinc_needs_monotone_density():
    """vapour fraction monotone at rounding level near its cap while the
    density is not: no THINC (its profile would leave [0, 1] and overflow);
    the face keeps the TDU state"""
    o, _ = _o()
    ps, rl = LIQ["psat"], LIQ["rho_sl"]
    rho4 = np.array([5.0084500000021928, 5.0084500000025729, 5.008450000002199, 5.0084500000023])
    p4 = ps * rho4 / rl
    W4 = np.zeros((4, 5))
    W4[:, 2] = p4
    c4 = np.array([o.forward(p, 0.0, np.array([0.0]))[2] for p in p4])
    av4 = np.array([0.99500000000001865, 0.99499999999999278, 0.99499999999998612, 0.9949999999999])
    F_plain = o.face_flux(0, W4, rho4, c4, f=1)
    F = o.face_flux(0, W4, rho4, c4, f=1, av4=av4)
    assert np.all(np.isfinite(F)) and np.array_equal(F, F_plain)


@pytest.mark.parametrize("xg", [0.0, 1e-6, 1e-3, 0.3])
def test_face_sound_speed_of_an_equilibrium_density(xg):
    """Sec. 3.4 Remark 2: a face state whose density comes from the
    liquid-vapour THINC gets its sound speed from (p, rho, xi).  Where that
    density is the closure's own density at (p, xi), the result is the
    closure's Wood sound speed, on both branches of Eq. 2-3/2-4."""
    o, _ = _o()
    for p in (400.0, 1000.0, 1342.0 * 1.01, 2e3, 1e5, 3e6):
        rho, _, c, _ = o.forward(p, 0.0, np.array([xg]))
        assert o.baro_sound_rho(p, rho, np.array([xg])) == pytest.approx(c, rel=1e-12, abs=0)


def test_vapour_sensor_argument_and_threshold():
    """App. D Eq. D.4's vapour term: theta^alpha of a cell is the sum over
    directions of |alpha_v,i - alpha_v,i-1| + |alpha_v,i+1 - alpha_v,i| with
    alpha_v of Eq. 2-7, and a cell is flagged exactly where one of its three
    arguments exceeds its threshold.  The threshold is set so that some
    cells lie between it and twice it."""
    o, W = _vapour_pocket(0.4)
    q = o.prim_to_cons(W)
    Wp = o.cons_to_prim(q)[:, 0]
    ny, nx = Wp.shape[1:]
    av = np.array([[o.vapour(Wp[2, j, i], o.forward(Wp[2, j, i], Wp[3, j, i], np.array([Wp[4, j, i]]))[3])
                    for i in range(nx)] for j in range(ny)])
    theta = np.zeros_like(av)
    for ax in (0, 1):
        theta += np.abs(av - np.roll(av, 1, axis=ax)) + np.abs(np.roll(av, -1, axis=ax) - av)
    s = o.sensor_args(q)[:, 0]
    assert np.allclose(s[2], theta, rtol=1e-12, atol=1e-15)
    nz = np.sort(theta[theta > 1e-3])
    thr = float(nz[len(nz) // 2]) / 1.5
    assert np.any((theta > thr) & (theta <= 2 * thr))
    o2, _ = _vapour_pocket(thr)
    f = o2.sensor(q)[0]
    s2 = o2.sensor_args(q)[:, 0]
    sch = o2.w.scheme
    want = (s2[0] > sch["thr_ducros"]) | (s2[1] > sch["thr_gas"]) | (s2[2] > thr)
    assert np.array_equal(f == 1.0, want)


def test_liquid_listed_first():
    """The liquid-vapour component is the one named liquid wherever it is
    listed: with the liquid first and the gas second, Eq. 2-7's vapour
    fraction takes the liquid's volume fraction and constants, and the
    face sound speed from (p, rho, xi) is still the closure's Wood speed."""
    w0 = wl.bubble_collapse("gas", n=(8, 6))
    liq, gas = w0.comps[1], w0.comps[0]
    w = dataclasses.replace(w0, comps=[liq, gas], liquid=0)
    o = oracle.Oracle(w)
    ps, rl, rv = LIQ["psat"], LIQ["rho_sl"], LIQ["rho_sv"]
    pm = ps * 0.5 * (rl + rv) / rl
    assert abs(o.vapour(pm, [0.8, 0.2]) - 0.8 * 0.5) < 1e-12
    assert abs(o.vapour(1e-6, [0.7, 0.3]) - 0.7 * 0.995) < 1e-15
    for p in (400.0, 1000.0, 2e3, 1e5):
        for xg in (0.0, 1e-6, 1e-3, 0.3):
            Yt = np.array([1.0 - xg])                     # the liquid is tracked now
            rho, _, c, _ = o.forward(p, 0.0, Yt)
            assert o.baro_sound_rho(p, rho, Yt) == pytest.approx(c, rel=1e-12, abs=0)
