"""Pins of the oracle functions behind readings whose value the paper does
not fix (no GPU): the acoustic/diffusive step limit, the mixture sound
speed, the THINC eligibility test of Sec. 3.4 and the Peng-Robinson mixing
rule of App. A.2.1.  The value
each reading takes is a choice; what is pinned here is that the function
computes that choice, against closed forms and invariants computed without
the oracle's own formula for it."""
import math

import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl

RU = 8.314462618


def _grid(nd, comps, n=(6, 5, 4), hi=(0.6, 0.2, 0.8), mu=None, kc=None):
    w = wl.Workload(name="readings", ndim=nd, n=[n[0], n[1], n[2] if nd == 3 else 1], lo=[0.0, 0.0, 0.0],
                    hi=[hi[0], hi[1], hi[2] if nd == 3 else 1.0], bc=[[wl.BC_PERIODIC] * 2] * 3, comps=comps,
                    liquid=1, scheme=wl.default_scheme(), steps=1, cfl=0.4, init="random")
    if mu is not None:
        w = wl.with_transport(w, mu, kc)
    return w


def _sg_sound_speed(comp, p, rho):
    """textbook stiffened-gas sound speed c^2 = gamma (p + pinf)/rho (App. A.1)"""
    return math.sqrt(comp["gamma"] * (p + comp["pinf"]) / rho)


def _sharp_state(w, rng, nd):
    """every cell one pure material (Y exactly 0 or 1), random u, p, T"""
    shape = (w.n[2], w.n[1], w.n[0])
    W = np.zeros((w.nvar,) + shape)
    W[:nd] = rng.uniform(-300.0, 300.0, size=(nd,) + shape)
    W[nd] = 10 ** rng.uniform(4.5, 8.5, size=shape)
    W[nd + 1] = rng.uniform(250.0, 900.0, size=shape)
    W[nd + 2] = (rng.random(shape) < 0.5).astype(float)
    return W


# ------------------------------------------------------------- step limit
@pytest.mark.parametrize("nd", [2, 3])
def test_cfl_step_of_pure_phase_cells(nd):
    """Reading of the acoustic step (the paper names CFL 0.4 and defines no
    step): dt = CFL / max over cells of sum_d (|u_d| + c)/dx_d.  On cells of
    one pure material each the sound speed is the textbook stiffened-gas
    one, sqrt(gamma (p + pinf)/rho), with rho the cell's conserved density;
    the grid's spacings differ per direction and the velocities have both
    signs, so a maximum over directions in place of the sum, a dropped
    |.|, a swapped spacing or the wrong cell fails."""
    comps = [wl.AIR, wl.WATER]
    w = _grid(nd, comps)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(31 + nd)
    for _ in range(4):
        W = _sharp_state(w, rng, nd)
        q = o.prim_to_cons(W)
        smax = 0.0
        for idx in np.ndindex(W.shape[1:]):
            comp = comps[0] if W[(nd + 2,) + idx] == 1.0 else comps[1]
            c = _sg_sound_speed(comp, W[(nd,) + idx], q[(0,) + idx])
            s = sum((abs(W[(d,) + idx]) + c) / w.dx[d] for d in range(nd))
            smax = max(smax, s)
        assert o.dt(q, 0.4) == pytest.approx(0.4 / smax, rel=1e-12, abs=0)
        assert o.dt(q, 0.8) == pytest.approx(0.8 / smax, rel=1e-12, abs=0)


@pytest.mark.parametrize("nd", [2, 3])
@pytest.mark.parametrize("mu,kc", [((2.0e-1, 1.8e-5), (0.0, 0.0)), ((1.0e-3, 1.8e-5), (60.0, 2.6e-2))])
def test_diffusive_step_of_pure_phase_cells(nd, mu, kc):
    """Reading of the diffusive limit (none given): the step's denominator
    gains 2 D sum_d 1/dx_d^2 with D = max(4/3 mu, k_c/cv_min)/rho, cv_min the
    smallest component cv.  On pure cells mu and k_c are the material's own
    (Eq. 2-8 with one volume fraction 1); the second case is conduction-bound
    in the water cells, whose cv is not the smallest and comes first.  The
    spacing is fine enough that the diffusive part outweighs the acoustic one
    in the cell that sets the step."""
    comps = [wl.WATER, wl.AIR]
    w = _grid(nd, comps, hi=(6e-6, 2e-6, 8e-6), mu=list(mu), kc=list(kc))
    o = oracle.Oracle(w)
    rng = np.random.default_rng(7 + nd)
    cvmin = min(c["cv"] for c in comps)
    idx2 = sum(1.0 / w.dx[d] ** 2 for d in range(nd))
    W = _sharp_state(w, rng, nd)
    q = o.prim_to_cons(W)
    smax, share = 0.0, 0.0
    for idx in np.ndindex(W.shape[1:]):
        k = 0 if W[(nd + 2,) + idx] == 1.0 else 1
        rho = q[(0,) + idx]
        c = _sg_sound_speed(comps[k], W[(nd,) + idx], rho)
        acoustic = sum((abs(W[(d,) + idx]) + c) / w.dx[d] for d in range(nd))
        diff = 2.0 * max(4.0 / 3.0 * mu[k], kc[k] / cvmin) / rho * idx2
        if acoustic + diff > smax:
            smax, share = acoustic + diff, diff / (acoustic + diff)
    assert share > 0.5
    assert o.dt(q, 0.4) == pytest.approx(0.4 / smax, rel=1e-12, abs=0)


# ------------------------------------------------- mixture sound speed
@pytest.mark.parametrize("comps", [[wl.AIR, wl.WATER], [wl.N2_IG, wl.CH4_IG, wl.DODECANE_SG]])
def test_wood_sound_speed_of_mixtures(comps):
    """Reading of the mixture sound speed (App. A.1 gives the pure phases
    only): Wood's 1/(rho c^2) = sum_k alpha_k/(rho_k c_k^2), with each pure
    phase's rho_k and c_k taken from the closure at the same (p, T) with that
    phase alone (pinned by the pure-phase tests) and alpha_k = Y_k rho/rho_k,
    rho = 1/sum_k Y_k/rho_k (Table A.1).  A Wood sum weighted by mass
    fractions, or a mixture density from mass-weighted phase densities,
    fails."""
    n = len(comps)
    w = wl.Workload(name="wood", ndim=1, n=[4, 1, 1], lo=[0.0, 0, 0], hi=[1.0, 1, 1],
                    bc=[[wl.BC_OUTFLOW] * 2, [0, 0], [0, 0]], comps=comps, liquid=n - 1,
                    scheme=wl.default_scheme(), steps=1, cfl=0.4, init="random")
    o = oracle.Oracle(w)
    rng = np.random.default_rng(17 + n)
    pure = np.eye(n)
    for _ in range(100):
        p, T = 10 ** rng.uniform(4.0, 8.5), rng.uniform(250.0, 1200.0)
        Yt = list(rng.dirichlet(np.ones(n) * 0.3)[:n - 1])
        Y = np.array(Yt + [1.0 - sum(Yt)])     # the last fraction as the closure forms it
        phase = [o.forward(p, T, list(pure[k][:n - 1])) for k in range(n)]
        rk = np.array([ph[0] for ph in phase])
        ck = np.array([ph[2] for ph in phase])
        rho_mix = 1.0 / np.sum(Y / rk)
        alpha = Y * rho_mix / rk
        c_wood = 1.0 / math.sqrt(rho_mix * np.sum(alpha / (rk * ck * ck)))
        rho, e, c, al = o.forward(p, T, Yt)
        assert rho == pytest.approx(rho_mix, rel=1e-13, abs=0)
        assert np.allclose(al, alpha, rtol=1e-12, atol=0)
        assert c == pytest.approx(c_wood, rel=1e-12, abs=0)


# ----------------------------------------------------- THINC eligibility
EPS = 1e-4


def _one_dim(comps, **scheme):
    return wl.Workload(name="1d", ndim=1, n=[4, 1, 1], lo=[0.0, 0, 0], hi=[1.0, 1, 1],
                       bc=[[wl.BC_OUTFLOW] * 2, [0, 0], [0, 0]], comps=comps, liquid=1,
                       scheme=wl.default_scheme(thinc_eps=EPS, **scheme), steps=1, cfl=0.4, init="random")


def _face_Y(o, xi4, u):
    """mass fraction of the upwind face state: the species flux over the mass
    flux of the face (reading 10: the upwind side's own rho and rho Y)"""
    W4 = np.array([[u, 1.3e5, 310.0, x] for x in xi4])
    F = o.face_flux(0, W4)
    return F[3] / F[0]


def _expect(eligible, xi4, side):
    beta = 1.6
    th = oracle.thinc(beta, 1e-20, *xi4)
    mu = oracle.muscl(wl.LIM_MINMOD, *xi4)
    return (th if eligible else mu)[side], th[side], mu[side]


# (stencil x1..x4, L side eligible, R side eligible); each case puts the
# centre value of one side just inside or just outside (eps, 1 - eps), or
# breaks the monotonicity of that side's three cells
_CASES = [
    ((0.0, EPS * (1 + 1e-3), 0.5, 0.9), True, True),
    ((0.0, EPS * (1 - 1e-3), 0.5, 0.9), False, True),
    ((0.2, 0.5, 1 - EPS * (1 + 1e-3), 1.0), True, True),
    ((0.2, 0.5, 1 - EPS * (1 - 1e-3), 1.0), True, False),
    ((0.9, 0.6, EPS * (1 + 1e-3), 0.0), True, True),
    ((0.9, 0.6, EPS * (1 - 1e-3), 0.0), True, False),
    ((1.0, 1 - EPS * (1 - 1e-3), 0.3, 0.1), False, True),
    ((0.2, 0.5, 0.3, 0.1), False, True),      # L: peak at x2; R: x2 > x3 > x4
    ((0.1, 0.3, 0.6, 0.4), True, False),      # R: peak at x3
]


@pytest.mark.parametrize("xi4,elig_L,elig_R", _CASES)
def test_thinc_eligibility_thresholds_and_stencil(xi4, elig_L, elig_R):
    """Sec. 3.4: THINC replaces the upwind-biased value of a face side only
    where that side's cell holds eps < xi < 1 - eps, strictly, with xi
    strictly between its two neighbours (for the L state cells i-1, i, i+1;
    for the R state cells i, i+1, i+2).  The face value is read off the
    oracle's flux with the velocity towards the face from each side, and
    compared with the THINC (Eq. 3-3/3-4) and Minmod values of the stencil,
    which differ in every case."""
    o = oracle.Oracle(_one_dim([wl.AIR, wl.WATER]))
    for side, u, elig in ((0, 40.0, elig_L), (1, -40.0, elig_R)):
        want, th, mu = _expect(elig, xi4, side)
        assert abs(th - mu) > 1e-6 * max(abs(th), abs(mu), 1e-12)
        got = _face_Y(o, xi4, u)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-18), (side, got, th, mu)


def test_thinc_off_gives_the_limited_value():
    """With THINC switched off every face side takes the Minmod value."""
    o = oracle.Oracle(_one_dim([wl.AIR, wl.WATER], thinc=0))
    for xi4, _, _ in _CASES:
        for side, u in ((0, 40.0), (1, -40.0)):
            _, _, mu = _expect(False, xi4, side)
            assert _face_Y(o, xi4, u) == pytest.approx(mu, rel=1e-12, abs=1e-18)


# ------------------------------------------------ Peng-Robinson mixture
def _pr_oracle(comps):
    w = wl.Workload(name="pr", ndim=1, n=[4, 1, 1], lo=[0, 0, 0], hi=[1, 1, 1], bc=[[2, 2], [0, 0], [0, 0]],
                    comps=comps, liquid=len(comps) - 1, scheme=wl.default_scheme(), steps=1, cfl=0.4,
                    init="random")
    return oracle.Oracle(w)


def _second_virial(o, T, Y):
    """B = lim_{v -> inf} v (p v/(R T) - 1) from the oracle's pressure at two
    large molar volumes (Richardson on the 1/v term)"""
    def Bv(v):
        return v * (o.pr_state(T, v, Y)["p"] * v / (RU * T) - 1.0)
    v = 20.0
    return 2.0 * Bv(2.0 * v) - Bv(v)


def _mass_fraction(X, M1, M2):
    return X * M1 / (X * M1 + (1.0 - X) * M2)


def _pure_ab(comp, T):
    """textbook Peng-Robinson constants of one substance at T"""
    Tc, pc, w = comp["Tc"], comp["pc"], comp["omega"]
    cc = 0.37464 + 1.5422 * w - 0.26992 * w * w
    a = 0.457236 * (RU * Tc) ** 2 / pc * (1.0 + cc * (1.0 - math.sqrt(T / Tc))) ** 2
    b = 0.077796 * RU * Tc / pc
    return a, b


@pytest.mark.parametrize("T", [400.0, 900.0])
def test_pr_mixture_second_virial(T):
    """The second virial coefficient of a mixture is a quadratic form in the
    mole fractions, B = sum_ij X_i X_j B_ij (statistical mechanics: it counts
    pairs), and a cubic equation of state gives B = b - a/(R T).  Read off the
    oracle's pressure at low density:
      - B(X) is quadratic in the mole fraction X of N2 (a mixing done in mass
        fractions, or mole fractions not normalised, is not);
      - the pure ends are the textbook PR values b_i - a_i/(R T);
      - the cross coefficient is App. A.2.1's combining rule with k = 0 and
        the reading Zc = 0.3074, vc = Zc R Tc/pc for both species:
        Tc_12 = sqrt(Tc_1 Tc_2), vc_12 = ((vc_1^(1/3) + vc_2^(1/3))/2)^3,
        pc_12 = Zc R Tc_12/vc_12, omega_12 the mean, b_12 the mean of b_i;
      - listing the species in the other order changes nothing."""
    N2, C12 = wl.N2_PR, wl.DODECANE_PR
    o = _pr_oracle([N2, C12])
    M1, M2 = N2["M"], C12["M"]
    Xs = np.array([0.0, 0.15, 0.4, 0.5, 0.7, 0.85, 1.0])
    B = np.array([_second_virial(o, T, [_mass_fraction(X, M1, M2)]) for X in Xs])
    scale = np.abs(B).max()
    coef = np.polyfit(Xs, B, 2)
    assert np.abs(np.polyval(coef, Xs) - B).max() < 1e-9 * scale
    # as a function of the mass fraction the same values are far from quadratic
    Ys = np.array([_mass_fraction(X, M1, M2) for X in Xs])
    assert np.abs(np.polyval(np.polyfit(Ys, B, 2), Ys) - B).max() > 1e-3 * scale
    (a1, b1), (a2, b2) = _pure_ab(N2, T), _pure_ab(C12, T)
    B11, B22 = b1 - a1 / (RU * T), b2 - a2 / (RU * T)
    # B = b - a/(R T) cancels near the Boyle temperature: tolerances are
    # relative to the largest |B|
    assert B[-1] == pytest.approx(B11, rel=0, abs=1e-9 * scale)
    assert B[0] == pytest.approx(B22, rel=0, abs=1e-9 * scale)
    B12 = 2.0 * B[3] - 0.5 * (B11 + B22)
    zc = 0.3074
    vc1, vc2 = zc * RU * N2["Tc"] / N2["pc"], zc * RU * C12["Tc"] / C12["pc"]
    Tc12 = math.sqrt(N2["Tc"] * C12["Tc"])
    vc12 = ((vc1 ** (1 / 3) + vc2 ** (1 / 3)) / 2) ** 3
    pc12 = zc * RU * Tc12 / vc12
    a12, _ = _pure_ab(dict(Tc=Tc12, pc=pc12, omega=0.5 * (N2["omega"] + C12["omega"])), T)
    assert B12 == pytest.approx(0.5 * (b1 + b2) - a12 / (RU * T), rel=0, abs=1e-8 * scale)
    o2 = _pr_oracle([C12, N2])
    for X in (0.3, 0.8):
        Y1 = _mass_fraction(X, M1, M2)
        for v in (2e-4, 1e-3):
            assert o2.pr_state(T, v, [1.0 - Y1])["p"] == pytest.approx(o.pr_state(T, v, [Y1])["p"], rel=1e-13, abs=0)


# ------------------------------------------------------ mass fractions
def test_mass_fractions_entering_the_closure_are_clipped():
    """Reading of the mass fractions entering the closure: each tracked one
    is clipped to [0, 1] and the last is 1 minus their sum, clipped too, so
    face states that overshoot by rounding or reconstruction give the
    closure values of the clipped fractions."""
    o = oracle.Oracle(_grid(2, [wl.AIR, wl.WATER]))
    for p, T in ((1e5, 300.0), (3e7, 900.0)):
        for over, clip in (([1.0 + 1e-7], [1.0]), ([-1e-7], [0.0]), ([1.3], [1.0]), ([-0.2], [0.0])):
            a, b = o.forward(p, T, over), o.forward(p, T, clip)
            assert a[:3] == b[:3] and np.array_equal(a[3], b[3])
    o3 = oracle.Oracle(_grid(2, [wl.N2_IG, wl.CH4_IG, wl.DODECANE_SG]))
    for over, clip in (([1.2, -0.1], [1.0, 0.0]), ([0.7, 0.5], [0.7, 0.5])):
        a, b = o3.forward(2e6, 500.0, over), o3.forward(2e6, 500.0, clip)
        assert a[:3] == b[:3]
    # [0.7, 0.5]: the last fraction 1 - 1.2 is clipped to 0 (no negative phase)
    r, _, _, al = o3.forward(2e6, 500.0, [0.7, 0.5])
    assert al[2] == 0.0
    # in a Peng-Robinson mixture every fraction enters the molar mass and the
    # mixing rule: with the last one clipped to 0 its species does not matter
    ch4 = wl.comp_pr(190.56, 4.599e6, 0.011, 1709.0, 0.016043)
    pa = _pr_oracle([wl.N2_PR, wl.N2_PR, wl.DODECANE_PR]).forward(2e6, 500.0, [0.7, 0.5])
    pb = _pr_oracle([wl.N2_PR, wl.N2_PR, ch4]).forward(2e6, 500.0, [0.7, 0.5])
    assert pa[:3] == pb[:3]


# ------------------------------------------ Peng-Robinson root choice
def test_pr_root_of_lowest_gibbs_energy_in_the_three_root_region():
    """Reading of the root choice (the paper is silent): where the PR cubic
    has three real roots above B (pure n-dodecane below its critical
    temperature, pressures around saturation) the TDU takes the root of
    lowest Gibbs departure (numpy's roots of the cubic as an independent
    solver): the liquid root above the saturation pressure, the vapour root
    below it, so that both occur in the sample."""
    C12 = wl.DODECANE_PR
    o = _pr_oracle([wl.N2_PR, C12])
    s2 = math.sqrt(2.0)
    T = 500.0
    picked = set()
    for p in np.geomspace(2e4, 1.5e6, 60):
        st = o.pr_state(T, 1e-3, [0.0])
        A, B = st["a"] * p / (RU * T) ** 2, st["b"] * p / (RU * T)
        roots = np.roots([1.0, -(1 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)])
        real = sorted(r.real for r in roots if abs(r.imag) < 1e-10 and r.real > B)
        if len(real) < 3:
            continue
        g = lambda Z: Z - 1 - math.log(Z - B) - A / (2 * s2 * B) * math.log((Z + (1 + s2) * B) / (Z + (1 - s2) * B))
        Zbest = min(real, key=g)
        rho = o.forward(p, T, [0.0])[0]
        Z = p * (C12["M"] / rho) / (RU * T)
        assert Z == pytest.approx(Zbest, rel=1e-8, abs=0)
        picked.add("liquid" if Zbest == real[0] else "vapour" if Zbest == real[-1] else "middle")
    assert picked == {"liquid", "vapour"}
