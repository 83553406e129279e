"""Pins of the FP64 oracle against what the paper and the mathematics fix
(no GPU).  Each test names the passage it checks."""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from paper_2304_00140_gb300 import workloads as wl
from tests import exact_riemann as er

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return rows


def _one_dim(comps, n, lo=0.0, hi=1.0, bc=(wl.BC_OUTFLOW, wl.BC_OUTFLOW), liquid=None, **scheme):
    return wl.Workload(name="1d", ndim=1, n=[n, 1, 1], lo=[lo, 0, 0], hi=[hi, 1, 1],
                       bc=[list(bc), [0, 0], [0, 0]], comps=comps,
                       liquid=len(comps) - 1 if liquid is None else liquid,
                       scheme=wl.default_scheme(**scheme), steps=1, cfl=0.4, init="random")


# ---------------------------------------------------------------- closure
def test_table_4_1_ideal_gas_density():
    """Table 4.1: IG density p/(R T) at p = 1e7 Pa, T = 300 K, R = (gamma-1) cv."""
    for g, R, cv, rho in _gold("table_4_1.txt"):
        w = _one_dim([wl.comp_sg(g, 0.0, R / (g - 1.0)), wl.AIR], 4)
        o = oracle.Oracle(w)
        r, e, c, al = o.forward(1e7, 300.0, [1.0])
        assert abs(r - rho) / rho < 1e-4
        assert abs(R / (g - 1.0) - cv) / cv < 1e-5
        # ideal-gas sound speed sqrt(gamma R T) (App. A.1)
        assert abs(c - math.sqrt(g * R * 300.0)) / c < 1e-13


@pytest.mark.parametrize("comp", [wl.WATER, wl.DODECANE_SG, wl.AIR, wl.CH4_IG])
def test_pure_stiffened_gas_inverse_matches_A11(comp):
    """Eq. A.1.1 for a pure material: p = (gamma-1) rho (e - q) - gamma pinf."""
    w = _one_dim([wl.AIR, comp] if comp is not wl.AIR else [comp, wl.WATER], 4)
    o = oracle.Oracle(w)
    Yt = [0.0] if comp is not wl.AIR else [1.0]
    rng = np.random.default_rng(1)
    g, pi = comp["gamma"], comp["pinf"]
    for _ in range(50):
        p = 10 ** rng.uniform(4, 9)
        T = rng.uniform(200, 1500)
        rho, e, c, al = o.forward(p, T, Yt)
        assert abs(p - ((g - 1.0) * rho * e - g * pi)) <= 1e-9 * (p + g * pi)
        p2, T2 = o.inverse(rho, e, Yt)
        assert abs(p2 - p) <= 1e-10 * (p + pi)
        assert abs(T2 - T) <= 1e-10 * T
        # pure-phase sound speed sqrt(gamma (p + pinf) / rho) (App. A.1)
        assert abs(c - math.sqrt(g * (p + pi) / rho)) <= 1e-13 * c


def test_mixture_roundtrip_and_fractions():
    """Table A.1 / Eq. A.1.2-A.1.5: sum alpha = 1, rho = sum alpha_k rho_k,
    and the inverse of the forward closure returns (p, T)."""
    w = wl.advection(n=8)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(7)
    for _ in range(200):
        p = 10 ** rng.uniform(3.5, 9.5)
        T = rng.uniform(150, 2500)
        Y = rng.uniform(0, 1) ** rng.choice([1, 8, 30])
        rho, e, c, al = o.forward(p, T, [Y])
        assert abs(al.sum() - 1.0) < 1e-14
        # alpha_k rho_k = rho Y_k with rho_k = (p + pinf)/((g-1) cv T)
        for k, comp in enumerate(w.comps):
            rk = (p + comp["pinf"]) / ((comp["gamma"] - 1) * comp["cv"] * T)
            Yk = Y if k == 0 else 1 - Y
            assert abs(al[k] * rk - rho * Yk) <= 1e-13 * rho
        p2, T2 = o.inverse(rho, e, [Y])
        # conditioning of the stiff liquid: |dp| ~ eps (p + pinf)
        assert abs(p2 - p) <= 5e-14 * (p + 3.43e8) * 50
        assert abs(T2 - T) <= 1e-11 * T
        # Wood's mixture sound speed lies below the larger pure-phase value
        assert c <= max(math.sqrt(1.4 * p / (rho * 1.0)), 1e9)


# --------------------------------------------------------------- limiters
def test_limiters_consistency_and_symmetry():
    """Table 4.2: every limiter has f(1) = 1; the symmetric ones satisfy
    f(r)/r = f(1/r)."""
    for lid in range(7):
        assert oracle.limiter(lid, 1.0) == pytest.approx(1.0, abs=1e-15)
    for lid in (wl.LIM_MINMOD, wl.LIM_VANLEER, wl.LIM_VANALBADA, wl.LIM_MC, wl.LIM_SUPERBEE):
        for r in (0.1, 0.3, 0.7, 1.5, 3.0, 9.0):
            assert oracle.limiter(lid, r) / r == pytest.approx(oracle.limiter(lid, 1.0 / r), rel=1e-13)
    # TVD region (Sweby): 0 <= f <= min(2r, 2) for r > 0, f = 0 for r <= 0
    for lid in (wl.LIM_MINMOD, wl.LIM_KOREN, wl.LIM_MC, wl.LIM_SUPERBEE, wl.LIM_VANLEER):
        for r in np.linspace(-3, 6, 91):
            f = oracle.limiter(lid, r)
            assert f >= 0 and f <= max(0.0, min(2 * r, 2.0)) + 1e-15


def _cell_avg(poly, a, b):
    P = np.polyint(poly)
    return (np.polyval(P, b) - np.polyval(P, a)) / (b - a)


def test_koren_third_order_on_quadratics():
    """Sec. 3.3: Koren is 3rd-order accurate on smooth data -- the face value
    of cell averages of a quadratic is exact in the linear branch."""
    rng = np.random.default_rng(3)
    hits = 0
    for _ in range(200):
        poly = rng.normal(size=3)
        x = [_cell_avg(poly, i, i + 1) for i in range(4)]    # cells 1..4 on [0,4]
        dl, dc, dr = x[1] - x[0], x[2] - x[1], x[3] - x[2]
        rl, rr = dc / dl, dc / dr
        if not (0.3 < rl < 2.4 and 0.3 < rr < 2.4):
            continue
        hits += 1
        L, R = oracle.muscl(wl.LIM_KOREN, *x)
        exact = np.polyval(poly, 2.0)
        assert L == pytest.approx(exact, abs=1e-12 * (1 + abs(exact)))
        assert R == pytest.approx(exact, abs=1e-12 * (1 + abs(exact)))
    assert hits > 10


def test_minmod_linear_exact_and_bounded():
    """Sec. 3.3 MUSCL: 2nd order (linear data reconstructed exactly) and
    the face values stay within the neighbouring cell values."""
    for a, b in ((1.0, 0.5), (-2.0, 3.0)):
        x = [a + b * (i + 0.5) for i in range(4)]
        L, R = oracle.muscl(wl.LIM_MINMOD, *x)
        assert L == pytest.approx(a + 2 * b, abs=1e-13) and R == pytest.approx(a + 2 * b, abs=1e-13)
    rng = np.random.default_rng(5)
    for lid in (wl.LIM_MINMOD, wl.LIM_KOREN):
        for _ in range(500):
            x = rng.normal(size=4)
            L, R = oracle.muscl(lid, *x)
            assert min(x[0], x[1], x[2]) - 1e-14 <= L <= max(x[0], x[1], x[2]) + 1e-14
            assert min(x[1], x[2], x[3]) - 1e-14 <= R <= max(x[1], x[2], x[3]) + 1e-14


# ------------------------------------------------------------------ THINC
@pytest.mark.parametrize("beta", [1.6, 2.5])
@pytest.mark.parametrize("m,D,theta", [(0.0, 1.0, 1), (0.2, 0.5, 1), (0.1, 0.7, -1)])
def test_thinc_face_values_of_tanh_profile(beta, m, D, theta):
    """Eq. 3-3 / 3-4 are the exact face values of the tanh profile
    m + D/2 (1 + theta tanh(beta (x - x0))) whose cell average is the centre
    cell's value (x in cell units, the centre cell on [0, 1])."""
    for x0 in (-0.4, 0.1, 0.5, 0.8, 1.3):
        prof = lambda x: m + 0.5 * D * (1.0 + theta * math.tanh(beta * (x - x0)))
        avg = quad(prof, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13)[0]
        lo_v, hi_v = (m, m + D) if theta > 0 else (m + D, m)
        # L state: stencil (lo_v, avg, hi_v) -> value at the right face x = 1
        L, _ = oracle.thinc(beta, 1e-20, lo_v, avg, hi_v, 0.0)
        assert L == pytest.approx(prof(1.0), abs=1e-12)
        # R state: stencil (., lo_v, avg, hi_v) -> value at the left face x = 0
        _, R = oracle.thinc(beta, 1e-20, 0.0, lo_v, avg, hi_v)
        assert R == pytest.approx(prof(0.0), abs=1e-12)


# ------------------------------------------------------------------- flux
def _state(o, nd, u, p, T, Y):
    w = np.zeros(nd + 2 + len(Y))
    w[:nd] = u
    w[nd], w[nd + 1] = p, T
    w[nd + 2:] = Y
    return w


def test_uniform_state_gives_euler_flux():
    """Eq. 3-1 / 3-2 are consistent: a uniform state gives u* = u, p* = p and
    the exact flux u q + (0, p n, p u, 0) of Eq. 2-2."""
    w = wl.advection(n=8)
    o = oracle.Oracle(w)
    for d in (0, 1):
        for u in ((30.0, -12.0), (-45.0, 7.0)):
            Wc = _state(o, 2, u, 2.3e5, 310.0, [0.37])
            F = o.face_flux(d, np.tile(Wc, (4, 1)))
            rho, e, c, al = o.forward(2.3e5, 310.0, [0.37])
            E = e + 0.5 * (u[0] ** 2 + u[1] ** 2)
            un = u[d]
            exact = [rho * un, rho * un * u[0] + (2.3e5 if d == 0 else 0), rho * un * u[1] + (2.3e5 if d == 1 else 0),
                     un * (rho * E + 2.3e5), rho * un * 0.37]
            assert np.allclose(F, exact, rtol=1e-13, atol=1e-9)


def test_flux_mirror_symmetry():
    """Reflecting the stencil (cells 1..4 -> 4..1, u_n -> -u_n) negates the
    odd flux components and keeps the normal momentum flux."""
    w = wl.advection(n=8)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(11)
    for _ in range(100):
        W4 = np.array([_state(o, 2, (rng.normal(0, 40), rng.normal(0, 40)), 1e5 * (1 + 0.3 * rng.random()),
                              300 * (1 + 0.2 * rng.random()), [rng.random() ** 3]) for _ in range(4)])
        F = o.face_flux(0, W4)
        M = W4[::-1].copy()
        M[:, 0] *= -1
        Fm = o.face_flux(0, M)
        sign = np.array([-1, 1, -1, -1, -1])
        assert np.allclose(Fm, sign * F, rtol=1e-12, atol=1e-9 * np.abs(F).max())


# ---------------------------------------------------------------- stages
def test_conservation_periodic():
    """Fully conservative four-equation model (Sec. 2.1, App. B): on a
    periodic domain without surface tension the totals of rho, rho u,
    rho E, rho Y are unchanged up to rounding."""
    w = wl.random_state(n=(20, 14))
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    t0 = o.totals(q)
    q1, _ = o.step(q, 4, 0.4)
    t1 = o.totals(q1)
    scale = np.abs(q).sum(axis=(1, 2, 3))
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale


def test_uniform_pressure_velocity_preserved_across_interface():
    """TDU consistency (Sec. 3.3, Fig. 4.3): an advected stiffened-gas /
    ideal-gas interface keeps uniform p, u and T up to rounding."""
    w = wl.advection(n=24)
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    q1, _ = o.step(q, 30, 0.4)
    W = o.cons_to_prim(q1)
    assert np.abs(W[2] / 1e5 - 1).max() < 1e-10
    assert np.abs(W[0] / 50 - 1).max() < 1e-10 and np.abs(W[1] / 50 - 1).max() < 1e-10
    assert np.abs(W[3] / 300 - 1).max() < 1e-10
    # and the interface actually moved through THINC-eligible cells
    assert np.abs(W[4] - w.primitives()[4]).max() > 0.1


def _riemann_run(n, t_end, left, right, x0=0.5):
    comps = [wl.AIR, wl.WATER]
    w = _one_dim(comps, n)
    o = oracle.Oracle(w)
    x = (np.arange(n) + 0.5) / n
    W = np.zeros((4, 1, 1, n))
    for arr, st in ((x < x0, left), (x >= x0, right)):
        W[0, 0, 0, arr] = st["u"]
        W[1, 0, 0, arr] = st["p"]
        W[2, 0, 0, arr] = st["T"]
        W[3, 0, 0, arr] = st["Y"]
    q = o.prim_to_cons(W)
    t = 0.0
    while t < t_end * (1 - 1e-12):
        dt = min(o.dt(q, 0.4), t_end - t)
        q0 = q.copy()
        qa = o.stage(1, dt, q0, q0)
        qb = o.stage(2, dt, q0, qa)
        qa = o.stage(3, dt, q0, qb)
        q = o.stage(4, dt, q0, qa)
        t += dt
    return w, o, q, x


def test_two_material_riemann_problem_against_exact():
    """1D two-material stiffened-gas shock tube (water at 1e8 Pa | air at
    1e5 Pa, both 300 K, at rest) against its exact solution: the density
    L1 error falls with refinement and is below 1% (relative) at 400 cells;
    the diffuse-interface model differs from the sharp solution only in the
    smeared interface and wave cells."""
    left = dict(u=0.0, p=1e8, T=300.0, Y=0.0)    # water
    right = dict(u=0.0, p=1e5, T=300.0, Y=1.0)   # air
    w0 = _one_dim([wl.AIR, wl.WATER], 4)
    o0 = oracle.Oracle(w0)
    rl = o0.forward(left["p"], left["T"], [0.0])[0]
    rr = o0.forward(right["p"], right["T"], [1.0])[0]
    L = er.Side(rl, 0.0, left["p"], 6.12, 3.43e8)
    R = er.Side(rr, 0.0, right["p"], 1.4, 0.0)
    ps, us = er.solve(L, R)
    t_end = 0.2 / (L.c * 1.3)
    errs = []
    for n in (100, 200, 400):
        w, o, q, x = _riemann_run(n, t_end, left, right)
        rho_ex = np.array([er.sample(L, R, ps, us, (xi - 0.5) / t_end)[0] for xi in x])
        rho = q[0, 0, 0]
        errs.append(np.abs(rho - rho_ex).sum() / np.abs(rho_ex).sum())
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.01, errs


def test_threads_give_the_same_bits():
    """the oracle's cell loops run on several threads: every cell is computed
    on its own and the CFL maximum does not depend on the order, so one
    thread and all threads agree bit for bit (a 3D App. D / CSF case)"""
    w = wl.random_state(n=(12, 10, 9), ndim=3, ncomp=3, iles=1, sigma=5.0,
                        bc=[[wl.BC_OUTFLOW] * 2, [wl.BC_REFLECT] * 2, [wl.BC_PERIODIC] * 2])
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    n0 = oracle.threads()
    try:
        oracle.threads(1)
        a, ta = o.step(q, 2, w.cfl)
        oracle.threads(max(2, n0))
        b, tb = o.step(q, 2, w.cfl)
    finally:
        oracle.threads(n0)
    assert ta == tb and np.array_equal(a, b)


def test_opcount_build_reproduces_the_oracle():
    """the op-counting build (the FP64 roofline's flop count) computes the
    same stage bit for bit and counts a plausible amount of arithmetic"""
    w = wl.shock_bubble(nx=64, ny=32)
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    dt = 0.3 * o.dt(q, 1.0)
    got, stage, box = oracle.opcount_stage(o, 1, dt, q, q)
    assert np.array_equal(got, o.stage(1, dt, q, q))
    per_cell = sum(stage[k] - box[k] for k in ("add", "mul", "div", "sqrt", "minmax", "cmp")) / w.cells
    assert 200 < per_cell < 2000, per_cell


def test_totals_are_compensated_sums():
    """The conservation totals are compensated (Neumaier) sums: fields whose
    values span 32 orders of magnitude and cancel agree with math.fsum's correctly
    rounded total within Neumaier's error bound, where a plain running sum
    loses every small term."""
    w = wl.random_state(n=(20, 14))
    o = oracle.Oracle(w)
    rng = np.random.default_rng(9)
    q = rng.uniform(0.5, 1.5, size=(w.nvar, 1, 14, 20)) * 10.0 ** rng.integers(-16, 1, size=(w.nvar, 1, 14, 20))
    q[:, 0, 0, 0] = 1e16                  # every later term is below its half-ulp
    q[:, 0, -1, -1] = -1e16
    got = o.totals(q)
    for v in range(w.nvar):
        exact = math.fsum(q[v].ravel().tolist())
        # Neumaier's bound: 2 eps |S| + O(n eps^2) sum |x|
        assert abs(got[v] - exact) <= 4.5e-16 * abs(exact) + 1e-12, (got[v], exact)
        plain = float(np.cumsum(q[v].ravel())[-1])     # a running sum, term by term
        assert abs(plain - exact) > 1e-3 * abs(exact)


def test_formation_energy_enters_the_caloric_law():
    """Eq. A.1.1 with a formation energy q != 0: p = (gamma-1) rho (e - q)
    - gamma pinf, and the inverse recovers (p, T) (every workload has
    q = 0, so this is the only place q is exercised)."""
    gas_q = wl.comp_sg(1.4, 0.0, 718.0, q=2.5e5)
    liq_q = wl.comp_sg(6.12, 3.43e8, 1816.0, q=-1.2e6)
    w = _one_dim([gas_q, liq_q], 4)
    o = oracle.Oracle(w)
    for Y, comp in (([1.0], gas_q), ([0.0], liq_q)):
        g, pi, qf = comp["gamma"], comp["pinf"], comp["q"]
        for p, T in ((1e5, 300.0), (4e7, 800.0)):
            rho, e, c, al = o.forward(p, T, Y)
            assert abs(p - ((g - 1.0) * rho * (e - qf) - g * pi)) <= 1e-9 * (p + g * pi)
            p2, T2 = o.inverse(rho, e, Y)
            assert abs(p2 - p) <= 1e-9 * (p + pi) and abs(T2 - T) <= 1e-10 * T
    # a mixture: e is the mass-weighted sum, so q enters with Y_k
    rho, e, _, _ = o.forward(2e5, 350.0, [0.3])
    e0 = 0.3 * o.forward(2e5, 350.0, [1.0])[1] + 0.7 * o.forward(2e5, 350.0, [0.0])[1]
    assert e == pytest.approx(e0, rel=1e-14, abs=0)
    p2, T2 = o.inverse(rho, e, [0.3])
    assert p2 == pytest.approx(2e5, rel=1e-9, abs=0) and T2 == pytest.approx(350.0, rel=1e-10, abs=0)


def _three(ndim=2, n=(7, 5)):
    return wl.Workload(name="three", ndim=ndim, n=[n[0], n[1], 1], lo=[0, 0, 0], hi=[1e-3, 1e-3 * n[1] / n[0], 1.0],
                       bc=[[0, 0]] * 3, comps=[wl.N2_IG, wl.CH4_IG, wl.DODECANE_SG], liquid=2,
                       scheme=wl.default_scheme(), steps=1, cfl=0.4, init="random")


def test_three_component_conversions():
    """Table A.1 with three components: the conserved species are rho Y_k
    for each tracked k (rho the closure's mixture density), and the
    recovery returns every Y_k, u, p and T."""
    w = _three()
    o = oracle.Oracle(w)
    rng = np.random.default_rng(13)
    shape = (1, w.n[1], w.n[0])
    W = np.zeros((w.nvar,) + shape)
    W[0], W[1] = rng.uniform(-50, 50, shape), rng.uniform(-50, 50, shape)
    W[2], W[3] = 10 ** rng.uniform(5, 7, shape), rng.uniform(300, 900, shape)
    Y = rng.dirichlet([1.0, 1.0, 1.0], size=shape)
    W[4], W[5] = Y[..., 0], Y[..., 1]
    q = o.prim_to_cons(W)
    for idx in np.ndindex(shape):
        rho = o.forward(W[(2,) + idx], W[(3,) + idx], [W[(4,) + idx], W[(5,) + idx]])[0]
        assert q[(0,) + idx] == pytest.approx(rho, rel=1e-15, abs=0)
        for k in range(2):
            assert q[(4 + k,) + idx] == pytest.approx(rho * W[(4 + k,) + idx], rel=1e-15, abs=0)
    W2 = o.cons_to_prim(q)
    for v in (0, 1, 4, 5):
        assert np.allclose(W2[v], W[v], rtol=1e-12, atol=1e-14 * np.abs(W[v]).max())
    assert np.allclose(W2[2], W[2], rtol=1e-9, atol=0) and np.allclose(W2[3], W[3], rtol=1e-10, atol=0)


def test_three_component_euler_flux():
    """Eq. 2-2's species fluxes with three components: a uniform state gives
    u_n rho Y_k for each tracked species k."""
    o = oracle.Oracle(_three())
    for d, u in ((0, (30.0, -12.0)), (1, (-45.0, 7.0))):
        Wc = np.array([u[0], u[1], 2.3e6, 410.0, 0.23, 0.61])
        F = o.face_flux(d, np.tile(Wc, (4, 1)))
        rho = o.forward(2.3e6, 410.0, [0.23, 0.61])[0]
        assert F[4] == pytest.approx(rho * u[d] * 0.23, rel=1e-13, abs=0)
        assert F[5] == pytest.approx(rho * u[d] * 0.61, rel=1e-13, abs=0)
