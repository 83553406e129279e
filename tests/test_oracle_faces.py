"""Pins of the oracle's face and switch logic (no GPU): the all-Mach contact
velocity against the exact Riemann solution at small amplitude (Eq. 3-2),
Table 4.2's limiter per variable, the App. D smooth-face values (Eq. D.1 and
the 2nd-order mass fractions), the Ducros sensor on exact linear velocity
fields (Eq. D.4), the face switch as the larger of the two cell flags, the
capillary jump's pressure work (Sec. 3.5) and the curvature cut-off in a
bulk phase.  Face states are read off the oracle's fluxes: the mass flux is
u* rho of the upwind side, its species flux u* rho Y, and with the face
velocity zero on both sides the normal momentum flux is the face pressure."""
import math

import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl
from tests import exact_riemann as er


def _line(comps=(wl.AIR, wl.WATER), ndim=1, n=(4, 1, 1), bc=wl.BC_OUTFLOW, aspect=(1.0, 1.0), **scheme):
    return wl.Workload(name="faces", ndim=ndim, n=list(n), lo=[0.0, 0.0, 0.0],
                       hi=[1e-3, 1e-3 * aspect[0] * n[1] / n[0], 1e-3 * aspect[1] * n[2] / n[0]], bc=[[bc, bc]] * 3,
                       comps=list(comps),
                       liquid=len(comps) - 1, scheme=wl.default_scheme(**scheme), steps=1, cfl=0.4, init="random")


def _cell(u, p, T, Y):
    return [u, p, T, Y]


# ------------------------------------------------------------ Eq. 3-2
@pytest.mark.parametrize("left_liquid", [True, False])
@pytest.mark.parametrize("du,dp", [((1.0, -0.5), 300.0), ((-2.0, 1.5), -800.0), ((0.3, 0.3), 2000.0)])
def test_contact_velocity_is_the_small_amplitude_riemann_solution(left_liquid, du, dp):
    """Eq. 3-2's u* is the contact velocity of the acoustic (linearised)
    Riemann problem, (Z_L u_L + Z_R u_R + p_L - p_R)/(Z_L + Z_R), Z = rho c.
    Against the exact solution of the two-material Riemann problem (water /
    air, stiffened gas / ideal gas; Toro's exact solver with p + pinf) for
    small jumps, the mass flux of a face between two uniform states gives
    u* within the second-order amplitude error.  The impedance ratio is 3600,
    so an impedance attached to the wrong side's velocity fails."""
    o = oracle.Oracle(_line())
    p0, T = 1e5, 300.0
    uL, uR = du
    pL, pR = p0 + dp, p0
    YL, YR = (0.0, 1.0) if left_liquid else (1.0, 0.0)    # Y tracks air
    cL, cR = _cell(uL, pL, T, YL), _cell(uR, pR, T, YR)
    F = o.face_flux(0, np.array([cL, cL, cR, cR]))
    rL, _, sL, _ = o.forward(pL, T, [YL])
    rR, _, sR, _ = o.forward(pR, T, [YR])
    comp = lambda Y: wl.AIR if Y == 1.0 else wl.WATER
    L = er.Side(rL, uL, pL, comp(YL)["gamma"], comp(YL)["pinf"])
    R = er.Side(rR, uR, pR, comp(YR)["gamma"], comp(YR)["pinf"])
    ps, us_exact = er.solve(L, R)
    us = F[0] / (rL if us_exact >= 0 else rR)
    # the second-order error: relative pressure jump on the compliant side
    amp = max(abs(ps - pL) / (pL + L.pi), abs(ps - pR) / (pR + R.pi))
    assert amp < 0.05
    scale = max(abs(uL), abs(uR), abs(dp) / min(rL * sL, rR * sR))
    assert abs(us - us_exact) <= 2.0 * amp * scale + 1e-12 * scale, (us, us_exact)


# --------------------------------------------------------- Table 4.2
def _four(v_idx, vals, base):
    rows = []
    for x in vals:
        r = list(base)
        r[v_idx] = x
        rows.append(r)
    return np.array(rows)


def test_table_4_2_limiter_of_each_variable():
    """Table 4.2 (plain mode): Koren for the velocity, Minmod for p, T and the
    mass fractions; each stencil below gives different Koren and Minmod face
    values, so a limiter attached to the wrong variable fails."""
    o = oracle.Oracle(_line(comps=(wl.AIR, wl.N2_IG), thinc=0))
    K = lambda x: oracle.muscl(wl.LIM_KOREN, *x)
    Mm = lambda x: oracle.muscl(wl.LIM_MINMOD, *x)
    # pressure: no velocity anywhere, so the normal momentum flux is p*
    pv = (1.0e5, 1.3e5, 1.45e5, 2.1e5)
    assert abs(sum(K(pv)) - sum(Mm(pv))) > 1.0
    F = o.face_flux(0, _four(1, pv, _cell(0.0, 0.0, 300.0, 0.4)))
    assert F[1] == pytest.approx(0.5 * sum(Mm(pv)), rel=1e-14, abs=0)
    # velocity: uniform p, T, Y give equal impedances, u* = (u_L + u_R)/2
    uv = (3.0, 10.0, 12.0, 30.0)
    assert abs(sum(K(uv)) - sum(Mm(uv))) > 0.1
    F = o.face_flux(0, _four(0, uv, _cell(0.0, 2e5, 300.0, 0.4)))
    rho = o.forward(2e5, 300.0, [0.4])[0]
    assert F[0] / rho == pytest.approx(0.5 * sum(K(uv)), rel=1e-13, abs=0)
    # temperature and mass fraction: uniform u > 0, the upwind (left) state's
    # rho follows from T_L, and rho Y / rho is Y_L
    Tv = (250.0, 300.0, 320.0, 420.0)
    F = o.face_flux(0, _four(2, Tv, _cell(20.0, 2e5, 0.0, 0.4)))
    assert F[0] / 20.0 == pytest.approx(o.forward(2e5, Mm(Tv)[0], [0.4])[0], rel=1e-13, abs=0)
    assert abs(K(Tv)[0] - Mm(Tv)[0]) > 1.0
    Yv = (0.1, 0.3, 0.35, 0.8)
    F = o.face_flux(0, _four(3, Yv, _cell(20.0, 2e5, 300.0, 0.0)))
    assert F[3] / F[0] == pytest.approx(Mm(Yv)[0], rel=1e-13, abs=0)
    assert abs(K(Yv)[0] - Mm(Yv)[0]) > 1e-3


# ------------------------------------------------------ App. D faces
def _cubic_avgs(rng, lo, hi):
    poly = rng.normal(size=4)
    P = np.polyint(poly)
    a = np.array([np.polyval(P, i + 1) - np.polyval(P, i) for i in range(4)])
    return lo + (hi - lo) * (a - a.min()) / (a.max() - a.min() + 1e-300)


def test_smooth_face_values():
    """App. D smooth faces (f = 0): p and T take Eq. D.1,
    (7 (x_i + x_{i+1}) - x_{i-1} - x_{i+2})/12, the mass fractions the
    2nd-order mean (x_i + x_{i+1})/2 (the text after Eq. D.4)."""
    o = oracle.Oracle(_line(comps=(wl.AIR, wl.N2_IG), iles=1))
    rng = np.random.default_rng(12)
    D1 = lambda x: (7.0 * (x[1] + x[2]) - x[0] - x[3]) / 12.0
    for _ in range(10):
        pv = _cubic_avgs(rng, 1.5e5, 3e5)
        W4 = _four(1, pv, _cell(0.0, 0.0, 300.0, 0.4))
        r4 = np.array([o.forward(p, 300.0, [0.4])[0] for p in pv])
        c4 = np.array([o.forward(p, 300.0, [0.4])[2] for p in pv])
        F = o.face_flux(0, W4, rho4=r4, c4=c4, f=0)
        assert F[1] == pytest.approx(D1(pv), rel=1e-14, abs=0)
        Tv = _cubic_avgs(rng, 250.0, 450.0)
        W4 = _four(2, Tv, _cell(20.0, 2e5, 0.0, 0.4))
        r4 = np.array([o.forward(2e5, T, [0.4])[0] for T in Tv])
        c4 = np.array([o.forward(2e5, T, [0.4])[2] for T in Tv])
        F = o.face_flux(0, W4, rho4=r4, c4=c4, f=0)
        assert F[0] / 20.0 == pytest.approx(o.forward(2e5, D1(Tv), [0.4])[0], rel=1e-13, abs=0)
        Yv = _cubic_avgs(rng, 0.05, 0.95)
        W4 = _four(3, Yv, _cell(20.0, 2e5, 300.0, 0.0))
        r4 = np.array([o.forward(2e5, 300.0, [Y])[0] for Y in Yv])
        c4 = np.array([o.forward(2e5, 300.0, [Y])[2] for Y in Yv])
        F = o.face_flux(0, W4, rho4=r4, c4=c4, f=0)
        assert F[3] / F[0] == pytest.approx(0.5 * (Yv[1] + Yv[2]), rel=1e-13, abs=0)
        assert abs(D1(Yv) - 0.5 * (Yv[1] + Yv[2])) > 1e-4


# ------------------------------------------------------ Ducros sensor
@pytest.mark.parametrize("ndim", [2, 3])
def test_ducros_sensor_of_linear_velocity_fields(ndim):
    """Eq. D.4 on u = u0 + A x: central differences are exact, so every
    interior cell gives div u = tr A, the vorticity the antisymmetric part
    (A_zy - A_yz, A_xz - A_zx, A_yx - A_xy) and theta^D =
    (tr A)^2/((tr A)^2 + |curl u|^2 + eps).  The three spacings differ."""
    n = (8, 7, 6) if ndim == 3 else (8, 7, 1)
    w = _line(ndim=ndim, n=n, aspect=(0.6, 1.7), iles=1)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(40 + ndim)
    x = [(np.arange(n[d]) + 0.5) * w.dx[d] for d in range(3)]
    Z, Yc, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    pos = [X, Yc, Z]
    inner = (slice(1, -1) if ndim == 3 else slice(None), slice(1, -1), slice(1, -1))
    for _ in range(6):
        A = rng.normal(size=(ndim, ndim)) * 2e4
        W = np.zeros((w.nvar,) + Z.shape)
        for a in range(ndim):
            W[a] = rng.normal() * 10 + sum(A[a, b] * pos[b] for b in range(ndim))
        W[ndim], W[ndim + 1], W[ndim + 2] = 2e5, 300.0, 1.0
        s = o.sensor_args(o.prim_to_cons(W))
        div = np.trace(A)
        if ndim == 3:
            curl = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
        else:
            curl = np.array([A[1, 0] - A[0, 1]])
        c2 = float(curl @ curl)
        theta = div * div / (div * div + c2 + w.scheme["eps_ducros"])
        assert np.allclose(s[0][inner], theta, rtol=1e-9, atol=0)
        assert np.allclose(s[3][inner], abs(div), rtol=1e-9, atol=0)
        assert np.allclose(s[4][inner], math.sqrt(c2), rtol=1e-9, atol=0)


# ------------------------------------------------ face switch, assembly
def test_stage_face_switch_is_the_larger_cell_flag():
    """App. D: a face takes the upwind branch (f = 1) where either of its two
    cells is flagged.  The first stage of the oracle equals an assembly of
    its own face fluxes (cell flags from its sensor, f = max of the two,
    cell density and sound speed for the impedances of Eq. D.5) into
    q0 + a_1 dt (-sum_d dF_d/dx_d) on a periodic grid with a water column
    in air (gas-fraction flags at its edges) and a shear flow (Ducros flags
    in part of it)."""
    nx, ny = 12, 8
    w = _line(ndim=2, n=(nx, ny, 1), bc=wl.BC_PERIODIC, iles=1)
    o = oracle.Oracle(w)
    W = np.zeros((w.nvar, 1, ny, nx))
    ii = np.arange(nx)[None, :]
    jj = np.arange(ny)[:, None]
    W[0, 0] = 30.0 + 4.0 * np.sin(2 * np.pi * jj / ny) + 0.0 * ii
    W[1, 0] = 2.0 * np.cos(2 * np.pi * ii / nx) + 0.0 * jj
    W[2, 0] = 2e5 * (1 + 0.01 * np.cos(2 * np.pi * (ii + 2 * jj) / nx))
    W[3, 0] = 300.0
    W[4, 0] = np.where((ii >= 4) & (ii < 8), 0.0, 1.0) + 0.0 * jj
    q = o.prim_to_cons(W)
    flag = o.sensor(q)[0]
    assert 0 < flag.sum() < flag.size
    Wp = o.cons_to_prim(q)[:, 0]
    rho = q[0, 0]
    c = np.array([[o.forward(Wp[2, j, i], Wp[3, j, i], [Wp[4, j, i]])[2] for i in range(nx)] for j in range(ny)])
    dt = 0.3 * o.dt(q, 1.0)
    R = np.zeros((w.nvar, ny, nx))
    mixed_faces = 0
    for d, (n_d, dx) in enumerate(((nx, w.dx[0]), (ny, w.dx[1]))):
        Fd = np.zeros((w.nvar, ny, nx))      # flux through the high face of each cell
        for j in range(ny):
            for i in range(nx):
                cells = [((i + s) % nx, j) if d == 0 else (i, (j + s) % ny) for s in (-1, 0, 1, 2)]
                W4 = np.array([Wp[:, b, a] for a, b in cells])
                r4 = np.array([rho[b, a] for a, b in cells])
                c4 = np.array([c[b, a] for a, b in cells])
                fl, fr = flag[cells[1][1], cells[1][0]], flag[cells[2][1], cells[2][0]]
                mixed_faces += fl != fr
                Fd[:, j, i] = o.face_flux(d, W4, rho4=r4, c4=c4, f=int(max(fl, fr)))
        R -= (Fd - np.roll(Fd, 1, axis=2 - d)) / dx
    assert mixed_faces > 0
    got = o.stage(1, dt, q, q)[:, 0]
    want = q[:, 0] + 0.25 * dt * R
    scale = np.abs(q[:, 0]).reshape(w.nvar, -1).max(axis=1)[:, None, None]
    assert np.all(np.abs(got - want) <= 1e-13 * scale)


# --------------------------------------------------- capillary jump
def test_capillary_jump_pressure_work():
    """Sec. 3.5 capillary jump: each side of the face sees its own pressure,
    p* -/+ J/2, in the normal momentum flux, and that pressure does work at
    the contact velocity u* in the energy flux: the jump parts of the two
    fluxes are (J/2, u* J/2), for any velocities and pressures."""
    w = wl.droplet(n=16, sigma=0.07)
    w.scheme = dict(w.scheme, st_model=1)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(8)
    for _ in range(20):
        kap = rng.uniform(-5e3, 5e3)
        pl, pg = 2e5 + rng.uniform(-500, 500), 2e5
        ul, ug = rng.uniform(-3, 3), rng.uniform(-3, 3)
        liq = [ul, 0.0, pl, 300.0, 0.0]
        gas = [ug, 0.0, pg, 300.0, 1.0]
        F, G = o.face_flux_kappa(0, [liq, liq, gas, gas], kap, kap, [1.0, 0.0])
        J = 0.07 * kap * (0.0 - 1.0)
        assert G[0] == pytest.approx(0.5 * J, rel=1e-14, abs=0)
        us = F[0] / o.forward(pl if F[0] >= 0 else pg, 300.0, [0.0 if F[0] >= 0 else 1.0])[0]
        assert G[1] == pytest.approx(us * G[0], rel=1e-12, abs=1e-12 * abs(G[0]))


# -------------------------------------------------- curvature cut-off
def test_no_curvature_in_a_bulk_phase():
    """Reading of the CSF normal (Sec. 3.5): where the smoothed fraction's
    gradient is at rounding level (|grad alpha~| dx below 1e-5) the normal is
    zero, so a bulk liquid whose fraction carries only 1e-13 noise has zero
    curvature, while a drop in the same grid has curvature of order 1/R."""
    n = 16
    w = wl.droplet(n=n, sigma=0.07)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(3)
    W = w.primitives()
    Wb = W.copy()
    Wb[w.ndim + 2] = rng.uniform(0.0, 1e-13, size=Wb[w.ndim + 2].shape)    # almost pure liquid
    assert np.all(o.curvature(o.prim_to_cons(Wb)) == 0.0)
    kap = o.curvature(o.prim_to_cons(W))
    R = 0.25 * (w.hi[0] - w.lo[0])
    assert np.abs(kap).max() > 0.3 / R


def test_ducros_sensor_keeps_the_papers_epsilon_at_small_gradients():
    """Eq. D.4's eps is the paper's 1e-20 (dimensional, 1/s^2): on a linear
    field whose gradients are of order 1e-3 1/s, theta^D is still
    (tr A)^2/((tr A)^2 + |curl u|^2) to rounding; a larger eps would show."""
    w = _line(ndim=2, n=(8, 7, 1), aspect=(0.6, 1.0), iles=1)
    assert w.scheme["eps_ducros"] == 1e-20
    o = oracle.Oracle(w)
    x = [(np.arange(w.n[d]) + 0.5) * w.dx[d] for d in range(2)]
    Yc, X = np.meshgrid(x[1], x[0], indexing="ij")
    rng = np.random.default_rng(3)
    for _ in range(4):
        A = rng.normal(size=(2, 2)) * 1e-3
        W = np.zeros((w.nvar, 1) + X.shape)
        W[0, 0], W[1, 0] = A[0, 0] * X + A[0, 1] * Yc, A[1, 0] * X + A[1, 1] * Yc
        W[2], W[3], W[4] = 2e5, 300.0, 1.0
        s = o.sensor_args(o.prim_to_cons(W))
        div, curl = np.trace(A), A[1, 0] - A[0, 1]
        theta = div * div / (div * div + curl * curl + 1e-20)
        assert np.allclose(s[0][0, 1:-1, 1:-1], theta, rtol=1e-6, atol=0)


def test_gas_sensor_argument_and_threshold():
    """Eq. D.4's gas term: theta^Gas of a cell is the sum over directions of
    |a_i - a_i-1| + |a_i+1 - a_i| with a = 1 - alpha_liquid the cell's gas
    volume fraction, and a cell is flagged where one of the arguments
    exceeds its threshold.  The threshold is set so that some cells lie
    between it and twice it."""
    n = (24, 20, 1)
    base = _line(ndim=2, n=n, bc=wl.BC_PERIODIC, iles=1)
    o = oracle.Oracle(base)
    x = [(np.arange(n[d]) + 0.5) * base.dx[d] for d in range(2)]
    Yc, X = np.meshgrid(x[1], x[0], indexing="ij")
    r = np.hypot(X - 0.5e-3, Yc - 0.42e-3)
    h = wl.tanh_indicator(r - 0.25e-3, 2.5 * base.dx[0])          # liquid indicator, a wide interface
    W = np.zeros((base.nvar, 1) + X.shape)
    W[2], W[3], W[4] = 2e5, 300.0, 1.0 - h
    q = o.prim_to_cons(W)
    a = np.array([[1.0 - o.forward(2e5, 300.0, [W[4, 0, j, i]])[3][1] for i in range(n[0])] for j in range(n[1])])
    theta = np.zeros_like(a)
    for ax in (0, 1):
        theta += np.abs(a - np.roll(a, 1, axis=ax)) + np.abs(np.roll(a, -1, axis=ax) - a)
    s = o.sensor_args(q)[:, 0]
    assert np.allclose(s[1], theta, rtol=1e-12, atol=1e-15)
    nz = np.sort(theta[theta > 1e-3])
    thr = float(nz[len(nz) // 2]) / 1.5
    assert np.any((theta > thr) & (theta <= 2 * thr))
    o2 = oracle.Oracle(_line(ndim=2, n=n, bc=wl.BC_PERIODIC, iles=1, thr_gas=thr))
    f = o2.sensor(q)[0]
    s2 = o2.sensor_args(q)[:, 0]
    want = (s2[0] > o2.w.scheme["thr_ducros"]) | (s2[1] > thr) | (s2[2] > o2.w.scheme["thr_vap"])
    assert np.array_equal(f == 1.0, want) and want.any() and not want.all()
