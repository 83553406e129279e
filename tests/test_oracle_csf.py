"""Pins of the oracle's CSF source (Sec. 2.3, Sec. 3.5, Eq. 3-9/3-10)
against the Laplace pressure jump of a static drop: the momentum balance
grad p = sigma kappa grad(alpha) integrated along a ray from the drop centre
gives p_in - p_out, which must be sigma/R in 2D (Eq. 4-4) and 2 sigma/R in
3D (App. C), with R the equivalent radius of the liquid volume."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl

RHO_WATER = (1e5 + 3.43e8) / (5.12 * 1816.0 * 300.0)   # pure water at 1e5 Pa, 300 K


def _drop(ndim, n, Rcells, sigma=1.0, L=1e-3):
    dx = L / n
    w = wl.Workload(name="drop", ndim=ndim, n=[n, n, n if ndim == 3 else 1], lo=[0, 0, 0],
                    hi=[L, L, L if ndim == 3 else 1.0], bc=[[0, 0]] * 3, comps=[wl.AIR, wl.WATER],
                    liquid=1, scheme=wl.default_scheme(sigma=sigma), steps=1, cfl=0.4, init="random")
    x = (np.arange(n) + 0.5) * dx - 0.5 * L
    if ndim == 3:
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    else:
        Y, X = np.meshgrid(x, x, indexing="ij")
        r = np.sqrt(X ** 2 + Y ** 2)[None]
    h = wl.tanh_indicator(r - Rcells * dx, 1.5 * dx)
    W = np.zeros((w.nvar,) + r.shape)
    W[ndim] = 1e5
    W[ndim + 1] = 300.0
    W[ndim + 2] = 1.0 - h
    o = oracle.Oracle(w)
    q = o.prim_to_cons(W)
    alpha = q[0] * (1.0 - W[ndim + 2]) / RHO_WATER
    return o, q, alpha, dx


def test_laplace_jump_2d():
    n = 96
    o, q, alpha, dx = _drop(2, n, 32)
    S = o.csf_source(q)
    Req = np.sqrt(alpha.sum() * dx * dx / np.pi)
    assert Req / dx > 28
    c = n // 2
    for comp, ray in ((0, S[0, 0, c, c:]), (1, S[1, 0, c:, c])):
        jump = -ray.sum() * dx
        assert jump > 0                                   # p_in > p_out (kappa > 0 for a drop)
        assert abs(jump / (1.0 / Req) - 1.0) < 0.02, jump * Req


def test_laplace_jump_3d():
    n = 64
    o, q, alpha, dx = _drop(3, n, 24)
    S = o.csf_source(q)
    Req = (alpha.sum() * dx ** 3 * 3.0 / (4.0 * np.pi)) ** (1.0 / 3.0)
    c = n // 2
    jump = -S[0, c, c, c:].sum() * dx
    assert abs(jump / (2.0 / Req) - 1.0) < 0.02, jump * Req / 2


def test_csf_energy_source_is_u_dot_force():
    """Eq. 2-2: the energy source is u . f (here with a uniform velocity)."""
    w = wl.droplet(n=40, A=0.15, sigma=0.3)
    W = w.primitives()
    W[0] = 3.0
    W[1] = -2.0
    o = oracle.Oracle(w)
    q = o.prim_to_cons(W)
    S = o.csf_source(q)
    assert np.allclose(S[2], 3.0 * S[0] - 2.0 * S[1], rtol=1e-12, atol=1e-12 * np.abs(S[2]).max())
    # no force without an interface
    W[4] = 1.0
    assert np.abs(o.csf_source(o.prim_to_cons(W))).max() == 0.0


def _gold(name):
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return rows


def test_oscillating_drop_period_eq_4_3():
    """Sec. 4.4: the ellipse of Eq. 4-2 (semi-axes 0.4 mm along x, 0.3 mm
    along y) in the two ideal gases of Table 4.5 at 1e7 Pa and 300 K
    (densities 117.647 and 4.444 kg/m^3), sigma = 80 N/m, oscillates with
    the period of Eq. 4-3, 2 pi sqrt((rho_1 + rho_2) (ab)^{3/2} / (48 sigma))
    with the full axes a = 0.6 mm, b = 0.8 mm (about 2.04e-5 s).  The drop's
    mode-2 symmetry allows a quarter of the paper's 1.58 mm box: walls
    through the centre, the paper's non-reflective sides as zero-gradient
    outflow; 12 x 12 cells of 66 um (the equivalent radius is 5.3 cells), the
    initial liquid fraction the exact area fraction of each cell.  The
    ratio of the second moments of the liquid fraction, sum(alpha y^2) /
    sum(alpha x^2), starts below 1, peaks after half a period and returns to
    its minimum after one period; both times are checked against Eq. 4-3."""
    rho1, rho2, a, b, sigma, _, _, _ = _gold("laplace_4_4.txt")[0]
    T43 = 2 * np.pi * np.sqrt((rho1 + rho2) * (a * b) ** 1.5 / (48 * sigma))
    assert abs(T43 - 2.0e-5) < 0.05 * 2.0e-5                   # the paper's "T about 2e-5 s"
    n, L = 12, 0.79e-3
    gas = wl.comp_sg(5.0, 0.0, 7500.75 / 4.0)                   # Table 4.5 component 1 (ambient)
    liq = wl.comp_sg(1.6, 0.0, 283.33 / 0.6)                    # component 2 (the drop)
    w = wl.Workload(name="osc_drop", ndim=2, n=[n, n, 1], lo=[0, 0, 0], hi=[L, L, 1.0],
                    bc=[[wl.BC_REFLECT, wl.BC_OUTFLOW], [wl.BC_REFLECT, wl.BC_OUTFLOW], [0, 0]],
                    comps=[gas, liq], liquid=1, scheme=wl.default_scheme(sigma=sigma), steps=1, cfl=0.4,
                    init="random")
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    Y, X = np.meshgrid(x, x, indexing="ij")
    sub = (np.arange(8) + 0.5) / 8 - 0.5
    inside = np.zeros_like(X)
    for sa in sub:
        for sb in sub:
            inside += (((X + sa * dx) / (0.5 * b)) ** 2 + ((Y + sb * dx) / (0.5 * a)) ** 2 <= 1.0)
    inside /= 64.0
    W = np.zeros((w.nvar, 1, n, n))
    W[2], W[3], W[4] = 1e7, 300.0, 1.0 - inside
    o = oracle.Oracle(w)
    q = o.prim_to_cons(W)
    assert abs(q[0].max() / rho1 - 1) < 1e-4 and abs(q[0].min() / rho2 - 1) < 1e-4

    def moment_ratio(q):
        Wp = o.cons_to_prim(q)[:, 0]
        alpha = q[0, 0] * (1.0 - Wp[4]) / (Wp[2] / (0.6 * liq["cv"] * Wp[3]))
        return (alpha * Y ** 2).sum() / (alpha * X ** 2).sum()

    ts, rs, t = [0.0], [moment_ratio(q)], 0.0
    while t < 1.15 * T43:
        q, t = o.step(q, 40, w.cfl, t)
        ts.append(t)
        rs.append(moment_ratio(q))
    ts, rs = np.array(ts), np.array(rs)

    def extremum(i):
        c = np.polyfit(ts[i - 2:i + 3], rs[i - 2:i + 3], 2)
        return -c[1] / (2 * c[0])
    imax = int(np.argmax(rs[:np.searchsorted(ts, 0.8 * T43)]))
    j0 = np.searchsorted(ts, 0.75 * T43)
    imin = j0 + int(np.argmin(rs[j0:]))
    assert rs[imax] > 1.5 and rs[0] < 0.6 and imin + 3 <= len(ts)
    t_half, t_full = extremum(imax), extremum(imin)
    print(f"Eq. 4-3 period {T43:.4e} s; measured {t_full:.4e} s, half period {t_half:.4e} s")
    assert abs(t_full / T43 - 1.0) < 0.03, t_full / T43
    assert abs(2 * t_half / T43 - 1.0) < 0.06, 2 * t_half / T43


def test_smoothing_kernel_moments():
    """Eq. 3-9's kernel (1/16 in 2D, 1/64 in 3D: the binomial weights 1, 2, 1
    along each direction) keeps a linear field and adds h_d^2/2 times the
    coefficient of each x_d^2: on alpha = c0 + sum_d (b_d x_d + c_d x_d^2)
    the smoothed fraction of every cell whose neighbours are interior is
    alpha + sum_d c_d h_d^2/2 (a box filter would add 2 h_d^2/3)."""
    rng = np.random.default_rng(21)
    for ndim, n, hi in ((2, (9, 7, 1), (1e-3, 1.4e-3, 1.0)), (3, (7, 6, 8), (1e-3, 0.9e-3, 1.6e-3))):
        w = wl.Workload(name="kernel", ndim=ndim, n=list(n), lo=[0, 0, 0], hi=list(hi),
                        bc=[[wl.BC_OUTFLOW] * 2] * 3, comps=[wl.AIR, wl.WATER], liquid=1,
                        scheme=wl.default_scheme(sigma=0.07), steps=1, cfl=0.4, init="random")
        o = oracle.Oracle(w)
        dx = w.dx
        xs = [(np.arange(n[d]) + 0.5) * dx[d] for d in range(3)]
        Z, Yc, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
        pos = [X, Yc, Z]
        b = rng.uniform(-0.1, 0.1, size=3) / np.array(hi)
        c = rng.uniform(-0.1, 0.1, size=3) / np.array(hi) ** 2
        alpha = 0.5 + sum(b[d] * pos[d] + c[d] * pos[d] ** 2 for d in range(ndim))
        assert 0.05 < alpha.min() and alpha.max() < 0.95
        rho_l = o.forward(1e5, 300.0, [0.0])[0]
        rho_g = o.forward(1e5, 300.0, [1.0])[0]
        Yl = alpha * rho_l / (alpha * rho_l + (1.0 - alpha) * rho_g)
        W = np.zeros((w.nvar,) + alpha.shape)
        W[ndim], W[ndim + 1], W[ndim + 2] = 1e5, 300.0, 1.0 - Yl
        got = o.smoothed_fraction(o.prim_to_cons(W))
        want = alpha + sum(c[d] * dx[d] ** 2 / 2.0 for d in range(ndim))
        inner = (slice(1, -1) if ndim == 3 else slice(None), slice(1, -1), slice(1, -1))
        assert np.allclose(got[inner], want[inner], rtol=0, atol=1e-13)


def test_curvature_of_a_circle_on_an_anisotropic_grid():
    """Sec. 3.5's vertex normals and kappa = -div n on a grid with
    dy = dx/2: the tanh-smoothed circle of radius R = 12 dx has a mean
    curvature 1/R within 2% over the interface band, as on a square grid
    (each direction's differences divide by that direction's spacing)."""
    nx, ny, L = 48, 96, 1e-3
    dx = L / nx
    dy = 0.5 * dx
    w = wl.Workload(name="aniso", ndim=2, n=[nx, ny, 1], lo=[0, 0, 0], hi=[L, ny * dy, 1.0], bc=[[0, 0]] * 3,
                    comps=[wl.AIR, wl.WATER], liquid=1, scheme=wl.default_scheme(sigma=1.0), steps=1, cfl=0.4,
                    init="random")
    o = oracle.Oracle(w)
    x = (np.arange(nx) + 0.5) * dx - 0.5 * L - 0.13 * dx
    y = (np.arange(ny) + 0.5) * dy - 0.5 * ny * dy + 0.21 * dy
    Y, X = np.meshgrid(y, x, indexing="ij")
    R = 12 * dx
    h = wl.tanh_indicator(np.sqrt(X ** 2 + Y ** 2)[None] - R, 1.5 * dx)
    W = np.zeros((w.nvar,) + h.shape)
    W[2], W[3], W[4] = 1e5, 300.0, 1.0 - h
    k = o.curvature(o.prim_to_cons(W))
    band = (h > 0.2) & (h < 0.8)
    assert abs((k[band] * R).mean() - 1.0) < 0.02


@pytest.mark.parametrize("order", ["liquid_first", "liquid_last_of_three"])
def test_laplace_jump_wherever_the_liquid_is_listed(order):
    """The liquid fraction that CSF (and the gas sensor) use is that of the
    component named liquid, whatever its place in the list: water listed
    first of two, or last of three (two gases, as in the jet), gives the
    same Laplace jump sigma/R as the drop above."""
    n, Rc = 96, 32
    dx = 1e-3 / n
    comps = [wl.WATER, wl.AIR] if order == "liquid_first" else [wl.N2_IG, wl.AIR, wl.WATER]
    liquid = 0 if order == "liquid_first" else 2
    w = wl.Workload(name="drop", ndim=2, n=[n, n, 1], lo=[0, 0, 0], hi=[1e-3, 1e-3, 1.0], bc=[[0, 0]] * 3,
                    comps=comps, liquid=liquid, scheme=wl.default_scheme(sigma=1.0), steps=1, cfl=0.4,
                    init="random")
    x = (np.arange(n) + 0.5) * dx - 0.5e-3
    Y, X = np.meshgrid(x, x, indexing="ij")
    h = wl.tanh_indicator(np.sqrt(X ** 2 + Y ** 2)[None] - Rc * dx, 1.5 * dx)
    W = np.zeros((w.nvar,) + h.shape)
    W[2], W[3] = 1e5, 300.0
    if order == "liquid_first":
        W[4] = h                                   # water tracked
    else:
        W[4], W[5] = 0.5 * (1.0 - h), 0.5 * (1.0 - h)   # N2 and air tracked, water implied
    o = oracle.Oracle(w)
    q = o.prim_to_cons(W)
    alpha = q[0] * (h if order == "liquid_first" else 1.0 - W[4] - W[5]) / RHO_WATER
    S = o.csf_source(q)
    Req = np.sqrt(alpha.sum() * dx * dx / np.pi)
    c = n // 2
    jump = -S[0, 0, c, c:].sum() * dx
    assert abs(jump / (1.0 / Req) - 1.0) < 0.02, jump * Req
