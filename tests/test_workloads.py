"""The seeded input generator: Rankine-Hugoniot states (Table 4.3) and
determinism of the splitmix64 stream."""
import os

import numpy as np
import pytest

from paper_2304_00140_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_rankine_hugoniot_table_4_3():
    """Table 4.3: Ms = 1.22 in air (gamma 1.4) at 101325 Pa, 1.225 kg/m^3."""
    row = [float(x) for x in open(os.path.join(GOLD, "table_4_3.txt")).read().split("\n")[-2].split()]
    p2_t, u2_t, rho2_t, pr_t, rr_t = row
    g, p1, rho1 = 1.4, 101325.0, 1.225
    Ms = 1.22
    p2 = p1 * (1 + 2 * g / (g + 1) * (Ms ** 2 - 1))      # normal-shock pressure ratio
    cv = 718.0
    T1 = p1 / ((g - 1) * cv * rho1)
    r1, r2, u2, T2 = wl.rh_post_shock_sg(p1, T1, p2, wl.comp_sg(g, 0.0, cv))
    assert abs(r1 - rho1) < 1e-12 * rho1
    assert abs(p2 - p2_t) / p2_t < 1e-5 and abs(p2 / p1 - pr_t) < 1e-4
    assert abs(r2 - rho2_t) / rho2_t < 1e-3 and abs(r2 / r1 - rr_t) < 1e-4
    assert abs(u2 - u2_t) / u2_t < 1e-3


def test_splitmix64_reference_values():
    # first outputs of splitmix64 seeded with 0 (published test vector)
    s = wl.SplitMix64(0)
    assert s.next_u64() == 0xE220A8397B1DCDAF
    assert s.next_u64() == 0x6E789E6AA1B965F4


def test_ensemble_deterministic_and_in_range():
    a = wl.droplet_ensemble(ncases=64)
    b = wl.droplet_ensemble(ncases=64)
    assert [c.n for c in a] == [c.n for c in b]
    sides = {c.n[0] for c in a}
    assert sides <= set(wl.DROPLET_SIDES) and len(sides) >= 4
    amps = np.array([c.params["A"] / c.params["R"] for c in a])
    assert amps.min() >= 0.05 and amps.max() <= 0.2


def _sg_h(p, rho, comp):
    """specific enthalpy of a stiffened gas, e = (p + g pinf)/((g-1) rho)"""
    g, pi = comp["gamma"], comp["pinf"]
    return (p + g * pi) / ((g - 1.0) * rho) + p / rho


def test_shock_bubble_recipe():
    """The 2048 x 1024 shock-bubble: [0, 2] x [0, 1] mm, equal spacings,
    walls top and bottom, outflow sides; water at 1e5 Pa and 300 K at rest;
    an air bubble of radius 0.2 mm at (0.6, 0.5) mm; behind x = 0.3 mm the
    1 GPa post-shock state, which with the shock speed from mass
    conservation satisfies the momentum and energy jumps of a stiffened-gas
    shock."""
    w = wl.shock_bubble()
    assert w.n[:2] == [2048, 1024] and w.hi[:2] == [2e-3, 1e-3] and w.dx[0] == w.dx[1]
    assert w.bc[0] == [wl.BC_OUTFLOW, wl.BC_OUTFLOW] and w.bc[1] == [wl.BC_REFLECT, wl.BC_REFLECT]
    W = w.primitives()
    x, y, _ = w.centres()
    i_pre, i_post = np.searchsorted(x, 0.4e-3), np.searchsorted(x, 0.2e-3)
    j = np.searchsorted(y, 0.9e-3)
    assert W[0, 0, j, i_pre] == 0.0 and W[2, 0, j, i_pre] == 1e5 and W[3, 0, j, i_pre] == 300.0
    assert W[4, 0, j, i_pre] < 1e-12                                # water (air fraction tracked)
    ib, jb = np.searchsorted(x, 0.6e-3), np.searchsorted(y, 0.5e-3)
    assert W[4, 0, jb, ib] > 1 - 1e-12
    r = np.hypot(x[None, :] - 0.6e-3, y[:, None] - 0.5e-3)
    edge = np.abs(r - 0.2e-3) < 0.5 * w.dx[0]
    assert np.all(np.abs(W[4, 0][edge] - 0.5) < 0.2)
    u2, p2, T2 = W[0, 0, j, i_post], W[2, 0, j, i_post], W[3, 0, j, i_post]
    assert p2 == 1e9 and u2 > 0
    water = wl.WATER
    rho = lambda p, T: (p + water["pinf"]) / ((water["gamma"] - 1) * water["cv"] * T)
    r1, r2 = rho(1e5, 300.0), rho(p2, T2)
    S = r2 * u2 / (r2 - r1)                                      # shock speed from the mass jump
    assert abs((1e5 + r1 * S * S) - (p2 + r2 * (S - u2) ** 2)) < 1e-9 * p2
    assert abs((_sg_h(1e5, r1, water) + S * S / 2) - (_sg_h(p2, r2, water) + (S - u2) ** 2 / 2)) \
        < 1e-9 * _sg_h(p2, r2, water)


def test_pr_shock_droplet_recipe():
    """1024 x 1024 cells of 0.115 mm, an n-dodecane droplet of radius 128
    cells at 363 K in N2 at 6 MPa and 900 K, and a Mach 2 shock in the N2:
    the post-shock state satisfies the ideal-gas normal-shock jumps at the
    shock speed 2 c1."""
    w = wl.pr_shock_droplet()
    assert w.n[:2] == [1024, 1024] and abs(w.dx[0] - 0.115e-3) < 1e-18
    assert abs(w.params["R"] / w.dx[0] - 128.0) < 1e-9
    n2 = w.comps[0]
    Rs = 8.314462618 / n2["M"]
    g = 1.0 + Rs / n2["cv"]
    W = w.primitives()
    x, y, _ = w.centres()
    jc, ic = np.searchsorted(y, 0.5 * w.hi[1]), np.searchsorted(x, 0.5 * w.hi[0])
    assert W[3, 0, jc, ic] == pytest.approx(363.0) and W[4, 0, jc, ic] < 1e-12     # the droplet
    i1 = np.searchsorted(x, 0.3 * w.hi[0])
    assert W[2, 0, 0, i1] == 6e6 and W[3, 0, 0, i1] == 900.0 and W[0, 0, 0, i1] == 0.0
    i2 = np.searchsorted(x, 0.2 * w.hi[0])
    p2, T2, u2 = W[2, 0, 0, i2], W[3, 0, 0, i2], W[0, 0, 0, i2]
    r1, r2 = 6e6 / (Rs * 900.0), p2 / (Rs * T2)
    S = 2.0 * np.sqrt(g * Rs * 900.0)
    assert r1 * S == pytest.approx(r2 * (S - u2), rel=1e-12)
    assert 6e6 + r1 * S * S == pytest.approx(p2 + r2 * (S - u2) ** 2, rel=1e-12)
    h = lambda p, r: g / (g - 1) * p / r
    assert h(6e6, r1) + S * S / 2 == pytest.approx(h(p2, r2) + (S - u2) ** 2 / 2, rel=1e-12)


def test_jet_recipe():
    """512 x 256^2 cells on a 4 x 2 x 2 mm box; the liquid (pure dodecane-like
    stiffened gas at 363 K) enters through a disc of radius 16 cells on the
    x-low side at 300 m/s with a perturbation of at most 5%, seeded; the
    ambient N2/CH4 (Y_CH4 = 0.1) is at rest at 6 MPa and 900 K."""
    w = wl.jet3d()
    assert w.n == [512, 256, 256] and w.hi == [4e-3, 2e-3, 2e-3]
    f = w.inflow
    assert f["radius"] == pytest.approx(16 * w.dx[1]) and f["T"] == 363.0 and f["Y"] == [0.0, 0.0]
    assert w.bc[0][0] == wl.BC_INFLOW and w.comps[2] is wl.DODECANE_SG
    s = wl.jet3d(n=(64, 32, 32))
    W = s.primitives()
    assert np.all(W[3] == 6e6) and np.all(W[4] == 900.0) and np.all(W[6] == 0.1) and np.all(W[:3] == 0.0)
    u = wl.jet_inflow_velocity(w)
    assert np.all(np.abs(u[0] / 300.0 - 1.0) <= 0.05 + 1e-15) and np.all(u[1:] == 0.0)
    assert np.array_equal(u, wl.jet_inflow_velocity(wl.jet3d()))
    assert abs(u[0].mean() / 300.0 - 1.0) < 2e-3 and u[0].std() > 0.005 * 300.0


def test_droplet_and_advection_recipes():
    """The ensemble's droplets: R = 0.25 L, at rest, 1e5 Pa, 300 K,
    sigma = 0.07 N/m; the advection column: radius 0.2 m, centred, 50 m/s
    in x and y, 1e5 Pa, 300 K; both tanh-smoothed over 1.5 cells."""
    for c in wl.droplet_ensemble(ncases=16):
        assert c.params["R"] == 0.25 * (c.hi[0] - c.lo[0]) and c.scheme["sigma"] == 0.07
        assert c.params["p"] == 1e5 and c.params["T"] == 300.0 and c.params["width"] == 1.5
        assert all(b == [wl.BC_PERIODIC] * 2 for b in c.bc[:2])
    w = wl.advection()
    W = w.primitives()
    assert np.all(W[0] == 50.0) and np.all(W[1] == 50.0) and np.all(W[2] == 1e5) and np.all(W[3] == 300.0)
    x, y, _ = w.centres()
    r = np.hypot(x[None, :] - 0.5, y[:, None] - 0.5)
    h = 1.0 - W[4, 0]
    assert np.allclose(h, 0.5 * (1 - np.tanh((r - 0.2) / (1.5 / 128))), rtol=0, atol=1e-15)


def test_rising_bubble_recipe():
    """Table 4.4 case 2: liquid and gas densities 1000 and 1 kg/m^3 at
    1e5 Pa and 300 K (the closures' cv are chosen for that), g = 0.98 m/s^2
    down, sigma = 1.96 N/m; the liquid's pressure hydrostatic from 1e5 Pa at
    the top, the bubble's the liquid's at its centre plus sigma/R."""
    import oracle
    w = wl.rising_bubble(2, n=(40, 80))
    o = oracle.Oracle(w)
    assert o.forward(1e5, 300.0, [0.0])[0] == pytest.approx(1000.0, rel=1e-12)
    assert o.forward(1e5, 300.0, [1.0])[0] == pytest.approx(1.0, rel=1e-12)
    assert w.scheme["gravity"] == (0.0, -0.98, 0.0) and w.scheme["sigma"] == 1.96
    W = w.primitives()
    x, y, _ = w.centres()
    j = np.searchsorted(y, 1.6)
    assert W[2, 0, j, 2] == pytest.approx(1e5 + 1000.0 * 0.98 * (w.hi[1] - y[j]), rel=1e-14)
    jc, ic = np.searchsorted(y, 0.5), np.searchsorted(x, 0.5)
    assert W[4, 0, jc, ic] > 1 - 1e-4                    # tanh-smoothed over 1.5 cells
    p_in = 1e5 + 1000.0 * 0.98 * (w.hi[1] - 0.5) + 1.96 / 0.25
    assert abs(W[2, 0, jc, ic] - p_in) < 1e-8 * p_in


def test_bubble_collapse_recipe():
    """Sec. 4.9: R = 400 um at H = 440 um above the wall on the
    [-2, 2] x [0, 4] mm box, 4 um cells at 1000^2; the liquid pressure
    p_inf + (R/r)(p_b - p_inf) outside the bubble, p_inf = 10 MPa, the gas
    bubble at 3000 Pa."""
    w = wl.bubble_collapse("gas", n=(1000, 1000))
    assert w.dx[0] == pytest.approx(4e-6) and w.dx[1] == pytest.approx(4e-6)
    assert w.lo[:2] == [-2e-3, 0.0] and w.bc[1][0] == wl.BC_REFLECT
    s = wl.bubble_collapse("gas", n=(200, 200))
    W = s.primitives()
    x, y, _ = s.centres()
    for (xi, yi) in ((1.5e-3, 3.5e-3), (-1.0e-3, 0.1e-3), (0.0, 1.5e-3)):
        i, j = np.searchsorted(x, xi), np.searchsorted(y, yi)
        r = np.hypot(x[i], y[j] - 440e-6)
        want = 1e7 + (400e-6 / r) * (s.params["p_b"] - 1e7)
        assert W[2, 0, j, i] == pytest.approx(want, rel=1e-9)
    assert s.params["p_b"] == 3000.0 and s.params["p_inf"] == 1e7
    i0, j0 = np.searchsorted(x, 0.0), np.searchsorted(y, 440e-6)
    assert W[2, 0, j0, i0] == pytest.approx(3000.0, rel=1e-6) and W[4, 0, j0, i0] > 1 - 1e-6
