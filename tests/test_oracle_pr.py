"""Pins of the oracle's Peng-Robinson closure (App. A.2.1) against the
critical point, the ideal-gas limit and thermodynamic identities."""
import math

import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl

RU = 8.314462618


def _o(comps=None):
    comps = comps or [wl.N2_PR, wl.DODECANE_PR]
    w = wl.Workload(name="pr", ndim=1, n=[4, 1, 1], lo=[0, 0, 0], hi=[1, 1, 1], bc=[[2, 2], [0, 0], [0, 0]],
                    comps=comps, liquid=len(comps) - 1, scheme=wl.default_scheme(), steps=1, cfl=0.4,
                    init="random")
    return oracle.Oracle(w)


@pytest.mark.parametrize("Y,comp", [([1.0], wl.N2_PR), ([0.0], wl.DODECANE_PR)])
def test_pure_component_critical_point(Y, comp):
    """At (Tc, pc) the PR cubic has its critical triple root Z_c = 0.3074:
    p(Tc, v_c) = pc and dp/dv = d2p/dv2 = 0 (A.2.1 with a_aa, b_a)."""
    o = _o()
    Tc, pc = comp["Tc"], comp["pc"]
    vc = 0.3074 * RU * Tc / pc
    s = o.pr_state(Tc, vc, Y)
    assert s["p"] == pytest.approx(pc, rel=2e-3)
    h = 1e-4 * vc
    p = [o.pr_state(Tc, vc + k * h, Y)["p"] for k in (-1, 0, 1)]
    dp = (p[2] - p[0]) / (2 * h)
    d2p = (p[2] - 2 * p[1] + p[0]) / h ** 2
    scale = pc / vc
    assert abs(dp) / scale < 2e-2 and abs(d2p) * vc / scale < 5e-2
    # the TDU at (pc, Tc) returns that root
    rho, e, c, al = o.forward(pc, Tc, Y)
    assert rho == pytest.approx(comp["M"] / vc, rel=5e-2)


def test_ideal_gas_limit():
    """v -> infinity: rho -> p M/(R T), e -> cv T, c -> sqrt(gamma R T / M)."""
    o = _o()
    for Y, comp in (([1.0], wl.N2_PR), ([0.0], wl.DODECANE_PR)):
        M, cv = comp["M"], comp["cv"]
        T, p = 900.0, 1.0
        rho, e, c, al = o.forward(p, T, Y)
        assert rho == pytest.approx(p * M / (RU * T), rel=1e-6)
        assert e == pytest.approx(cv * T, rel=1e-6)
        g = 1.0 + RU / (M * cv)
        assert c == pytest.approx(math.sqrt(g * RU * T / M), rel=1e-6)


@pytest.mark.parametrize("T,v,Y", [(900.0, 1.3e-3, [0.95]), (363.0, 3.0e-4, [0.0]), (500.0, 6e-4, [0.5])])
def test_thermodynamic_identities(T, v, Y):
    """(de/dv)_T = (T (dp/dT)_v - p)/M (molar v), cv = (de/dT)_v and
    c^2 = (dp/drho)_T + T (dp/dT)^2/(rho^2 cv), by central differences."""
    o = _o()
    s = o.pr_state(T, v, Y)
    M = s["M"]
    hv, hT = 1e-5 * v, 1e-4 * T
    e_v = (o.pr_state(T, v + hv, Y)["e"] - o.pr_state(T, v - hv, Y)["e"]) / (2 * hv)
    p_T = (o.pr_state(T + hT, v, Y)["p"] - o.pr_state(T - hT, v, Y)["p"]) / (2 * hT)
    p_v = (o.pr_state(T, v + hv, Y)["p"] - o.pr_state(T, v - hv, Y)["p"]) / (2 * hv)
    e_T = (o.pr_state(T + hT, v, Y)["e"] - o.pr_state(T - hT, v, Y)["e"]) / (2 * hT)
    assert e_v == pytest.approx((T * p_T - s["p"]) / M, rel=1e-5)
    assert e_T == pytest.approx(s["cv"], rel=1e-5)
    rho = M / v
    c2 = -(v * v / M) * p_v + T * p_T ** 2 / (rho ** 2 * e_T)
    assert s["c"] == pytest.approx(math.sqrt(c2), rel=1e-5)


def test_root_choice_and_roundtrip():
    """The TDU root is the lowest-Gibbs real root of the cubic (numpy roots
    as an independent solver) and the inverse recovers (p, T)."""
    o = _o()
    rng = np.random.default_rng(4)
    cases = [(6e6, 363.0, 0.0), (6e6, 900.0, 1.0), (6e6, 600.0, 0.3), (3e5, 450.0, 0.05), (2.7e7, 1518.0, 1.0)]
    cases += [(10 ** rng.uniform(5, 7.5), rng.uniform(350, 1500), rng.random()) for _ in range(20)]
    for p, T, Y in cases:
        rho, e, c, al = o.forward(p, T, [Y])
        Yf = np.array([Y, 1 - Y])
        M = 1.0 / (Yf[0] / wl.N2_PR["M"] + Yf[1] / wl.DODECANE_PR["M"])
        s = o.pr_state(T, M / rho, [Y])
        A, B = s["a"] * p / (RU * T) ** 2, s["b"] * p / (RU * T)
        roots = np.roots([1.0, -(1 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)])
        real = [r.real for r in roots if abs(r.imag) < 1e-9 * max(1, abs(r)) and r.real > B]
        s2 = math.sqrt(2)
        g = lambda Z: Z - 1 - math.log(Z - B) - A / (2 * s2 * B) * math.log((Z + (1 + s2) * B) / (Z + (1 - s2) * B))
        Zbest = min(real, key=g)
        Z = p * (M / rho) / (RU * T)
        assert Z == pytest.approx(Zbest, rel=1e-8)
        p2, T2 = o.inverse(rho, e, [Y])
        assert p2 == pytest.approx(p, rel=1e-8) and T2 == pytest.approx(T, rel=1e-10)
