"""Seeded synthetic workloads: grids, materials, scheme switches and initial
primitive fields.

This module is shared by the CUDA path, the tests and the benchmark.  It holds
none of the scheme's arithmetic: it only places materials on a grid (tanh
smoothed interfaces, a planar shock, droplets and a jet inflow disc) and draws
the random numbers the workloads need from a splitmix64 stream.  Each consumer
turns the primitive fields (u, p, T, Y) into conserved variables with its own
closure.

The one piece of physics it evaluates is the Rankine-Hugoniot jump of a pure
stiffened gas (Sec. 4.2, Table 4.3 gives the ideal-gas case), written with the
single-material relation rho = (p + pinf) / ((gamma - 1) cv T) of Eq. A.1.1.
That is initial-condition data, not the mixture closure the scheme uses.

Layouts
-------
* Primitive fields: float64 array ``[nv, nz, ny, nx]`` with variables
  ``u_0 .. u_{d-1}, p, T, Y_0 .. Y_{N-2}`` (Y of the last component is
  implied by sum Y = 1).
* Conserved fields (produced elsewhere): ``rho, rho u_0 .. rho u_{d-1},
  rho E, rho Y_0 .. rho Y_{N-2}`` in the same ``[nv, nz, ny, nx]`` layout,
  x fastest.  This is the four-equation state vector of Eq. 2-1.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

SEED = 20230401
MASK64 = (1 << 64) - 1

# boundary kinds
BC_PERIODIC, BC_REFLECT, BC_OUTFLOW, BC_INFLOW = 0, 1, 2, 3
# limiter ids (Table 4.2 plus the Superbee form printed in Sec. 3.3)
LIM_MINMOD, LIM_KOREN, LIM_VANLEER, LIM_VANALBADA, LIM_CHAKRAVARTHY, LIM_MC, LIM_SUPERBEE = range(7)
# component kinds
KIND_SG, KIND_PR, KIND_BARO = 0, 1, 2


# --------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------
class SplitMix64:
    """splitmix64 (Steele, Lea & Flood 2014): state += golden gamma, then
    two xor-shift-multiply rounds.  ``uniform()`` maps the top 53 bits to
    [0, 1)."""

    def __init__(self, seed: int = SEED):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def uniforms(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        return np.array([self.uniform(lo, hi) for _ in range(n)], dtype=np.float64)


# --------------------------------------------------------------------------
# materials (parameters of Eq. A.1.1 / A.2.1)
# --------------------------------------------------------------------------
def comp_sg(gamma, pinf, cv, q=0.0, M=0.0, mu=0.0, kc=0.0):
    """stiffened gas (ideal gas when pinf = 0); mu, kc: dynamic viscosity
    (Pa s) and thermal conductivity (W/(m K)) of Eq. 2-2, 0 = inviscid"""
    return dict(kind=KIND_SG, gamma=float(gamma), pinf=float(pinf), cv=float(cv), q=float(q),
                Tc=0.0, pc=0.0, omega=0.0, M=float(M), mu=float(mu), kc=float(kc))


def comp_baro_liquid(psat, rho_sl, rho_sv, cl):
    """barotropic liquid / liquid-vapour mixture (Sec. 2.2, Eq. 2-3, 2-4,
    2-7): saturation pressure, saturated liquid and vapour densities, liquid
    sound speed"""
    return dict(kind=KIND_BARO, gamma=0.0, pinf=0.0, cv=1.0, q=0.0, Tc=0.0, pc=0.0, omega=0.0, M=0.0,
                mu=0.0, kc=0.0, psat=float(psat), rho_sl=float(rho_sl), rho_sv=float(rho_sv), cl=float(cl), rt=0.0)


def comp_baro_gas(R, T_ref):
    """non-condensable ideal gas at the fixed temperature T_ref (Eq. 2-5)"""
    return dict(kind=KIND_BARO, gamma=0.0, pinf=0.0, cv=1.0, q=0.0, Tc=0.0, pc=0.0, omega=0.0, M=0.0,
                mu=0.0, kc=0.0, psat=0.0, rho_sl=0.0, rho_sv=0.0, cl=0.0, rt=float(R) * float(T_ref))


def comp_pr(Tc, pc, omega, cv, M):
    return dict(kind=KIND_PR, gamma=0.0, pinf=0.0, cv=float(cv), q=0.0,
                Tc=float(Tc), pc=float(pc), omega=float(omega), M=float(M), mu=0.0, kc=0.0)


WATER = comp_sg(6.12, 3.43e8, 1816.0)
AIR = comp_sg(1.4, 0.0, 718.0)
DODECANE_SG = comp_sg(2.35, 4.0e8, 1077.0)
N2_IG = comp_sg(1.4, 0.0, 743.0)
CH4_IG = comp_sg(1.304, 0.0, 1709.0)
DODECANE_PR = comp_pr(658.1, 1.817e6, 0.574, 2200.0, 0.170338)
N2_PR = comp_pr(126.2, 3.396e6, 0.037, 743.0, 0.0280134)


def default_scheme(**kw) -> Dict:
    s = dict(iles=0, thinc=1, beta=1.6, thinc_eps=1e-4, thinc_gamma=1e-20,
             lim_vel=LIM_KOREN, lim_scalar=LIM_MINMOD,
             thr_ducros=0.95, thr_gas=0.4, eps_ducros=1e-20, d3p_coef=0.5,
             sigma=0.0, grad_eps=1e-5, precision=0, p_ref=1e5, T_ref=300.0,
             gravity=(0.0, 0.0, 0.0), thr_vap=0.4, curvature=0)
    s.update(kw)
    return s


def with_transport(w: "Workload", mu, kc=None, gravity=None) -> "Workload":
    """Copy of a workload with per-component viscosities ``mu`` and
    conductivities ``kc`` (Eq. 2-2; lists in component order) and, if given,
    the body force per unit mass ``gravity`` (3 components, m/s^2)."""
    kc = kc if kc is not None else [0.0] * len(w.comps)
    comps = [dict(c, mu=float(m), kc=float(k)) for c, m, k in zip(w.comps, mu, kc)]
    scheme = dict(w.scheme)
    if gravity is not None:
        scheme["gravity"] = tuple(float(g) for g in gravity)
    return dataclasses.replace(w, comps=comps, scheme=scheme)


@dataclasses.dataclass
class Workload:
    name: str
    ndim: int
    n: List[int]                 # interior cells (nx, ny, nz); nz = 1 in 2D
    lo: List[float]
    hi: List[float]
    bc: List[List[int]]          # [dim][low, high]
    comps: List[Dict]
    liquid: int                  # index of the liquid component (CSF, sensors)
    scheme: Dict
    steps: int
    cfl: float
    init: str                    # initial-condition recipe name
    params: Dict = dataclasses.field(default_factory=dict)
    inflow: Optional[Dict] = None

    @property
    def ncomp(self) -> int:
        return len(self.comps)

    @property
    def nvar(self) -> int:
        return self.ndim + 2 + self.ncomp - 1

    @property
    def cells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def dx(self) -> List[float]:
        return [(self.hi[d] - self.lo[d]) / self.n[d] for d in range(3)]

    def centres(self):
        """cell-centre coordinates x[nx], y[ny], z[nz]"""
        return [self.lo[d] + (np.arange(self.n[d]) + 0.5) * self.dx[d] for d in range(3)]

    def primitives(self) -> np.ndarray:
        return _INIT[self.init](self)


# --------------------------------------------------------------------------
# initial-condition helpers
# --------------------------------------------------------------------------
def tanh_indicator(dist, width):
    """1 inside (dist < 0), 0 outside, smoothed by tanh over ``width``."""
    return 0.5 * (1.0 - np.tanh(dist / width))


def rh_post_shock_sg(p1, T1, p2, comp):
    """Post-shock (rho2, u2, T2) of a right-moving shock into a pure
    stiffened gas at rest (p1, T1).  Shock adiabat with p -> p + pinf:
    rho2/rho1 = ((g+1)(p2+pi) + (g-1)(p1+pi)) / ((g-1)(p2+pi) + (g+1)(p1+pi)),
    u2 = sqrt((p2-p1)(1/rho1 - 1/rho2))."""
    g, pi, cv = comp["gamma"], comp["pinf"], comp["cv"]
    rho1 = (p1 + pi) / ((g - 1.0) * cv * T1)
    a, b = p2 + pi, p1 + pi
    rho2 = rho1 * ((g + 1.0) * a + (g - 1.0) * b) / ((g - 1.0) * a + (g + 1.0) * b)
    u2 = math.sqrt((p2 - p1) * (1.0 / rho1 - 1.0 / rho2))
    T2 = (p2 + pi) / ((g - 1.0) * cv * rho2)
    return rho1, rho2, u2, T2


def _alloc(w: Workload):
    return np.zeros((w.nvar, w.n[2], w.n[1], w.n[0]), dtype=np.float64)


def _grid(w: Workload):
    x, y, z = w.centres()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def _init_column(w: Workload):
    """Advection: a water column of radius R (centred) in air, uniform p, T
    and velocity; Y_water tanh-smoothed over ``width`` cells."""
    P = w.params
    X, Y, _ = _grid(w)
    xc = 0.5 * (w.lo[0] + w.hi[0]); yc = 0.5 * (w.lo[1] + w.hi[1])
    r = np.sqrt((X - xc) ** 2 + (Y - yc) ** 2)
    h = tanh_indicator(r - P["R"], P["width"] * w.dx[0])     # liquid indicator
    W = _alloc(w)
    W[0] = P["u"][0]; W[1] = P["u"][1]
    W[w.ndim] = P["p"]; W[w.ndim + 1] = P["T"]
    # component 0 = air (tracked), component 1 = water (implied)
    W[w.ndim + 2] = 1.0 - h
    return W


def _init_shock_bubble(w: Workload):
    """Shock-bubble: planar shock in water (post-shock p2, RH states) at x_s
    moving +x, air bubble (radius R at (xb, yb)) tanh-smoothed."""
    P = w.params
    X, Y, _ = _grid(w)
    water = w.comps[1]
    _, _, u2, T2 = rh_post_shock_sg(P["p"], P["T"], P["p2"], water)
    r = np.sqrt((X - P["xb"]) ** 2 + (Y - P["yb"]) ** 2)
    gas = tanh_indicator(r - P["R"], P["width"] * w.dx[0])
    post = X < P["xs"]
    W = _alloc(w)
    W[0] = np.where(post, u2, 0.0)
    W[1] = 0.0
    W[w.ndim] = np.where(post, P["p2"], P["p"])
    W[w.ndim + 1] = np.where(post, T2, P["T"])
    W[w.ndim + 2] = gas
    return W


def _init_droplet(w: Workload):
    """Oscillating droplet: a water droplet with an elliptical (mode-2) radius
    perturbation r_i(theta) = R + A cos(2 theta), at rest, uniform p and T.
    ``dp`` optionally presets a pressure jump inside (static-drop tests)."""
    P = w.params
    X, Y, _ = _grid(w)
    xc = 0.5 * (w.lo[0] + w.hi[0]); yc = 0.5 * (w.lo[1] + w.hi[1])
    dxx, dyy = X - xc, Y - yc
    r = np.sqrt(dxx ** 2 + dyy ** 2)
    th = np.arctan2(dyy, dxx)
    ri = P["R"] + P.get("A", 0.0) * np.cos(2.0 * th)
    h = tanh_indicator(r - ri, P["width"] * w.dx[0])
    W = _alloc(w)
    W[0] = P.get("u", 0.0)
    W[w.ndim] = P["p"] + P.get("dp", 0.0) * h
    W[w.ndim + 1] = P["T"]
    W[w.ndim + 2] = 1.0 - h           # air tracked, water implied
    return W


def _init_random(w: Workload):
    """Smooth random state with a material interface, for stage parity: all
    variables carry seeded perturbations so every branch (both upwind
    signs, limiter regimes, THINC eligible and not) is exercised."""
    P = w.params
    rng = SplitMix64(P.get("seed", SEED))
    X, Y, Z = _grid(w)
    L = [w.hi[d] - w.lo[d] for d in range(3)]
    W = _alloc(w)

    def field(amp):
        f = np.zeros_like(X)
        for _ in range(4):
            kx, ky, kz = (int(rng.uniform(1, 4)) for _ in range(3))
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-1, 1)
            arg = 2 * math.pi * (kx * X / L[0] + ky * Y / L[1] + (kz * Z / L[2] if w.ndim == 3 else 0.0)) + ph
            f += a * np.sin(arg)
        return amp * f / 4.0

    for d in range(w.ndim):
        W[d] = P.get("u0", [0.0, 0.0, 0.0])[d] + field(P.get("du", 30.0))
    W[w.ndim] = P["p"] * (1.0 + field(P.get("dp_rel", 0.2)))
    W[w.ndim + 1] = P["T"] * (1.0 + field(P.get("dT_rel", 0.1)))
    Tl = P.get("T_liquid")
    xc = [w.lo[d] + 0.5 * L[d] for d in range(3)]
    r2 = (X - xc[0]) ** 2 + (Y - xc[1]) ** 2
    if w.ndim == 3:
        r2 = r2 + (Z - xc[2]) ** 2
    h = tanh_indicator(np.sqrt(r2) - P["R"] * (1.0 + field(0.3)), P["width"] * w.dx[0])
    if Tl is not None:        # liquid colder than the gas (temperature blended by the indicator)
        W[w.ndim + 1] = (Tl * h + W[w.ndim + 1] * (1.0 - h))
    nc = w.ncomp
    if nc == 2:
        W[w.ndim + 2] = 1.0 - h
    else:
        # gas split into two species (N2, CH4) with a smooth ratio; liquid implied
        ratio = np.clip(0.5 + field(0.8), 0.0, 1.0)
        W[w.ndim + 2] = (1.0 - h) * ratio
        W[w.ndim + 3] = (1.0 - h) * (1.0 - ratio)
    return W


def _init_jet(w: Workload):
    """3D jet: ambient N2/CH4 gas at rest filling the box; the liquid
    enters through the inflow disc on the x-low face (boundary data)."""
    P = w.params
    W = _alloc(w)
    W[w.ndim] = P["p"]
    W[w.ndim + 1] = P["T"]
    W[w.ndim + 2] = 1.0 - P["Y_ch4"]      # N2
    W[w.ndim + 3] = P["Y_ch4"]            # CH4 (dodecane implied = 0)
    return W


def rh_post_shock_ig(p1, T1, Ms, gamma, Rs):
    """Ideal-gas normal-shock state behind a shock of Mach number Ms moving
    into gas at rest (p1, T1): pressure and density ratios and u2."""
    g = gamma
    pr_ = (2.0 * g * Ms * Ms - (g - 1.0)) / (g + 1.0)
    rr_ = (g + 1.0) * Ms * Ms / ((g - 1.0) * Ms * Ms + 2.0)
    c1 = math.sqrt(g * Rs * T1)
    u2 = Ms * c1 * (1.0 - 1.0 / rr_)
    return p1 * pr_, T1 * pr_ / rr_, u2


def _init_pr_drop(w: Workload):
    """Near-critical shock/droplet: n-dodecane droplet (radius R) at T_l in N2 at (p, T), Mach
    Ms shock in the N2 at x_s moving +x.  READING: the post-shock state is
    the ideal-gas Rankine-Hugoniot state of N2 (gamma = 1 + R/(M cv)); with
    the PR closure the jump sheds a weak wave."""
    P = w.params
    X, Y, _ = _grid(w)
    n2 = w.comps[0]
    Rs = 8.314462618 / n2["M"]
    p2, T2, u2 = rh_post_shock_ig(P["p"], P["T"], P["Ms"], 1.0 + Rs / n2["cv"], Rs)
    xc, yc = 0.5 * (w.lo[0] + w.hi[0]), 0.5 * (w.lo[1] + w.hi[1])
    r = np.sqrt((X - xc) ** 2 + (Y - yc) ** 2)
    h = tanh_indicator(r - P["R"], P["width"] * w.dx[0])   # liquid indicator
    post = X < P["xs"]
    W = _alloc(w)
    W[0] = np.where(post, u2, 0.0)
    W[w.ndim] = np.where(post, p2, P["p"])
    W[w.ndim + 1] = np.where(post, T2, P["T_l"] * h + P["T"] * (1.0 - h))
    W[w.ndim + 2] = 1.0 - h                                 # N2 tracked, dodecane implied
    return W


def _init_bubble(w: Workload):
    """Rising bubble: a gas bubble of radius R at (xb, yb) in liquid at rest,
    hydrostatic pressure p_top + rho_l |g| (H - y) in the liquid, the liquid
    pressure at the bubble centre plus the Laplace jump sigma / R inside,
    uniform T; the gas fraction tanh-smoothed."""
    P = w.params
    X, Y, _ = _grid(w)
    r = np.sqrt((X - P["xb"]) ** 2 + (Y - P["yb"]) ** 2)
    gas = tanh_indicator(r - P["R"], P["width"] * w.dx[0])
    g = abs(w.scheme["gravity"][1])
    p_liq = P["p"] + P["rho_l"] * g * (w.hi[1] - Y)
    p_in = P["p"] + P["rho_l"] * g * (w.hi[1] - P["yb"]) + w.scheme["sigma"] / P["R"]
    W = _alloc(w)
    W[w.ndim] = gas * p_in + (1.0 - gas) * p_liq
    W[w.ndim + 1] = P["T"]
    W[w.ndim + 2] = gas               # gas tracked, liquid implied
    return W


def _init_collapse(w: Workload):
    """Bubble collapse near a wall: bubble of radius R centred at (0, H),
    liquid at rest with the pressure p_inf + (R / r)(p_b - p_inf) outside
    the bubble (r from the bubble centre), p_b inside; tanh-smoothed.  Gas
    bubble: non-condensable gas (Y = 1) at p_b.  Vapour bubble: no gas, the
    liquid-vapour mixture at the pressure p_b that the barotropic law gives
    for the capped vapour fraction."""
    P = w.params
    X, Y, Z = _grid(w)
    r2 = X ** 2 + (Y - P["H"]) ** 2
    if w.ndim == 3:
        r2 = r2 + Z ** 2
    r = np.sqrt(r2)
    h = tanh_indicator(r - P["R"], P["width"] * w.dx[0])      # bubble indicator
    pb, pinf = P["p_b"], P["p_inf"]
    ramp = pinf + (P["R"] / np.maximum(r, P["R"])) * (pb - pinf)
    W = _alloc(w)
    W[w.ndim] = h * pb + (1.0 - h) * ramp
    W[w.ndim + 1] = P["e"]
    W[w.ndim + 2] = h if P["gas"] else 0.0
    return _split_gas(W, w)


_INIT = {"collapse": _init_collapse, "bubble": _init_bubble, "pr_drop": _init_pr_drop, "column": _init_column, "shock_bubble": _init_shock_bubble,
         "droplet": _init_droplet, "random": _init_random, "jet": _init_jet}


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------
def advection(n=128, steps=200, **scheme):
    """Plain method, 2D periodic advection of a water column in air, n x n
    cells on [0, 1]^2 m, uniform p = 1e5 Pa, T = 300 K, u = (50, 50) m/s,
    column radius 0.2 m, THINC on, no surface tension, CFL 0.4."""
    nx, ny = (n, n) if isinstance(n, int) else n
    return Workload(
        name=f"advection_{nx}x{ny}", ndim=2, n=[nx, ny, 1], lo=[0.0, 0.0, 0.0], hi=[1.0, 1.0 * ny / nx, 1.0],
        bc=[[BC_PERIODIC] * 2, [BC_PERIODIC] * 2, [BC_PERIODIC] * 2],
        comps=[AIR, WATER], liquid=1, scheme=default_scheme(**scheme), steps=steps, cfl=0.4,
        init="column", params=dict(R=0.2, width=1.5, u=(50.0, 50.0), p=1e5, T=300.0))


def shock_bubble(nx=2048, ny=1024, steps=4000, **scheme):
    """2D shock-bubble interaction: nx x ny cells on [0, 2] x [0, 1] mm,
    water at 1e5 Pa / 300 K, air bubble of radius 0.2 mm at (0.6, 0.5) mm,
    planar shock with post-shock p = 1e9 Pa at x = 0.3 mm moving +x.
    Reflective top/bottom, outflow right (and left), CFL 0.4."""
    L = 1e-3
    return Workload(
        name=f"shock_bubble_{nx}x{ny}", ndim=2, n=[nx, ny, 1], lo=[0.0, 0.0, 0.0],
        hi=[2 * L, 2 * L * ny / nx, 1.0],
        bc=[[BC_OUTFLOW, BC_OUTFLOW], [BC_REFLECT, BC_REFLECT], [BC_PERIODIC] * 2],
        comps=[AIR, WATER], liquid=1, scheme=default_scheme(**scheme), steps=steps, cfl=0.4,
        init="shock_bubble",
        params=dict(p=1e5, T=300.0, p2=1e9, xs=0.3e-3, xb=0.6e-3, yb=0.5e-3 * (2 * ny / nx), R=0.2e-3,
                    width=1.5))


def droplet(n=128, A=0.1, L=1e-3, sigma=0.07, steps=500, dp=0.0, **scheme):
    """One oscillating water droplet in air: n x n periodic cells on an
    L x L box, R = 0.25 L, elliptical perturbation amplitude A*R, at rest,
    p = 1e5 Pa, T = 300 K, CSF with the given sigma."""
    nx, ny = (n, n) if isinstance(n, int) else n
    R = 0.25 * L
    sch = default_scheme(sigma=sigma, **scheme)
    return Workload(
        name=f"droplet_{nx}x{ny}", ndim=2, n=[nx, ny, 1], lo=[0.0, 0.0, 0.0], hi=[L, L * ny / nx, 1.0],
        bc=[[BC_PERIODIC] * 2, [BC_PERIODIC] * 2, [BC_PERIODIC] * 2],
        comps=[AIR, WATER], liquid=1, scheme=sch, steps=steps, cfl=0.4, init="droplet",
        params=dict(R=R, A=A * R, width=1.5, p=1e5, T=300.0, dp=dp))


DROPLET_SIDES = (64, 96, 128, 192, 256)


def droplet_ensemble(ncases=1024, seed=SEED, steps=500, **scheme):
    """Batched ensemble: ncases independent oscillating droplets, sides drawn
    uniformly from {64, 96, 128, 192, 256}, amplitude uniform in
    [0.05, 0.2] x R, sigma = 0.07 N/m.  Returns the list of cases."""
    rng = SplitMix64(seed)
    cases = []
    for _ in range(ncases):
        side = DROPLET_SIDES[min(int(rng.uniform(0, len(DROPLET_SIDES))), len(DROPLET_SIDES) - 1)]
        amp = rng.uniform(0.05, 0.2)
        cases.append(droplet(n=side, A=amp, steps=steps, **scheme))
    return cases


def random_state(n=(24, 20), ncomp=2, seed=SEED, bc=None, ndim=2, pr=False, **scheme):
    """Seeded smooth random state with a material interface for stage-level
    parity (every branch of the stage is exercised).  pr=True: N2 / n-dodecane
    on Peng-Robinson at 6 MPa, gas near 900 K around a 363 K liquid."""
    nx, ny = n[0], n[1]
    nz = n[2] if ndim == 3 else 1
    L = 1e-3
    if pr:
        comps = [N2_PR, DODECANE_PR]
        params = dict(seed=seed, p=6e6, T=900.0, T_liquid=363.0, dT_rel=0.05, dp_rel=0.1, R=0.3e-3,
                      width=1.5, du=40.0)
        scheme = dict(dict(p_ref=6e6, T_ref=900.0), **scheme)
    else:
        comps = [AIR, WATER] if ncomp == 2 else [N2_IG, CH4_IG, DODECANE_SG]
        params = dict(seed=seed, p=2e6, T=320.0, R=0.3e-3, width=1.5, du=40.0)
    bc = bc or [[BC_PERIODIC] * 2, [BC_PERIODIC] * 2, [BC_PERIODIC] * 2]
    return Workload(
        name=f"random_{nx}x{ny}x{nz}", ndim=ndim, n=[nx, ny, nz], lo=[0.0, 0.0, 0.0],
        hi=[L, L * ny / nx, L * nz / nx], bc=bc, comps=comps, liquid=len(comps) - 1,
        scheme=default_scheme(**scheme), steps=1, cfl=0.4, init="random", params=params)


def jet3d(n=(512, 256, 256), steps=1000, seed=SEED, **scheme):
    """3D liquid jet primary break-up: n cells on a 4 x 2 x 2 mm box,
    dodecane-like stiffened-gas liquid (gamma 2.35, pinf 4e8, cv 1077) at
    363 K injected through a circular inflow of radius 16 cells (scaled with
    ny/256) at 300 m/s, into an N2/CH4 ideal-gas mixture (Y_CH4 = 0.1) at
    6 MPa and 900 K at rest; outflow elsewhere; App. D switch and CSF with
    sigma = 0.025 N/m."""
    nx, ny, nz = n
    L = 4e-3
    hi = [L, L * ny / nx, L * nz / nx]
    dy = hi[1] / ny
    radius = 16.0 * dy * ny / 256.0
    sch = default_scheme(**dict(dict(iles=1, sigma=0.025, p_ref=6e6, T_ref=900.0), **scheme))
    w = Workload(
        name=f"jet3d_{nx}x{ny}x{nz}", ndim=3, n=[nx, ny, nz], lo=[0.0, 0.0, 0.0], hi=hi,
        bc=[[BC_INFLOW, BC_OUTFLOW], [BC_OUTFLOW, BC_OUTFLOW], [BC_OUTFLOW, BC_OUTFLOW]],
        comps=[N2_IG, CH4_IG, DODECANE_SG], liquid=2, scheme=sch, steps=steps, cfl=0.4, init="jet",
        params=dict(p=6e6, T=900.0, Y_ch4=0.1, seed=seed, U=300.0, amp=0.05),
        inflow=dict(yc=0.5 * hi[1], zc=0.5 * hi[2], radius=radius, T=363.0, Y=[0.0, 0.0], u0=(300.0, 0.0, 0.0)))
    return w


def jet_inflow_velocity(w: Workload) -> np.ndarray:
    """[3][nz][ny] inflow velocity of the jet: U (1 + amp (sin(4 phi) / 2 +
    r_i / 2)) along x with r_i seeded uniform in [-1, 1] per face cell and phi
    the polar angle around the disc centre (READING: a steady 5% sinusoidal
    plus random perturbation).  Outside the disc the values are unused."""
    P, f = w.params, w.inflow
    ny, nz = w.n[1], w.n[2]
    rng = SplitMix64(P["seed"] ^ 0x4A4554)
    rnd = np.array([rng.uniform(-1.0, 1.0) for _ in range(ny * nz)]).reshape(nz, ny)
    y = w.lo[1] + (np.arange(ny) + 0.5) * w.dx[1] - f["yc"]
    z = w.lo[2] + (np.arange(nz) + 0.5) * w.dx[2] - f["zc"]
    Z, Y = np.meshgrid(z, y, indexing="ij")
    phi = np.arctan2(Z, Y)
    u = np.zeros((3, nz, ny))
    u[0] = P["U"] * (1.0 + P["amp"] * (0.5 * np.sin(4.0 * phi) + 0.5 * rnd))
    return u


def pr_shock_droplet(n=1024, steps=2000, **scheme):
    """2D near-critical shock/droplet on Peng-Robinson: n x n cells of
    0.115 mm (READING of the unstated spacing), an n-dodecane droplet of
    radius n/8 cells at 363 K in N2 at 6 MPa and 900 K, a Mach 2 shock in the
    N2 at x = L/4 moving +x, outflow on every side, FP32-mixed with the FP64
    Newton inversion.  CFL 0.4."""
    dx = 0.115e-3
    L = n * dx
    sch = default_scheme(**dict(dict(precision=1, p_ref=6e6, T_ref=900.0), **scheme))
    return Workload(
        name=f"pr_shock_droplet_{n}x{n}", ndim=2, n=[n, n, 1], lo=[0.0, 0.0, 0.0], hi=[L, L, 1.0],
        bc=[[BC_OUTFLOW] * 2, [BC_OUTFLOW] * 2, [BC_PERIODIC] * 2], comps=[N2_PR, DODECANE_PR], liquid=1,
        scheme=sch, steps=steps, cfl=0.4, init="pr_drop",
        params=dict(p=6e6, T=900.0, T_l=363.0, Ms=2.0, xs=0.25 * L, R=n / 8 * dx, width=1.5))


# Table 4.4: liquid / gas densities, viscosities, gravity and surface tension
RISING_BUBBLE_CASES = {1: dict(rho_l=1000.0, rho_g=100.0, mu_l=10.0, mu_g=1.0, g=0.98, sigma=24.5),
                       2: dict(rho_l=1000.0, rho_g=1.0, mu_l=10.0, mu_g=0.1, g=0.98, sigma=1.96)}


def rising_bubble(case=1, n=None, steps=1000, **scheme):
    """Rising bubble (Sec. 4.3, Table 4.4): a 1 x 2 m box of n cells
    (100 x 200 for case 1, 160 x 320 for case 2), a gas bubble of radius
    0.25 m at (0.5, 0.5) m in liquid, gravity 0.98 m/s^2 along -y, walls on
    every side, CSF and viscous stresses on.  The paper closes both fluids
    with its barotropic relations; here the liquid is a stiffened gas
    (gamma 6.12, pinf 3.43e8 Pa) and the gas an ideal gas (gamma 1.4), their
    cv chosen so that the densities of Table 4.4 hold at 1e5 Pa and 300 K.
    No heat conduction."""
    c = RISING_BUBBLE_CASES[case]
    nx, ny = n if n is not None else ((100, 200) if case == 1 else (160, 320))
    p0, T0 = 1e5, 300.0
    liquid = comp_sg(6.12, 3.43e8, (p0 + 3.43e8) / (5.12 * c["rho_l"] * T0), mu=c["mu_l"])
    gas = comp_sg(1.4, 0.0, p0 / (0.4 * c["rho_g"] * T0), mu=c["mu_g"])
    sch = default_scheme(**dict(dict(sigma=c["sigma"], gravity=(0.0, -c["g"], 0.0)), **scheme))
    return Workload(
        name=f"rising_bubble{case}_{nx}x{ny}", ndim=2, n=[nx, ny, 1], lo=[0.0, 0.0, 0.0], hi=[1.0, 1.0 * ny / nx, 1.0],
        bc=[[BC_REFLECT] * 2, [BC_REFLECT] * 2, [BC_PERIODIC] * 2], comps=[gas, liquid], liquid=1,
        scheme=sch, steps=steps, cfl=0.4, init="bubble",
        params=dict(p=p0, T=T0, rho_l=c["rho_l"], xb=0.5, yb=0.5, R=0.25, width=1.5))


# water near 11 C: saturation pressure 1342 Pa (Sec. 4.9), saturated liquid
# and vapour densities, liquid sound speed; air as the non-condensable gas
WATER_BARO = comp_baro_liquid(1342.0, 999.7, 0.0100, 1450.0)
AIR_BARO = comp_baro_gas(287.05, 293.15)


def bubble_collapse3d(kind="gas", n=(48, 48, 48), p_inf=1e7, gases=1, steps=200, **scheme):
    """3D form of the bubble collapse near a wall: the 4 x 4 x 4 mm box
    [-2, 2] x [0, 4] x [-2, 2] mm, bubble centred at (0, H, 0), wall at
    y = 0, outflow elsewhere.  gases = 2 splits the non-condensable gas
    into air and a second ideal gas (R T_ref = 189 * 293.15, CO2-like) in
    equal mass shares."""
    w = bubble_collapse(kind, n=(n[0], n[1]), p_inf=p_inf, steps=steps, **scheme)
    L = 4e-3
    w.name = f"{kind}_bubble_collapse3d_{n[0]}x{n[1]}x{n[2]}"
    w.ndim = 3
    w.n = [n[0], n[1], n[2]]
    w.lo = [-0.5 * L, 0.0, -0.5 * L]
    w.hi = [0.5 * L, L * n[1] / n[0], 0.5 * L * n[2] / n[0]]
    w.bc = [[BC_OUTFLOW] * 2, [BC_REFLECT, BC_OUTFLOW], [BC_OUTFLOW] * 2]
    if gases == 2:
        w.comps = [AIR_BARO, comp_baro_gas(188.9, 293.15), w.comps[1]]
        w.liquid = 2
    return w


def _split_gas(W, w):
    """equal mass shares of the two gases (3D, gases = 2)"""
    if w.ncomp == 3:
        g = W[w.ndim + 2].copy()
        W[w.ndim + 2] = 0.5 * g
        W[w.ndim + 3] = 0.5 * g
    return W


def bubble_collapse(kind="vapour", n=(1000, 1000), p_inf=1e7, steps=2000, **scheme):
    """Gas / vapour bubble collapse near a wall (Sec. 4.9): bubble radius
    R = 400 um centred H = 440 um above a wall at y = 0, on a 4 x 4 mm box
    ([-2, 2] x [0, 4] mm; n = 1000 gives the paper's finest 4 um cells
    everywhere), barotropic closure (Sec. 2.2).  Gas bubble: air at
    3000 Pa.  Vapour bubble: the liquid-vapour mixture at the capped vapour
    fraction (0.995), whose barotropic pressure is 6.7 Pa (p_sat = 1342 Pa).
    Ambient liquid p_inf = 10 MPa with the 1/r pressure ramp, at rest; wall
    below, outflow elsewhere; App. D switch off, THINC on.  CFL 0.4.  The
    FP32-mixed form's pressure offset is p_sat.  The passive internal
    energy starts uniform at 4.2e5 J/kg (about c_v T of water)."""
    nx, ny = n
    L = 4e-3
    liq = WATER_BARO
    rho_m = liq["rho_sl"] - 0.995 * (liq["rho_sl"] - liq["rho_sv"])
    p_b = 3000.0 if kind == "gas" else liq["psat"] * rho_m / liq["rho_sl"]
    # the FP32 arithmetic carries p - p_sat: vapour regions sit a few Pa above 0
    sch = default_scheme(**dict(dict(p_ref=liq["psat"]), **scheme))
    return Workload(
        name=f"{kind}_bubble_collapse_{nx}x{ny}", ndim=2, n=[nx, ny, 1], lo=[-0.5 * L, 0.0, 0.0],
        hi=[0.5 * L, L * ny / nx, 1.0], bc=[[BC_OUTFLOW] * 2, [BC_REFLECT, BC_OUTFLOW], [BC_PERIODIC] * 2],
        comps=[AIR_BARO, liq], liquid=1, scheme=sch, steps=steps, cfl=0.4, init="collapse",
        params=dict(R=400e-6, H=440e-6, p_b=p_b, p_inf=p_inf, e=4.2e5, gas=(kind == "gas"), width=1.5))
