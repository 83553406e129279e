"""Pins of the oracle's capillary-jump surface tension (the Sec. 3.5
alternative to the CSF force: the contact's pressure jump [P] = sigma k
[alpha] inside the Riemann solver), no GPU.

The face balance: when the two cells' pressures differ by exactly the
Laplace jump sigma kappa (alpha_i - alpha_i+1), no mass crosses the face and
each side sees its own pressure (a discretely balanced surface force).  The
force the face jumps exert on the cells, integrated along a ray through a
static drop, is the Laplace jump sigma/R (2D) and 2 sigma/R (3D) (Eq. 4-4,
App. C), as for the CSF force."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl
from tests.test_oracle_csf import RHO_WATER, _drop


def _capj(w):
    w.scheme = dict(w.scheme, st_model=1)
    return oracle.Oracle(w)


@pytest.mark.parametrize("kappa", [4000.0, -2500.0])
def test_face_at_the_laplace_balance_is_stationary(kappa):
    w = wl.droplet(n=16, sigma=0.07)
    o = _capj(w)
    sigma = w.scheme["sigma"]
    p_gas = 2e5
    p_liq = p_gas + sigma * kappa          # alpha_L = 1 (liquid), alpha_R = 0
    liq = [0.0, 0.0, p_liq, 300.0, 0.0]    # Y_air = 0
    gas = [0.0, 0.0, p_gas, 300.0, 1.0]
    F, G = o.face_flux_kappa(0, [liq, liq, gas, gas], kappa, kappa, [1.0, 0.0])
    rho_l = o.forward(p_liq, 300.0, [0.0])[0]
    assert abs(F[0]) <= 1e-12 * rho_l                       # no mass crosses: u* = 0
    assert abs((F[1] - G[0]) - p_liq) <= 1e-12 * p_liq       # the liquid side sees p_liq
    assert abs((F[1] + G[0]) - p_gas) <= 1e-12 * p_gas       # the gas side sees p_gas
    # the same face without the jump term is not at rest
    w0 = wl.droplet(n=16, sigma=0.07)
    F0 = oracle.Oracle(w0).face_flux(0, [liq, liq, gas, gas])
    assert abs(F0[0]) > 1e-6 * rho_l


def test_capillary_force_laplace_jump_2d():
    n = 96
    o, q, alpha, dx = _drop(2, n, 32)
    o = _capj(o.w)
    S = o.capillary_force(q)
    Req = np.sqrt(alpha.sum() * dx * dx / np.pi)
    c = n // 2
    for comp, ray in ((0, S[0, 0, c, c:]), (1, S[1, 0, c:, c])):
        jump = -ray.sum() * dx
        assert abs(jump / (1.0 / Req) - 1.0) < 0.02, jump * Req


def test_capillary_force_laplace_jump_3d():
    n = 64
    o, q, alpha, dx = _drop(3, n, 24)
    o = _capj(o.w)
    S = o.capillary_force(q)
    Req = (alpha.sum() * dx ** 3 * 3.0 / (4.0 * np.pi)) ** (1.0 / 3.0)
    c = n // 2
    jump = -S[0, c, c, c:].sum() * dx
    assert abs(jump / (2.0 / Req) - 1.0) < 0.02, jump * Req / 2


def test_capillary_model_replaces_the_csf_source():
    """with the jump model the stage carries no CSF volume source: a
    single-phase state with sigma > 0 (no interface, no jump) steps exactly
    like sigma = 0, and on a drop the two models differ"""
    w = wl.droplet(n=24, A=0.15, sigma=30.0)
    W = w.primitives()
    W[4] = 0.0                                  # water everywhere
    o1 = _capj(wl.droplet(n=24, A=0.15, sigma=30.0))
    o0 = oracle.Oracle(wl.droplet(n=24, A=0.15, sigma=0.0))
    q = o0.prim_to_cons(W)
    dt = 0.3 * o0.dt(q, 1.0)
    assert np.array_equal(o1.stage(1, dt, q, q), o0.stage(1, dt, q, q))
    wd = wl.droplet(n=24, A=0.15, sigma=30.0)
    qd = o0.prim_to_cons(wd.primitives())
    a = _capj(wl.droplet(n=24, A=0.15, sigma=30.0)).stage(1, dt, qd, qd)
    b = oracle.Oracle(wd).stage(1, dt, qd, qd)
    assert np.abs(a - b).max() > 0


@pytest.mark.parametrize("kappa", [4000.0, -2500.0])
def test_smooth_face_at_the_laplace_balance_is_stationary(kappa):
    """The same balance on an App. D smooth face (f = 0, Eq. D.5 with the
    jump in the contact condition): across a pressure step Delta^3 p with
    the scale 1/2 equals the step p_L - p_R, so the jump J cancels it and no
    mass crosses, as on the upwind branch."""
    w = wl.droplet(n=16, sigma=0.07)
    w.scheme = dict(w.scheme, iles=1)
    o = _capj(w)
    sigma = w.scheme["sigma"]
    p_gas = 2e5
    p_liq = p_gas + sigma * kappa
    liq = [0.0, 0.0, p_liq, 300.0, 0.0]
    gas = [0.0, 0.0, p_gas, 300.0, 1.0]
    rl, _, cl, _ = o.forward(p_liq, 300.0, [0.0])
    rg, _, cg, _ = o.forward(p_gas, 300.0, [1.0])
    F, G = o.face_flux_kappa(0, [liq, liq, gas, gas], kappa, kappa, [1.0, 0.0], rho4=[rl, rl, rg, rg],
                             c4=[cl, cl, cg, cg], f=0)
    assert abs(F[0]) <= 1e-12 * rl
    assert G[0] == 0.5 * sigma * kappa * (0.0 - 1.0)
