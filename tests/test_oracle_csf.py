"""Pins of the oracle's CSF source (Sec. 2.3, Sec. 3.5, Eq. 3-9/3-10)
against the Laplace pressure jump of a static drop: the momentum balance
grad p = sigma kappa grad(alpha) integrated along a ray from the drop centre
gives p_in - p_out, which must be sigma/R in 2D (Eq. 4-4) and 2 sigma/R in
3D (App. C), with R the equivalent radius of the liquid volume."""
import numpy as np

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
