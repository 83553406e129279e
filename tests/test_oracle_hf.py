"""Pins of the oracle's height-function curvature (Sec. 3.5, the height
function option) against geometry: cell volume fractions of a circle,
a sphere and a tilted plane, integrated here by quadrature, give
kappa = 1/R (circle), 2/R (sphere) and 0 (plane) in the interface cells,
the circle's error falls as R grows, and the CSF force built on it gives the
Laplace jump sigma/R.  The Gaussian-smoothed curvature of the same fields is
reported beside it."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import workloads as wl

L = 1e-3
M = 400           # quadrature points per cell and direction (2D)


def _overlap(lo, hi, a, b):
    """length of [lo, hi] within [a, b] (arrays)"""
    return np.clip(np.minimum(hi, b) - np.maximum(lo, a), 0.0, None)


def _circle_fractions(n, xc, yc, R):
    """exact-to-quadrature area fraction of the disc in each cell: the
    chord length in y integrated over x (midpoint rule, M points a cell)"""
    dx = L / n
    xs = (np.arange(n * M) + 0.5) * (dx / M)
    h = np.sqrt(np.clip(R * R - (xs - xc) ** 2, 0.0, None))
    alpha = np.zeros((n, n))
    for j in range(n):
        y0, y1 = j * dx, (j + 1) * dx
        ov = _overlap(y0, y1, yc - h, yc + h)                 # per x sample
        alpha[j] = ov.reshape(n, M).mean(axis=1) / dx
    return alpha[None]


def _halfplane_fractions(n, a, b):
    """area fraction below the line y = b + a (x - L/2)"""
    dx = L / n
    xs = (np.arange(n * M) + 0.5) * (dx / M)
    yl = b + a * (xs - 0.5 * L)
    alpha = np.zeros((n, n))
    for j in range(n):
        ov = np.clip(yl - j * dx, 0.0, dx)
        alpha[j] = ov.reshape(n, M).mean(axis=1) / dx
    return alpha[None]


def _sphere_fractions(n, c0, R, m=48):
    """volume fraction of the ball: the z-chord integrated over (x, y) with
    m x m midpoints in cells the sphere crosses, 0 / 1 elsewhere"""
    dx = L / n
    ctr = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(ctr, ctr, ctr, indexing="ij")
    r = np.sqrt((X - c0) ** 2 + (Y - c0) ** 2 + (Z - c0) ** 2)
    alpha = (r < R).astype(float)
    near = np.abs(r - R) < 0.9 * dx
    s = (np.arange(m) + 0.5) / m
    for k, j, i in np.argwhere(near):
        xs = (i + s) * dx
        ys = (j + s) * dx
        XX, YY = np.meshgrid(xs, ys, indexing="ij")
        h = np.sqrt(np.clip(R * R - (XX - c0) ** 2 - (YY - c0) ** 2, 0.0, None))
        ov = _overlap(k * dx, (k + 1) * dx, c0 - h, c0 + h)
        alpha[k, j, i] = ov.mean() / dx
    return alpha


def _state(ndim, n, alpha, curvature=1, sigma=1.0):
    w = wl.Workload(name="hf", ndim=ndim, n=[n, n, n if ndim == 3 else 1], lo=[0, 0, 0],
                    hi=[L, L, L if ndim == 3 else 1.0], bc=[[0, 0]] * 3, comps=[wl.AIR, wl.WATER], liquid=1,
                    scheme=wl.default_scheme(sigma=sigma, curvature=curvature), steps=1, cfl=0.4, init="random")
    o = oracle.Oracle(w)
    rl = o.forward(1e5, 300.0, np.array([0.0]))[0]
    rg = o.forward(1e5, 300.0, np.array([1.0]))[0]
    Yl = alpha * rl / (alpha * rl + (1 - alpha) * rg)
    W = np.zeros((w.nvar,) + alpha.shape)
    W[ndim] = 1e5
    W[ndim + 1] = 300.0
    W[ndim + 2] = 1.0 - Yl                       # air tracked
    return o, o.prim_to_cons(W)


def _circle_errors(Rcells, n=64, curvature=1):
    R = Rcells * L / n
    c0 = 0.5 * L + 0.17 * L / n                  # off the grid's symmetry
    alpha = _circle_fractions(n, c0, c0, R)
    o, q = _state(2, n, alpha, curvature)
    k = o.curvature(q)
    band = (alpha > 0.02) & (alpha < 0.98)
    return np.abs(k[band] * R - 1.0)


def test_circle_curvature():
    e = _circle_errors(16)
    assert e.max() < 0.03 and e.mean() < 0.01, (e.max(), e.mean())


def test_circle_curvature_converges():
    e8, e16, e24 = (_circle_errors(r, n=80).mean() for r in (8, 16, 24))
    assert e16 < e8 and e24 < e16, (e8, e16, e24)


def test_gaussian_curvature_is_the_coarser_estimate():
    """context for the option: the smoothed-normal curvature of the same
    sharp circle has a larger error than the height function"""
    e_hf = _circle_errors(16).mean()
    e_g = _circle_errors(16, curvature=0).mean()
    assert e_hf < e_g, (e_hf, e_g)


def test_tilted_plane_has_zero_curvature():
    n = 40
    a, b = 0.37, 0.52
    alpha = _halfplane_fractions(n, a, b * L)
    o, q = _state(2, n, alpha)
    k = o.curvature(q)
    band = (alpha > 0.02) & (alpha < 0.98)
    band[:, :, :3] = band[:, :, -3:] = False      # away from the periodic seam
    assert np.abs(k[band]).max() * L < 1e-9


def test_sphere_curvature():
    n = 32
    R = 9.0 * L / n
    c0 = 0.5 * L + 0.13 * L / n
    alpha = _sphere_fractions(n, c0, R)
    o, q = _state(3, n, alpha)
    k = o.curvature(q)
    band = (alpha > 0.05) & (alpha < 0.95)
    e = np.abs(k[band] * R / 2.0 - 1.0)
    assert e.mean() < 0.03 and np.median(e) < 0.02, (e.mean(), np.median(e), e.max())


def test_laplace_jump_with_height_function():
    """sigma kappa grad(alpha) integrated along a ray from the centre gives
    p_in - p_out = sigma / R"""
    n, Rc = 96, 30
    R = Rc * L / n
    c0 = 0.5 * L + 0.21 * L / n
    alpha = _circle_fractions(n, c0, c0, R)
    o, q = _state(2, n, alpha, sigma=1.0)
    S = o.csf_source(q)
    dx = L / n
    jc = n // 2
    jump = -S[0, 0, jc, jc:].sum() * dx
    assert abs(jump * R - 1.0) < 0.02, jump * R


def test_quadratic_surface_on_an_anisotropic_grid():
    """The 3D height-function formula on heights it gets exactly: liquid
    below z = f(x, y), f quadratic with a cross term, on a grid whose three
    spacings differ.  The columns' liquid heights are the cell averages of
    f, whose central differences are f's exact derivatives at the column
    centre (H_x, H_y), 2a, 2b and c, so the curvature must be
    -(H_xx (1 + H_y^2) + H_yy (1 + H_x^2) - 2 H_xy H_x H_y)/(1 + H_x^2 + H_y^2)^(3/2)
    to rounding wherever the interface of all nine columns lies inside the
    five-cell window."""
    n = (10, 9, 14)
    dx = (1.0e-4, 0.7e-4, 0.5e-4)
    a, b, c, d, e = -300.0, 200.0, 150.0, 0.2, -0.15
    xc, yc, z0 = 5.1e-4, 3.2e-4, 3.4e-4
    w = wl.Workload(name="hf3", ndim=3, n=list(n), lo=[0, 0, 0], hi=[n[i] * dx[i] for i in range(3)],
                    bc=[[wl.BC_OUTFLOW] * 2] * 3, comps=[wl.AIR, wl.WATER], liquid=1,
                    scheme=wl.default_scheme(sigma=1.0, curvature=1), steps=1, cfl=0.4, init="random")
    o = oracle.Oracle(w)
    x = (np.arange(n[0]) + 0.5) * dx[0] - xc
    y = (np.arange(n[1]) + 0.5) * dx[1] - yc
    Yg, Xg = np.meshgrid(y, x, indexing="ij")
    favg = z0 + d * Xg + e * Yg + a * Xg ** 2 + b * Yg ** 2 + c * Xg * Yg + (a * dx[0] ** 2 + b * dx[1] ** 2) / 12.0
    k = np.arange(n[2])[:, None, None]
    alpha = np.clip((favg[None] - k * dx[2]) / dx[2], 0.0, 1.0)
    rl = o.forward(1e5, 300.0, np.array([0.0]))[0]
    rg = o.forward(1e5, 300.0, np.array([1.0]))[0]
    Yl = alpha * rl / (alpha * rl + (1 - alpha) * rg)
    W = np.zeros((w.nvar,) + alpha.shape)
    W[3], W[4], W[5] = 1e5, 300.0, 1.0 - Yl
    q = o.prim_to_cons(W)
    kap = o.curvature(q)
    axis, _ = o.hf_axis(q)
    layer = np.floor(favg / dx[2]).astype(int)          # the column's partly filled cell
    checked = 0
    for kk, j, i in np.argwhere((alpha > 0) & (alpha < 1)):
        if not (1 <= i < n[0] - 1 and 1 <= j < n[1] - 1 and 2 <= kk < n[2] - 2) or axis[kk, j, i] != 2:
            continue
        if np.abs(layer[j - 1:j + 2, i - 1:i + 2] - kk).max() > 1:
            continue
        X, Y = Xg[j, i], Yg[j, i]
        Hx, Hy = d + 2 * a * X + c * Y, e + 2 * b * Y + c * X
        want = -(2 * a * (1 + Hy ** 2) + 2 * b * (1 + Hx ** 2) - 2 * c * Hx * Hy) / (1 + Hx ** 2 + Hy ** 2) ** 1.5
        assert kap[kk, j, i] == pytest.approx(want, rel=1e-8, abs=0), (kk, j, i)
        checked += 1
    assert checked > 20
