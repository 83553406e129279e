"""Exact solution of the 1D Riemann problem for two stiffened gases
(each material obeys p + pinf = (gamma - 1) rho e - pinf..., i.e. the
ideal-gas exact solver with p -> p + pinf on each side; Toro, "Riemann
Solvers and Numerical Methods for Fluid Dynamics", ch. 4, extended to
stiffened gases as in Ivings, Causon & Toro 1998).  Test helper only."""
import math

from scipy.optimize import brentq


class Side:
    def __init__(self, rho, u, p, gamma, pinf):
        self.rho, self.u, self.p, self.g, self.pi = rho, u, p, gamma, pinf
        self.c = math.sqrt(gamma * (p + pinf) / rho)

    def f(self, ps):
        g, pi, pk, rk = self.g, self.pi, self.p, self.rho
        if ps > pk:  # shock
            A = 2.0 / ((g + 1.0) * rk)
            B = (g - 1.0) / (g + 1.0) * (pk + pi)
            return (ps - pk) * math.sqrt(A / (ps + pi + B))
        return 2.0 * self.c / (g - 1.0) * (((ps + pi) / (pk + pi)) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def solve(L: Side, R: Side):
    fn = lambda p: L.f(p) + R.f(p) + R.u - L.u
    lo = -min(L.pi, R.pi) + 1e-9 * max(1.0, min(L.pi, R.pi))
    hi = max(L.p, R.p) * 10 + 1.0
    while fn(hi) < 0:
        hi *= 2
    ps = brentq(fn, lo, hi, xtol=1e-14 * hi, rtol=1e-15, maxiter=500)
    us = 0.5 * (L.u + R.u) + 0.5 * (R.f(ps) - L.f(ps))
    return ps, us


def sample(L: Side, R: Side, ps, us, xi):
    """(rho, u, p, side) at similarity coordinate xi = x / t; side 0 = left material."""
    if xi <= us:
        K, s = L, -1.0
    else:
        K, s = R, 1.0
    g, pi = K.g, K.pi
    pr = (ps + pi) / (K.p + pi)
    if ps > K.p:  # shock
        S = K.u + s * K.c * math.sqrt((g + 1.0) / (2.0 * g) * pr + (g - 1.0) / (2.0 * g))
        if (s < 0 and xi <= S) or (s > 0 and xi >= S):
            return K.rho, K.u, K.p, 0 if s < 0 else 1
        gm = (g - 1.0) / (g + 1.0)
        return K.rho * (pr + gm) / (gm * pr + 1.0), us, ps, 0 if s < 0 else 1
    cs = K.c * pr ** ((g - 1.0) / (2.0 * g))
    head = K.u + s * K.c
    tail = us + s * cs
    if (s < 0 and xi <= head) or (s > 0 and xi >= head):
        return K.rho, K.u, K.p, 0 if s < 0 else 1
    if (s < 0 and xi >= tail) or (s > 0 and xi <= tail):
        return K.rho * pr ** (1.0 / g), us, ps, 0 if s < 0 else 1
    # inside the fan
    a = 2.0 / (g + 1.0) - s * (g - 1.0) / ((g + 1.0) * K.c) * (K.u - xi)
    rho = K.rho * a ** (2.0 / (g - 1.0))
    u = 2.0 / (g + 1.0) * (-s * K.c + (g - 1.0) / 2.0 * K.u + xi)
    p = (K.p + pi) * a ** (2.0 * g / (g - 1.0)) - pi
    return rho, u, p, 0 if s < 0 else 1
