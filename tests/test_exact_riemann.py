"""Pins of the exact two-stiffened-gas Riemann solver the oracle's pins use
(no GPU): the star states it returns satisfy the conditions that define the
exact solution, independently of how it finds them.  Across a shock, the
Rankine-Hugoniot jumps of mass, momentum and energy in the shock frame;
across a rarefaction, constant entropy (p + pinf)/rho^gamma and the
Riemann invariant u +/- 2c/(gamma - 1) (left/right fan); the fan is
continuous at its head and tail; and the contact carries equal p and u."""
import math

import numpy as np
import pytest

from tests import exact_riemann as er

GASES = [(1.4, 0.0), (6.12, 3.43e8), (2.35, 4.0e8), (1.3, 1e5)]


def _e(rho, p, g, pi):
    """specific internal energy of a stiffened gas, p = (g-1) rho e - g pi"""
    return (p + g * pi) / ((g - 1.0) * rho)


def _star(K, ps, us, s):
    """density behind the left (s = -1) or right (s = +1) wave"""
    g, pi = K.g, K.pi
    pr = (ps + pi) / (K.p + pi)
    if ps > K.p:
        gm = (g - 1.0) / (g + 1.0)
        return K.rho * (pr + gm) / (gm * pr + 1.0)
    return K.rho * pr ** (1.0 / g)


def _cases():
    rng = np.random.default_rng(77)
    out = []
    for _ in range(60):
        (gl, pil), (gr, pir) = (GASES[i] for i in rng.integers(0, len(GASES), 2))
        pl = 10 ** rng.uniform(4, 9)
        pr = 10 ** rng.uniform(4, 9)
        rl = (10 ** rng.uniform(0, 3)) if pil == 0 else 10 ** rng.uniform(2.5, 3.2)
        rr = (10 ** rng.uniform(0, 3)) if pir == 0 else 10 ** rng.uniform(2.5, 3.2)
        ul, ur = rng.uniform(-200, 200, 2)
        out.append((er.Side(rl, ul, pl, gl, pil), er.Side(rr, ur, pr, gr, pir)))
    return out


def test_star_states_satisfy_the_jump_conditions():
    checked = {"shock": 0, "fan": 0}
    for L, R in _cases():
        try:
            ps, us = er.solve(L, R)
        except ValueError:
            continue                      # vacuum-generating data have no star state
        for K, s in ((L, -1.0), (R, 1.0)):
            g, pi = K.g, K.pi
            rs = _star(K, ps, us, s)
            if ps > K.p:
                # shock speed from mass conservation, then momentum and energy
                S = (rs * us - K.rho * K.u) / (rs - K.rho)
                m = K.rho * (K.u - S)
                assert m == pytest.approx(rs * (us - S), rel=1e-9, abs=0)
                mom_scale = abs(m * (K.u - S)) + K.p + ps + pi
                assert abs((m * (K.u - S) + K.p) - (m * (us - S) + ps)) <= 1e-9 * mom_scale
                hK = _e(K.rho, K.p, g, pi) + K.p / K.rho + 0.5 * (K.u - S) ** 2
                hs = _e(rs, ps, g, pi) + ps / rs + 0.5 * (us - S) ** 2
                assert hK == pytest.approx(hs, rel=1e-9, abs=0)
                checked["shock"] += 1
            else:
                assert (K.p + pi) / K.rho ** g == pytest.approx((ps + pi) / rs ** g, rel=1e-10, abs=0)
                cs = math.sqrt(g * (ps + pi) / rs)
                # left fan: u + 2c/(g-1) is constant across it; right fan: u - 2c/(g-1)
                assert K.u - s * 2 * K.c / (g - 1) == pytest.approx(us - s * 2 * cs / (g - 1), rel=1e-9,
                                                                    abs=1e-9 * (K.c + cs))
                # the fan is continuous at its head and its tail
                head, tail = K.u + s * K.c, us + s * cs
                eps = 1e-9 * (abs(head) + abs(tail) + K.c)
                rin = er.sample(L, R, ps, us, head - s * eps)[0]
                rout = er.sample(L, R, ps, us, head + s * eps)[0]
                assert rin == pytest.approx(rout, rel=1e-6)
                if abs(tail - head) > 10 * eps:
                    rin = er.sample(L, R, ps, us, tail + s * eps)[0]
                    rout = er.sample(L, R, ps, us, tail - s * eps)[0]
                    assert rin == pytest.approx(rout, rel=1e-6)
                checked["fan"] += 1
        # the contact: each side's star state at xi = us -/+ 0
        a = er.sample(L, R, ps, us, us - 1e-9 * (abs(us) + 1.0))
        b = er.sample(L, R, ps, us, us + 1e-9 * (abs(us) + 1.0))
        assert a[3] == 0 and b[3] == 1
        assert a[1] == b[1] == us and a[2] == b[2] == ps
        # the sampled star densities are the ones checked above
        assert a[0] == pytest.approx(_star(L, ps, us, -1.0), rel=1e-13, abs=0)
        assert b[0] == pytest.approx(_star(R, ps, us, 1.0), rel=1e-13, abs=0)
    assert checked["shock"] > 20 and checked["fan"] > 20
