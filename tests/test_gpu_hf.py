"""GPU parity with the FP64 oracle for the height-function curvature option
of the CSF force (Sec. 3.5), 2D and 3D, and the FP32-mixed form's accuracy;
a static drop run with both curvatures reports the Laplace pressure and the
parasitic velocity (the comparison of Sec. 4.7)."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl
from tests.helpers import cell_rel_diff, gpu_stage, rel_l1_vec

pytestmark = pytest.mark.gpu


CASES = {
    "droplet_2d": lambda: wl.droplet(n=(48, 44), A=0.15, sigma=30.0, curvature=1),
    "random_2d_iles_3comp": lambda: wl.random_state(n=(40, 33), ncomp=3, iles=1, sigma=5.0, curvature=1),
    "random_3d_iles_3comp": lambda: wl.random_state(n=(18, 17, 21), ndim=3, ncomp=3, iles=1, sigma=5.0,
                                                    curvature=1),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_hf_parity_fp64(name):
    """Every stage of three steps, each fed the oracle's own stage inputs so
    that a difference cannot propagate: the GPU stage matches the oracle to
    1e-10 per field in every cell, except where the height-function column
    axis is a near-tie -- the two largest central differences of the liquid
    fraction within 1e-12 of each other, where rounding may pick the other
    axis; such flips are counted and reported."""
    w = CASES[name]()
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    k_hf = o.curvature(q)
    w0 = CASES[name]()
    w0.scheme = dict(w0.scheme, curvature=0)
    assert np.abs(k_hf - oracle.Oracle(w0).curvature(q)).max() > 0     # the option changes kappa
    dt = 0.3 * o.dt(q, 1.0)
    flips = 0
    q0 = q
    for step in range(3):
        prev = q0
        for k in (1, 2, 3, 4):
            ref = o.stage(k, dt, q0, prev)
            got = gpu_stage(w, fv.FV_FP64, k, dt, q0, prev)
            bad = cell_rel_diff(got, ref) > 1e-10
            if bad.any():
                _, gap = o.hf_axis(prev)
                assert np.all(gap[bad] < 1e-12), (step, k, gap[bad].min(), np.argwhere(bad)[:5])
                flips += int(bad.sum())
            prev = ref
        q0 = prev
    print(f"{name}: {flips} cell(s) differed at a height-function axis near-tie")
    assert flips <= 3


def test_hf_mixed_accuracy_droplet():
    """FP32-mixed droplet with the height-function curvature after 60 steps:
    density, energy, mass fraction within 1e-4 relative L1 of the oracle"""
    w = wl.droplet(n=64, A=0.15, curvature=1)
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    s = fv.Solver(w, precision=fv.FV_MIXED)
    s.set_state(q)
    s.step(60, w.cfl)
    ref, _ = o.step(q, 60, w.cfl)
    e = rel_l1_vec(s.get_state(), ref, w.ndim)
    assert np.all(np.r_[e[:1], e[1 + w.ndim:]] < 1e-4), e


def test_static_drop_both_curvatures():
    """a drop at rest with the Laplace jump preset (sigma = 1 N/m, R = 25
    cells, tanh-smoothed over 1.5 cells): 400 steps (about six acoustic
    times of the drop) with each curvature.  Reported, not bounded tightly:
    at this time the drop still rings acoustically, so the measured jump and
    the largest velocity are a transient, and the 5-cell height-function
    columns only just span the smoothed interface.  Both stay bounded."""
    out = {}
    for curv in (0, 1):
        n, L = 100, 1e-3
        R = 0.25 * L
        w = wl.droplet(n=n, A=0.0, sigma=1.0, dp=1.0 / R, curvature=curv)
        s = fv.Solver(w, precision=fv.FV_FP64)
        s.set_state(w.primitives(), kind=fv.FV_PRIMITIVE)
        s.step(400, w.cfl)
        W = s.get_state(fv.FV_PRIMITIVE)
        u = np.sqrt(W[0] ** 2 + W[1] ** 2).max()
        p = W[2][0]
        jump = p[n // 2 - 3:n // 2 + 3, n // 2 - 3:n // 2 + 3].mean() - p[:5, :5].mean()
        out[curv] = (jump * R, u)
    print("static drop: (jump * R / sigma, max |u| m/s) smoothed-normal", out[0], "height function", out[1])
    for curv, (j, u) in out.items():
        assert np.isfinite(j) and abs(j - 1.0) < 0.8 and u < 10.0, (curv, j, u)
