"""The App. D sensor (Eq. D.4) on its own: the flags diagnostic
(FV_DIAG_FLAGS, the stage kernel's sensor function over the primitive
arrays) against the oracle's sensor, cell by cell.  The FP64 form takes the
same decisions (bit-exact flags); the FP32-mixed form decides in FP32 and
may differ only on cells within rounding of a threshold."""
import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl
from tests.test_gpu_baro import _sheared

pytestmark = pytest.mark.gpu

CASES = {
    "2d_2comp": lambda: wl.random_state(n=(61, 47), iles=1),
    "2d_3comp_bc": lambda: wl.random_state(n=(40, 33), ncomp=3, iles=1,
                                           bc=[[wl.BC_REFLECT, wl.BC_OUTFLOW], [wl.BC_OUTFLOW, wl.BC_REFLECT], [0, 0]]),
    "3d_3comp": lambda: wl.random_state(n=(21, 18, 23), ndim=3, ncomp=3, iles=1),
    "jet3d_inflow": lambda: wl.jet3d(n=(40, 24, 24)),
}


def _flags(w, precision, W=None, inflow_u=None):
    o = oracle.Oracle(w, inflow_u=inflow_u)
    q = o.prim_to_cons(w.primitives() if W is None else W)
    s = fv.Solver(w, precision=precision, inflow_u=[inflow_u] if inflow_u is not None else None)
    s.set_state(q)
    return s.sensor_flags(), o.sensor(q).astype(np.uint8)


@pytest.mark.parametrize("name", sorted(CASES))
def test_sensor_flags_match_oracle(name):
    w = CASES[name]()
    u = wl.jet_inflow_velocity(w) if w.inflow else None
    got, ref = _flags(w, fv.FV_FP64, inflow_u=u)
    assert 0 < ref.sum() < ref.size or name == "jet3d_inflow"
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]
    got_m, _ = _flags(w, fv.FV_MIXED, inflow_u=u)
    assert (got_m != ref).mean() < 1e-3


def test_sensor_flags_barotropic_vapour_sensor():
    w, W = _sheared("vapour", 1)
    got, ref = _flags(w, fv.FV_FP64, W)
    assert 0 < ref.sum() < ref.size
    assert np.array_equal(got, ref)


def test_sensor_flags_need_app_d_mode():
    s = fv.Solver(wl.random_state(n=(16, 16)), precision=fv.FV_FP64)
    s.set_state(wl.random_state(n=(16, 16)).primitives(), kind=fv.FV_PRIMITIVE)
    with pytest.raises(fv.FVError) as ei:
        s.sensor_flags()
    assert ei.value.status == fv.FV_ERR_ARG
