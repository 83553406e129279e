"""The kernels' bounded waits (TMA copies complete on an mbarrier polled
with a limit): a wait that never completes must give up, leave the timeout
bit in the device error word and leave the device usable.  No copy is made
to fail: the probe waits on a barrier that nothing arrives at."""
import ctypes as C

import pytest

from paper_2304_00140_gb300 import fv, workloads as wl

pytestmark = pytest.mark.gpu

FV_ERRBIT_TIMEOUT = 4


def test_bounded_wait_gives_up_and_device_stays_usable():
    L = fv.load()
    err = C.c_int(0)
    assert L.fv_wait_selftest(2000, C.byref(err)) == fv.FV_OK
    assert err.value & FV_ERRBIT_TIMEOUT
    # the context is intact: a 3D mixed step (TMA waits) runs cleanly afterwards
    w = wl.random_state(n=(20, 14, 11), ndim=3)
    s = fv.Solver(w, precision=fv.FV_MIXED)
    s.set_state(w.primitives(), kind=fv.FV_PRIMITIVE)
    s.step(2, w.cfl)
    assert s.error_word() == 0


def test_wait_selftest_rejects_bad_arguments():
    L = fv.load()
    err = C.c_int(0)
    assert L.fv_wait_selftest(0, C.byref(err)) == fv.FV_ERR_ARG


def test_fp64_probe_reports_a_plausible_rate():
    """the FP64 rate probe behind the FP64 form's roofline: a positive rate
    well below the FP32 rate (GB300 issues a few FP64 FMA per SM clock)"""
    L = fv.load()
    ms, fl = C.c_double(), C.c_double()
    assert L.fv_probe_fp64(152, 256, 256, C.byref(ms), C.byref(fl)) == fv.FV_OK
    assert ms.value > 0 and fl.value == 2 * 8 * 152 * 256 * 256
    tflops = fl.value / (ms.value * 1e-3) / 1e12
    assert 0.05 < tflops < 20.0, tflops
    assert L.fv_probe_fp64(0, 256, 1, C.byref(ms), C.byref(fl)) == fv.FV_ERR_ARG
