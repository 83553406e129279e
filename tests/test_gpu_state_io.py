"""State I/O through the C ABI: pageable host memory (staged through a device
buffer), page-locked host memory (read and written by the conversion kernels
directly) and device memory must give bit-identical states, for conserved
and primitive input, in both forms."""
import ctypes as C

import numpy as np
import pytest

from paper_2304_00140_gb300 import fv, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
@pytest.mark.parametrize("kind", [fv.FV_CONSERVED, fv.FV_PRIMITIVE])
def test_state_io_paths_agree(precision, kind):
    import torch
    w = wl.random_state(n=(37, 23), bc=[[wl.BC_REFLECT, wl.BC_OUTFLOW], [wl.BC_PERIODIC] * 2, [0, 0]])
    s = fv.Solver(w, precision=precision)
    s.set_state(w.primitives(), kind=fv.FV_PRIMITIVE)
    x = s.get_state(kind)
    L = s.L

    # pageable host memory
    s.set_state(x, kind=kind)
    ref = s.get_state(kind)

    # page-locked host memory
    pin = torch.from_numpy(x.copy()).pin_memory()
    out = torch.zeros_like(pin).pin_memory()
    assert L.fv_set_state(s.ctx, 0, kind, C.c_void_p(pin.data_ptr())) == fv.FV_OK
    assert L.fv_get_state(s.ctx, 0, kind, C.c_void_p(out.data_ptr())) == fv.FV_OK
    assert np.array_equal(out.numpy(), ref)

    # device memory
    dev = torch.from_numpy(x.copy()).cuda()
    s.set_state_device(dev, kind=kind)
    dout = torch.zeros_like(dev)
    s.get_state_device(dout, kind=kind)
    torch.cuda.synchronize()
    assert np.array_equal(dout.cpu().numpy(), ref)

    # and a step from the page-locked state equals a step from the pageable one
    s.set_state(x, kind=kind)
    s.step(2, w.cfl)
    a = s.get_state()
    assert L.fv_set_state(s.ctx, 0, kind, C.c_void_p(pin.data_ptr())) == fv.FV_OK
    s.step(2, w.cfl)
    assert np.array_equal(s.get_state(), a)
