"""State I/O through the C ABI: pageable host memory (staged through a device
buffer), page-locked host memory (read and written by the conversion kernels
directly) and device memory must give bit-identical states, for conserved
and primitive input, in both forms."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2304_00140_gb300 import fv, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
@pytest.mark.parametrize("kind", [fv.FV_CONSERVED, fv.FV_PRIMITIVE])
@pytest.mark.parametrize("n", [(37, 23), (36, 22)])   # odd cell count: one value a time; even: 16-byte accesses
def test_state_io_paths_agree(precision, kind, n):
    import torch
    w = wl.random_state(n=n, bc=[[wl.BC_REFLECT, wl.BC_OUTFLOW], [wl.BC_PERIODIC] * 2, [0, 0]])
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


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_all_cases_io_matches_per_case(precision):
    """fv_set_state_all / fv_get_state_all on a batch of uneven cases: the
    concatenated blocks equal the per-case calls, from page-locked memory
    (one kernel over all cases) and from pageable memory (case by case)."""
    import torch
    cases = [wl.droplet(n=n, A=a, sigma=20.0) for n, a in ((24, 0.1), (40, 0.2), (33, 0.05), (16, 0.15))]
    s = fv.Solver(cases, precision=precision)
    for i, c in enumerate(cases):
        s.set_state(c.primitives(), kind=fv.FV_PRIMITIVE, case=i)
    s.step(2, 0.4)
    per_case = np.concatenate([s.get_state(case=i).ravel() for i in range(len(cases))])
    assert np.array_equal(s.get_state_all(), per_case)                  # pageable
    L = s.L
    out = torch.zeros(per_case.size, dtype=torch.float64).pin_memory()
    assert L.fv_get_state_all(s.ctx, fv.FV_CONSERVED, C.c_void_p(out.data_ptr())) == fv.FV_OK
    assert np.array_equal(out.numpy(), per_case)                       # page-locked
    # set from page-locked memory, step, compare with the per-case set
    pin = torch.from_numpy(per_case.copy()).pin_memory()
    assert L.fv_set_state_all(s.ctx, fv.FV_CONSERVED, C.c_void_p(pin.data_ptr())) == fv.FV_OK
    s.step(2, 0.4)
    a = s.get_state_all()
    off = 0
    for i, c in enumerate(cases):
        n = c.nvar * c.cells
        s.set_state(per_case[off:off + n].reshape(s.shape(i)), case=i)
        off += n
    s.step(2, 0.4)
    assert np.array_equal(s.get_state_all(), a)


@pytest.mark.parametrize("precision", [fv.FV_FP64, fv.FV_MIXED])
def test_pipelined_io_equals_blocking_calls(precision):
    """fv_upload_async / fv_commit_upload / fv_download_async: a stream of
    three different input states, each stepped twice while the next one is
    uploaded and the previous result downloaded, gives bit for bit what the
    blocking fv_set_state_all / fv_step / fv_get_state_all calls give; a
    second upload before a commit is refused"""
    import torch
    cases = [wl.random_state(n=(40, 24), seed=s) for s in (11, 12)]
    inputs = []
    for sd in (1, 2, 3):
        qs = [oracle.Oracle(c).prim_to_cons(wl.random_state(n=(40, 24), seed=sd * 7 + k).primitives())
              for k, c in enumerate(cases)]
        inputs.append(np.concatenate([q.ravel() for q in qs]))
    ref = []
    s = fv.Solver(cases, precision=precision)
    for q in inputs:
        s.set_state_all(q)
        s.step(2, 0.4)
        ref.append(s.get_state_all())
    s.close()
    s = fv.Solver(cases, precision=precision)
    L = s.L
    h_in = [torch.from_numpy(q.copy()).pin_memory() for q in inputs]
    h_out = [torch.zeros_like(h_in[0]).pin_memory() for _ in inputs]
    assert L.fv_upload_async(s.ctx, C.c_void_p(h_in[0].data_ptr())) == fv.FV_OK
    assert L.fv_upload_async(s.ctx, C.c_void_p(h_in[0].data_ptr())) == fv.FV_ERR_STATE
    for i in range(len(inputs)):
        assert L.fv_commit_upload(s.ctx) == fv.FV_OK
        if i + 1 < len(inputs):
            assert L.fv_upload_async(s.ctx, C.c_void_p(h_in[i + 1].data_ptr())) == fv.FV_OK
        assert L.fv_step_async(s.ctx, 2, 0.4) == fv.FV_OK
        assert L.fv_download_async(s.ctx, C.c_void_p(h_out[i].data_ptr())) == fv.FV_OK
    assert L.fv_io_wait(s.ctx) == fv.FV_OK
    for i in range(len(inputs)):
        assert np.array_equal(h_out[i].numpy(), ref[i]), i
    assert L.fv_commit_upload(s.ctx) == fv.FV_ERR_STATE
