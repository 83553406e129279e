"""The benchmark's roofline accounting (host arithmetic, no GPU): the
compulsory bytes of a stage are the ideal single-pass design's per
cell-update bytes over four stages (64 B per conserved field in the mixed
form, 88 B in FP64), the design bytes follow the kernel's own inputs and
outputs, and the FP64 flops come from the oracle's op-count table."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2304_00140_gb300 import workloads as wl  # noqa: E402

MIXED, FP64 = 1, 0


def _job(w):
    return bench.Job(w.name, [w])


@pytest.mark.parametrize("w,nv", [(wl.shock_bubble(), 5), (wl.jet3d(n=(64, 32, 32)), 7)])
def test_compulsory_bytes_per_stage(w, nv):
    """Per cell-update: FP64 reads q^0 once, every stage reads q^{k-1} (and
    q^0 from stage 2 on) and writes q^k, 8 bytes a value: 2 + 3 + 3 + 3 = 11
    values = 88 B per field.  The mixed form keeps q^A, q^B in 4 bytes:
    (8 + 4) + 2 (4 + 8 + 4) + (4 + 8 + 8) = 64 B per field.  A stage is a
    quarter of that."""
    job = _job(w)
    assert job.nvar == nv
    assert bench._compulsory_stage_bytes(job, MIXED) == job.cells * nv * 64 / 4
    assert bench._compulsory_stage_bytes(job, FP64) == job.cells * nv * 88 / 4
    if w.ndim == 2:
        assert bench._compulsory_stage_bytes(job, MIXED) / job.cells == 80.0
        assert bench._compulsory_stage_bytes(job, FP64) / job.cells == 110.0


def test_design_bytes_follow_the_kernels_inputs_and_outputs():
    """fused kernel: q^{k-1} and q^0 read, q^k written, 8 bytes a value;
    tiled kernel: the primitives read once (4 or 8 bytes), q^0 read and q^k
    written"""
    job = _job(wl.shock_bubble())
    assert bench._design_stage_bytes(job, MIXED, fused=True) == job.cells * 3 * 5 * 8
    np_ = bench._nprim(job.w)
    assert np_ == 5
    assert bench._design_stage_bytes(job, MIXED) == job.cells * (np_ * 4 + 2 * 5 * 8)
    assert bench._design_stage_bytes(job, FP64) == job.cells * (np_ * 8 + 2 * 5 * 8)


def test_primitive_fields_per_scheme():
    """the primitive array's fields: W, then rho and c (App. D, gravity or the
    barotropic closure), the liquid fraction (App. D or CSF), mu and k_c
    (viscous terms), the vapour fraction (barotropic closure)"""
    assert bench._nprim(wl.advection(n=8)) == 5
    assert bench._nprim(wl.advection(n=8, iles=1)) == 8
    assert bench._nprim(wl.advection(n=8, sigma=0.07)) == 6
    assert bench._nprim(wl.jet3d(n=(16, 8, 8))) == 7 + 3
    assert bench._nprim(wl.rising_bubble(2, n=(16, 32))) == 5 + 2 + 1 + 2
    assert bench._nprim(wl.bubble_collapse("vapour", n=(8, 8))) == 5 + 2 + 1


def test_fp64_flops_come_from_the_op_count_table():
    job = _job(wl.shock_bubble())
    fl = bench._alg_flops_per_cell(job)
    assert fl is not None and 300.0 < fl < 800.0
    assert bench._alg_flops_per_cell(job, fused=True) is None
