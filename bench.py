#!/usr/bin/env python
"""Benchmark of the All-Mach THINC-TDU step on one GB300 (or N replicas).

Workload: 2D shock-bubble interaction, 2048 x 1024 cells (water at 1e5 Pa /
300 K, air bubble of radius 0.2 mm, planar 1e9 Pa shock, reflective top and
bottom, outflow sides, CFL 0.4).  A step is one full four-stage LSRK step:
CFL reduction, then four stages of (boundary + primitive update, fused
sensor/reconstruction/TDU/Riemann/divergence/update pass).

The headline value is the FP32-mixed form; the FP64 form is measured in the
same run (``fp64`` key) with the L1 difference between the two.  Output: one
JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s, mixed vs FP64 on one GB300 at stated L1 error; % HBM roofline"
UNIT = "cell-updates/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=float(d["hbm_gbs"]), src="measured")
    return dict(hbm=6800.0, src="fallback")


def _workload(args):
    from paper_2304_00140_gb300 import workloads as wl
    return wl.shock_bubble(nx=args.nx, ny=args.ny)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# --------------------------------------------------------------- one form
def _algorithmic_stage_bytes(w, precision):
    """Compulsory HBM bytes of one stage_kernel launch: every interior cell's
    primitives read once (fp32 in the mixed form, fp64 otherwise), q^0 read
    and q^k written in FP64."""
    rs = 4 if precision == 1 else 8
    return w.cells * (w.nvar * rs + 2 * w.nvar * 8)


def run_form(w, W, precision, args, torch, dist, rank, world):
    from paper_2304_00140_gb300 import fv
    s = fv.Solver(w, precision=precision)
    s.set_state(W, kind=fv.FV_PRIMITIVE)
    stream = torch.cuda.current_stream()
    s.step_async(args.warmup, w.cfl)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device())
    time.sleep(0.25)
    l0 = s.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step_async(args.steps, w.cfl)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = s.launch_count() - l0
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    err = s.error_word()
    # per-kernel times with event pairs on the launching stream (no graph)
    kprof = max(4, min(args.steps, 50))
    s.profile(True)
    s.step_async(kprof, w.cfl)
    prof = s.profile_read()
    s.profile(False)
    state = s.get_state()
    res = dict(ms=ms, launches=launches, clocks=clocks, err=err, prof=prof, state=state, solver=s)
    return res


def e2e_form(w, precision, args, torch):
    """Same metric through the public API with host buffers: every step copies
    the state in from pinned host memory, advances one step and reads the
    state back."""
    import ctypes as C
    from paper_2304_00140_gb300 import fv
    s = fv.Solver(w, precision=precision)
    W = w.primitives()
    s.set_state(W, kind=fv.FV_PRIMITIVE)
    q = s.get_state()
    h_in = torch.from_numpy(q.copy()).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    L = s.L
    nsteps = max(3, min(args.steps, 30))
    L.fv_set_state(s.ctx, 0, fv.FV_CONSERVED, C.c_void_p(h_in.data_ptr()))
    L.fv_step(s.ctx, 1, w.cfl, None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(nsteps):
        st = L.fv_set_state(s.ctx, 0, fv.FV_CONSERVED, C.c_void_p(h_in.data_ptr()))
        st = st or L.fv_step_async(s.ctx, 1, w.cfl)
        st = st or L.fv_get_state(s.ctx, 0, fv.FV_CONSERVED, C.c_void_p(h_out.data_ptr()))
        if st:
            raise fv.FVError(st, L.fv_last_error(s.ctx).decode())
    t1 = time.perf_counter()
    nbytes = int(h_in.numel() * 8)
    s.close()
    return dict(value=w.cells * nsteps / (t1 - t0), unit=UNIT, h2d_bytes_per_step=nbytes,
                d2h_bytes_per_step=nbytes, steps=nsteps)


# ------------------------------------------------------------- CPU oracle
def oracle_window_step(o, q, dt, lo, hi):
    """one LSRK step of the oracle restricted to a window (stage k evaluated
    on the window grown by the stencil reach of the later stages)"""
    w = o.w
    prev = q
    for k in (1, 2, 3, 4):
        g = 2 * (4 - k)
        wl_ = [max(0, lo[d] - g) if d < w.ndim else 0 for d in range(3)]
        wh_ = [min(w.n[d], hi[d] + g) if d < w.ndim else 1 for d in range(3)]
        out = q.copy()
        o.stage(k, dt, q, prev, window=(wl_, wh_), out=out)
        prev = out
    return prev


def cpu_oracle_rate(w, rows, reps=1):
    """The FP64 oracle, as it stands, single-threaded on the host: one LSRK
    step on a band of ``rows`` full-width rows through the bubble."""
    import oracle
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    ny = w.n[1]
    y0 = max(0, ny // 2 - rows // 2)
    lo, hi = (0, y0, 0), (w.n[0], y0 + rows, 1)
    dt = 1e-12
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle_window_step(o, q, dt, lo, hi)
    t1 = time.perf_counter()
    cells = w.n[0] * rows * reps
    return cells / (t1 - t0), cells, t1 - t0


def run_reference(args):
    """--impl reference: the oracle (the only reference there is: the paper
    ships no code) timed on the host cores, each step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = _workload(args)
    import oracle
    o = oracle.Oracle(w)
    q = o.prim_to_cons(w.primitives())
    # band height sized so the whole run stays near two minutes of host time
    rows = args.ref_rows or int(min(64, max(2, 120.0 / ((args.steps + args.warmup) * 0.04))))
    ny = w.n[1]
    y0 = ny // 2 - rows // 2
    lo, hi = (0, y0, 0), (w.n[0], y0 + rows, 1)
    for _ in range(args.warmup):
        oracle_window_step(o, q, 1e-12, lo, hi)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_window_step(o, q, 1e-12, lo, hi)
    t1 = time.perf_counter()
    cells = w.n[0] * rows
    val = cells * args.steps / (t1 - t0)
    sample = f"one LSRK step per bench step on a {w.n[0]}x{rows} band of the {w.n[0]}x{ny} shock-bubble grid"
    line = dict(impl="reference", metric=METRIC, value=val, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * (t1 - t0) / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=w.name, grid=w.n[:2], band_rows=rows),
                cpu_baseline=dict(value=val, unit=UNIT, cores=1, kind="oracle", sample=sample),
                e2e=dict(value=val, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=192)
    ap.add_argument("--ref-rows", type=int, default=0)
    ap.add_argument("--fp64-steps", type=int, default=0, help="steps for the FP64 form (default: --steps)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)

    from paper_2304_00140_gb300 import fv
    fv.load()
    w = _workload(args)
    W = w.primitives()
    peaks = _peaks()

    mixed = run_form(w, W, fv.FV_MIXED, args, torch, dist, rank, world)
    fargs = argparse.Namespace(**vars(args))
    if args.fp64_steps:
        fargs.steps = args.fp64_steps
    f64 = run_form(w, W, fv.FV_FP64, fargs, torch, dist, rank, world)

    # accuracy of the mixed form against the FP64 form after the same steps
    # (both advanced warmup + steps + profiled steps from the same state)
    # relative L1 per conserved field; the momentum components are measured
    # against the L1 norm of the momentum vector (a component can be ~0)
    l1 = None
    if fargs.steps == args.steps:
        a, b = mixed["state"], f64["state"]
        nv = a.shape[0]
        den = np.abs(b).reshape(nv, -1).sum(1)
        den[1:1 + w.ndim] = np.sqrt((b[1:1 + w.ndim] ** 2).sum(0)).sum()
        l1 = (np.abs(a - b).reshape(nv, -1).sum(1) / den).tolist()

    def roof(res, precision):
        st = res["prof"]["stage"]
        avg_ms = st["ms"] / max(1, st["launches"])
        byt = _algorithmic_stage_bytes(w, precision)
        ach = byt / (avg_ms * 1e-3) / 1e9
        return dict(bound="hbm", achieved=ach, peak=peaks["hbm"], unit="GB/s", frac=ach / peaks["hbm"],
                    traffic=None, kernel="stage_kernel", avg_launch_ms=avg_ms,
                    algorithmic_bytes_per_launch=byt, peak_source=peaks["src"],
                    kernel_share={k: v["ms"] for k, v in res["prof"].items()})

    cells_all = w.cells * world
    val = cells_all * args.steps / (mixed["ms"] * 1e-3)
    v64 = cells_all * fargs.steps / (f64["ms"] * 1e-3)
    e2e = e2e_form(w, fv.FV_MIXED, args, torch) if rank == 0 else None
    if e2e is not None:
        e2e["value"] *= world

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cells, secs = cpu_oracle_rate(w, args.cpu_rows)
        cpu = dict(value=rate, unit=UNIT, cores=1, kind="oracle",
                   sample=f"one LSRK step of a {w.n[0]}x{args.cpu_rows} row band of the same grid "
                          f"({cells} cell-updates, {secs:.1f} s, single thread)")

    if rank == 0:
        line = dict(
            metric=METRIC, value=val, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=mixed["ms"] / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f32+f64", data="synthetic",
            config=dict(workload=w.name, grid=w.n[:2], cells=w.cells, cfl=w.cfl, precision="mixed",
                        parallelism=f"replicas{world}", l2="inputs larger than L2 (3 FP64 registers of "
                        f"{w.nvar * w.cells * 8 / 1e6:.0f} MB each plus primitives)"),
            roofline=roof(mixed, fv.FV_MIXED), cpu_baseline=cpu, e2e=e2e,
            gpu_launches=mixed["launches"], clocks=mixed["clocks"],
            fp64=dict(value=v64, unit=UNIT, dtype="f64", steps=fargs.steps, ms_per_step=f64["ms"] / fargs.steps,
                      roofline=roof(f64, fv.FV_FP64), gpu_launches=f64["launches"], clocks=f64["clocks"]),
            l1_mixed_vs_fp64=l1, device_errors=[mixed["err"], f64["err"]])
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
