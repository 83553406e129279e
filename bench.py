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


WORKLOADS = ("shock_bubble", "advection", "pr_shock_droplet", "droplet_ensemble", "jet3d", "rising_bubble",
             "vapour_bubble_collapse", "gas_bubble_collapse")


class Job:
    """the cases of one workload (a batch for the droplet ensemble)"""

    def __init__(self, name, cases, inflow=None):
        self.name, self.cases, self.inflow = name, cases, inflow
        self.cells = sum(c.cells for c in cases)
        self.w = cases[0]
        self.cfl = cases[0].cfl
        self.nvar = cases[0].nvar
        self.ndim = cases[0].ndim


def _workload_cases(args):
    return [None] * (args.ncases if args.workload == "droplet_ensemble" else 1)


def _workload(args):
    from paper_2304_00140_gb300 import workloads as wl
    k = args.workload
    if k == "shock_bubble":
        w = wl.shock_bubble(nx=args.nx, ny=args.ny)
        return Job(w.name, [w])
    if k == "advection":
        w = wl.advection(n=args.nx if args.nx != 2048 else 128)
        return Job(w.name, [w])
    if k == "pr_shock_droplet":
        w = wl.pr_shock_droplet(n=args.nx if args.nx != 2048 else 1024)
        return Job(w.name, [w])
    if k == "droplet_ensemble":
        cases = wl.droplet_ensemble(ncases=args.ncases)
        return Job(f"droplet_ensemble_{len(cases)}", cases)
    if k == "jet3d":
        n = (512, 256, 256) if args.nx == 2048 else (args.nx, args.nx // 2, args.nx // 2)
        w = wl.jet3d(n=n)
        return Job(w.name, [w], inflow=[wl.jet_inflow_velocity(w)])
    if k == "rising_bubble":
        # Table 4.4 case 2 (viscous stresses, gravity, CSF); --nx N: an N x 2N grid
        n = (160, 320) if args.nx == 2048 else (args.nx, 2 * args.nx)
        w = wl.rising_bubble(2, n=n)
        return Job(w.name, [w])
    if k in ("vapour_bubble_collapse", "gas_bubble_collapse"):
        # Sec. 4.9 on the paper's finest 4 um spacing everywhere; --nx N: N x N
        n = 1000 if args.nx == 2048 else args.nx
        w = wl.bubble_collapse(k.split("_")[0], n=(n, n))
        return Job(w.name, [w])
    raise SystemExit(f"unknown workload {k}")


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
def _alg_flops_per_cell(job, fused=False):
    """Algorithmic FP64 flops of one stage-kernel launch per interior cell:
    the op-counting build of the oracle (profiles/fp64_opcount.json, written
    by oracle/opcount_table.py) counts the stage's faces, sources and update
    (+, -, *, /, sqrt, min, max, compare = 1 each).  None for workloads it
    has no entry for, and for the fused kernel (which also recovers the
    primitives), where only the HBM roofline is reported."""
    p = os.path.join(ROOT, "profiles", "fp64_opcount.json")
    if fused or not os.path.exists(p):
        return None
    e = json.load(open(p))["workloads"].get(job.name)
    return e["flops_per_cell"] if e else None


KERNEL_SOURCES = {
    # the files each roofline kernel's code comes from
    "march2d_kernel": ("fv_march.cuh", "fv_march_inst.cuh", "fv_march.cu", "fv_march_f.cu", "fv_march_fc.cu", "fv_march_d.cu",
                       "fv_kernels.cuh", "fv_device.cuh", "fv_launch.h"),
    "stage_kernel": ("fv_kernels.cuh", "fv_device.cuh", "fv_launch.h", "fv_stage_inst.cuh", "fv_stage2d.cu",
                     "fv_stage2f.cu", "fv_stage3d.cu", "fv_stage3f.cu"),
    "zmarch_kernel": ("fv_zmarch.cuh", "fv_zmarch.cu", "fv_kernels.cuh", "fv_device.cuh", "fv_launch.h"),
}


def _source_hash(kernel):
    """sha1 of the CUDA sources a roofline kernel is built from: an ncu
    traffic figure is only quoted for the kernel version it was taken on."""
    import hashlib
    d = os.path.join(ROOT, "paper_2304_00140_gb300", "csrc")
    h = hashlib.sha1(kernel.encode())
    for f in KERNEL_SOURCES[kernel]:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def _ncu_traffic(job, form, kernel):
    """DRAM bytes (read + write) of one launch of the roofline kernel from the
    ncu capture recorded in profiles/stage_traffic.json for this kernel's
    source version, or None."""
    p = os.path.join(ROOT, "profiles", "stage_traffic.json")
    if not os.path.exists(p):
        return None
    return json.load(open(p)).get(f"{kernel}@{_source_hash(kernel)}", {}).get(f"{job.name}/{form}")


def record_traffic(args):
    """--record-traffic CSV: average DRAM bytes (read + write) per stage_kernel
    launch from an ncu ``--csv --log-file`` capture of this bench's own command
    (metrics dram__bytes_read.sum, dram__bytes_write.sum), stored in
    profiles/stage_traffic.json under the current CUDA source hash and the
    workload/form the capture ran."""
    import csv
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    per, names = {}, {}
    rows = [r for r in csv.reader(open(args.record_traffic)) if len(r) > 5]
    hdr = rows[0]
    ki, ii, mi, vi, ui = (hdr.index(k) for k in ("Kernel Name", "ID", "Metric Name", "Metric Value", "Metric Unit"))
    for r in rows[1:]:
        kern = next((k for k in KERNEL_SOURCES if k in r[ki]), None)
        if kern and r[mi] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            per[r[ii]] = per.get(r[ii], 0.0) + float(r[vi].replace(",", "")) * scale[r[ui]]
            names[r[ii]] = kern
    if not per or args.precision == "both" or len(set(names.values())) != 1:
        raise SystemExit("need one roofline kernel's DRAM metrics in the CSV and --precision mixed|fp64")
    kern = next(iter(names.values()))
    job = _workload(args)
    p = os.path.join(ROOT, "profiles", "stage_traffic.json")
    d = json.load(open(p)) if os.path.exists(p) else {}
    key = f"{kern}@{_source_hash(kern)}"
    # drop figures of older versions of this kernel
    d = {k: v for k, v in d.items() if not (k.split("@")[0] == kern and k != key)}
    d.setdefault(key, {})[f"{job.name}/{args.precision}"] = sum(per.values()) / len(per)
    json.dump(d, open(p, "w"), indent=1, sort_keys=True)
    print(json.dumps(dict(kernel=kern, launches=len(per), bytes_per_launch=sum(per.values()) / len(per))))


def _nprim(w):
    """primitive-array fields: W, then rho and c (App. D switch, gravity or
    the barotropic closure), the encoded liquid fraction (App. D or CSF), mu
    and k_c (viscous terms), the vapour fraction (barotropic closure)"""
    s = w.scheme
    grav = any(g != 0.0 for g in s.get("gravity", (0.0, 0.0, 0.0)))
    visc = any(c.get("mu", 0.0) > 0.0 or c.get("kc", 0.0) > 0.0 for c in w.comps)
    baro = w.comps[0]["kind"] == 2
    capj = s["sigma"] > 0 and s.get("st_model", 0) == 1
    return (w.nvar + (2 if (s["iles"] or grav or baro) else 0) + (1 if (s["iles"] or s["sigma"] > 0) else 0)
            + (2 if visc else 0) + (1 if baro else 0) + (1 if capj else 0))


def _design_stage_bytes(job, precision, fused=False):
    """HBM bytes one stage-kernel launch of this design must move per its
    inputs and outputs.  Tiled kernel: every interior cell's primitives read
    once (fp32 in the mixed form, fp64 otherwise), q^0 read and q^k written
    (8 bytes a value: FP64 or float-float).  Fused kernel: q^{k-1} and q^0
    read, q^k written."""
    if fused:
        return job.cells * 3 * job.nvar * 8
    rs = 4 if precision == 1 else 8
    return job.cells * (_nprim(job.w) * rs + 2 * job.nvar * 8)


def _compulsory_stage_bytes(job, precision):
    """Compulsory HBM bytes of one stage (average over the four) of an ideal
    single-pass design: per cell-update, FP64 reads q^0 once, every stage
    reads q^{k-1} (and q^0 for stages 2-4) and writes q^k, all 8 bytes a
    value: (2 + 3 + 3 + 3) x 8 = 88 bytes per conserved field; the mixed
    form keeps q^A, q^B in FP32 (4 bytes) and q^0, q^{n+1} in 8 bytes:
    (8 + 4) + 2 x (4 + 8 + 4) + (4 + 8 + 8) = 64 bytes per field."""
    per_field = 64 if precision == 1 else 88
    return job.cells * job.nvar * per_field / 4.0


def fp64_peak(torch):
    """Measured FP64 FMA rate of this GPU (TFLOP/s): the best of five
    launches of the library's FMA-chain probe over 8 blocks per SM."""
    import ctypes as C
    from paper_2304_00140_gb300 import fv
    L = fv.load()
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clk = ClockSampler(torch.cuda.current_device())
    time.sleep(0.2)
    best = 0.0
    for _ in range(5):
        ms, fl = C.c_double(), C.c_double()
        st = L.fv_probe_fp64(8 * nsm, 256, 4096, C.byref(ms), C.byref(fl))
        if st != fv.FV_OK:
            raise fv.FVError(st, "fp64 probe")
        best = max(best, fl.value / (ms.value * 1e-3) / 1e12)
    clocks = clk.stop()
    return dict(tflops=best, sms=nsm, clocks=clocks,
                how=f"FMA chains, 8 independent per thread, {8 * nsm} blocks x 256 threads x 4096 rounds, "
                    "best of 5 launches, CUDA events")


def _solver(job, precision):
    from paper_2304_00140_gb300 import fv
    s = fv.Solver(job.cases, precision=precision, inflow_u=job.inflow)
    for i, c in enumerate(job.cases):
        s.set_state(job.prims[i], kind=fv.FV_PRIMITIVE, case=i)
    return s


def run_form(job, precision, args, torch, dist, rank, world):
    from paper_2304_00140_gb300 import fv
    s = _solver(job, precision)
    w = job.w
    stream = torch.cuda.current_stream()
    s.step_async(args.warmup, w.cfl)
    torch.cuda.synchronize()
    tile = s.tile()
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
        from paper_2304_00140_gb300 import replicas
        ms = replicas.max_over_ranks(ms, dist, device="cuda")
        dist.barrier()
    err = s.error_word()
    # per-kernel times with event pairs on the launching stream (no graph)
    kprof = max(4, min(args.steps, 50))
    s.profile(True)
    s.step_async(kprof, w.cfl)
    prof = s.profile_read()
    s.profile(False)
    state = np.concatenate([s.get_state(case=i).reshape(job.nvar, -1) for i in range(len(job.cases))], axis=1)
    s.close()
    return dict(ms=ms, launches=launches, clocks=clocks, err=err, prof=prof, state=state, tile=tile,
                steps=args.steps)


def e2e_form(job, precision, args, torch):
    """Same metric through the public API with host buffers: every step's
    input state goes in from page-locked host memory and every step's result
    comes back.  The pipelined calls (fv_upload_async / fv_commit_upload /
    fv_download_async) move them on the copy engines while the previous step
    runs; the blocking calls (fv_set_state / fv_get_state, one synchronisation
    each) are timed too."""
    import ctypes as C
    from paper_2304_00140_gb300 import fv
    s = _solver(job, precision)
    nc = len(job.cases)
    L = s.L
    # the timed steps of the device leg, up to 200: a longer run amortises the
    # first upload and the last download, which overlap nothing
    nsteps = max(3, min(args.steps, 200))
    h_in = torch.from_numpy(s.get_state_all().copy()).pin_memory()
    h_out = [torch.empty_like(h_in).pin_memory() for _ in range(2)]
    pin = C.c_void_p(h_in.data_ptr())
    pout = [C.c_void_p(h.data_ptr()) for h in h_out]

    def check(st):
        if st:
            raise fv.FVError(st, L.fv_last_error(s.ctx).decode())
    # warm-up of the pipeline (staging buffers, graph)
    check(L.fv_upload_async(s.ctx, pin) or L.fv_commit_upload(s.ctx) or L.fv_step_async(s.ctx, 1, job.cfl)
          or L.fv_download_async(s.ctx, pout[0]) or L.fv_io_wait(s.ctx))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    check(L.fv_upload_async(s.ctx, pin))
    for i in range(nsteps):
        check(L.fv_commit_upload(s.ctx))
        if i + 1 < nsteps:
            check(L.fv_upload_async(s.ctx, pin))
        check(L.fv_step_async(s.ctx, 1, job.cfl) or L.fv_download_async(s.ctx, pout[i % 2]))
    check(L.fv_io_wait(s.ctx))
    t1 = time.perf_counter()
    # blocking calls, for comparison
    if nc == 1:
        put = lambda p: L.fv_set_state(s.ctx, 0, fv.FV_CONSERVED, p)
        take = lambda p: L.fv_get_state(s.ctx, 0, fv.FV_CONSERVED, p)
    else:
        put = lambda p: L.fv_set_state_all(s.ctx, fv.FV_CONSERVED, p)
        take = lambda p: L.fv_get_state_all(s.ctx, fv.FV_CONSERVED, p)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for _ in range(nsteps):
        check(put(pin) or L.fv_step_async(s.ctx, 1, job.cfl) or take(pout[0]))
    t3 = time.perf_counter()
    nbytes = int(h_in.numel() * 8)
    s.close()
    return dict(value=job.cells * nsteps / (t1 - t0), unit=UNIT, h2d_bytes_per_step=nbytes,
                d2h_bytes_per_step=nbytes, steps=nsteps, api="fv_upload_async / fv_commit_upload / fv_step_async / "
                "fv_download_async (copies overlap the steps)",
                blocking=dict(value=job.cells * nsteps / (t3 - t2), api="fv_set_state / fv_step_async / fv_get_state"))


# ------------------------------------------------------------- CPU oracle
def oracle_window_step(o, q, dt, lo, hi):
    """one LSRK step of the oracle restricted to a window (stage k evaluated
    on the window grown by the stencil reach of the later stages, two cells a
    stage; the capillary jump, which no benchmark workload uses, reaches
    three).  Inside the window it is the full step where the grown window
    stays off periodic sides; elsewhere it is a timing sample only."""
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


def cpu_oracle_rate(job, rows, reps=1, threads=1):
    """The FP64 oracle, as it stands, on ``threads`` host threads (its
    OpenMP cell loops): one LSRK step on a band of ``rows`` full-width rows
    (2D) or planes (3D) through the middle of the first case."""
    import oracle
    oracle.threads(threads)
    w = job.w
    o = oracle.Oracle(w, inflow_u=job.inflow[0] if job.inflow else None)
    q = o.prim_to_cons(w.primitives())
    ax = w.ndim - 1
    n = w.n[ax]
    rows = min(rows, n)
    a0 = max(0, n // 2 - rows // 2)
    lo, hi = [0, 0, 0], [w.n[0], w.n[1], w.n[2]]
    lo[ax], hi[ax] = a0, a0 + rows
    dt = 0.1 * o.dt(q, w.cfl) if w.cells <= 4_000_000 else 1e-12
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle_window_step(o, q, dt, lo, hi)
    t1 = time.perf_counter()
    cells = w.cells // n * rows * reps
    return cells / (t1 - t0), cells, t1 - t0


def run_reference(args):
    """--impl reference: the oracle (the only reference there is: the paper
    ships no code) timed on the host cores, each step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    job = _workload(args)
    w = job.w
    import oracle
    ncores = oracle.threads(os.cpu_count() or 1)
    o = oracle.Oracle(w, inflow_u=job.inflow[0] if job.inflow else None)
    q = o.prim_to_cons(w.primitives())
    # band height sized so the whole run stays near two minutes of host time
    # (about 0.04 s per row and step on one core)
    rows = args.ref_rows or int(min(w.n[1], max(2, 120.0 * ncores / ((args.steps + args.warmup) * 0.04 * 2))))
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
    sample = f"one LSRK step per bench step on a {w.n[0]}x{rows} band of the {w.n[0]}x{ny} grid of {w.name}"
    line = dict(impl="reference", metric=METRIC, value=val, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * (t1 - t0) / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=w.name, grid=w.n[:2], band_rows=rows),
                cpu_baseline=dict(value=val, unit=UNIT, cores=ncores, kind="oracle", sample=sample),
                e2e=dict(value=val, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 400; 100 for the 33.5 M-cell jet3d, whose FP64 form takes "
                         "0.6 s a step)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=0,
                    help="rows (2D) or planes (3D) of the CPU-baseline band (default: about 1e6 cells, 10-20 s)")
    ap.add_argument("--ref-rows", type=int, default=0)
    ap.add_argument("--fp64-steps", type=int, default=0, help="steps for the FP64 form (default: --steps)")
    ap.add_argument("--workload", default="shock_bubble", choices=WORKLOADS)
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--ncases", type=int, default=1024)
    ap.add_argument("--record-traffic", default="", help="ncu CSV of this command: store its stage_kernel DRAM "
                    "bytes per launch in profiles/stage_traffic.json and exit")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 100 if args.workload == "jet3d" else 400
    if args.warmup < 3:
        args.warmup = 3
    if args.record_traffic:
        record_traffic(args)
        return
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
    job = _workload(args)
    if dist and len(job.cases) > 1:
        # a batch is split across ranks (longest-processing-time on cells)
        from paper_2304_00140_gb300 import replicas
        mine = replicas.lpt_partition([c.cells for c in job.cases], world)[rank]
        job = Job(job.name, [job.cases[i] for i in mine])
    job.prims = [c.primitives() for c in job.cases]
    w = job.w
    peaks = _peaks()

    forms = {"both": ("mixed", "fp64"), "mixed": ("mixed",), "fp64": ("fp64",)}[args.precision]
    res = {}
    fargs = argparse.Namespace(**vars(args))
    if args.fp64_steps:
        fargs.steps = args.fp64_steps
    if "mixed" in forms:
        res["mixed"] = run_form(job, fv.FV_MIXED, args, torch, dist, rank, world)
    if "fp64" in forms:
        res["fp64"] = run_form(job, fv.FV_FP64, fargs, torch, dist, rank, world)

    # accuracy of the mixed form against the FP64 form after the same steps
    # (both advanced warmup + steps + profiled steps from the same state):
    # relative L1 per conserved field; the momentum components are measured
    # against the L1 norm of the momentum vector (a component can be ~0)
    l1 = None
    if len(res) == 2 and fargs.steps == args.steps:
        a, b = res["mixed"]["state"], res["fp64"]["state"]
        nv = a.shape[0]
        den = np.abs(b).reshape(nv, -1).sum(1)
        den[1:1 + w.ndim] = np.sqrt((b[1:1 + w.ndim] ** 2).sum(0)).sum()
        num = np.abs(a - b).reshape(nv, -1).sum(1)
        # a field that is zero in both forms (no gas in the vapour collapse) has error 0
        l1 = np.where(num == 0.0, 0.0, num / np.maximum(den, 1e-300)).tolist()

    f64peak = fp64_peak(torch) if (rank == 0 and "fp64" in forms) else None

    def roof(r, precision):
        st = r["prof"]["stage"]
        avg_ms = st["ms"] / max(1, st["launches"])
        fused = bool(r["tile"].get("fused"))
        design = _design_stage_bytes(job, precision, fused)
        byt = _compulsory_stage_bytes(job, precision)
        ach = byt / (avg_ms * 1e-3) / 1e9
        form = "mixed" if precision == fv.FV_MIXED else "fp64"
        kname = "march2d_kernel" if fused else ("zmarch_kernel" if r["tile"].get("zmarch") else "stage_kernel")
        step_ms = r["ms"] / r["steps"]
        step = dict(compulsory_bytes_per_step=4 * byt, ms_per_step=step_ms,
                    achieved=4 * byt / (step_ms * 1e-3) / 1e9, frac=4 * byt / (step_ms * 1e-3) / 1e9 / peaks["hbm"])
        out = dict(bound="hbm", achieved=ach, peak=peaks["hbm"], unit="GB/s", frac=ach / peaks["hbm"],
                   traffic=_ncu_traffic(job, form, kname),
                   kernel=kname,
                   avg_launch_ms=avg_ms, algorithmic_bytes_per_launch=byt,
                   algorithmic_basis=("compulsory bytes of one stage, the four stages' average: "
                                      + ("64" if precision == fv.FV_MIXED else "88") + " B per conserved field "
                                      "per cell-update / 4"),
                   design_bytes_per_launch=design, design_frac=design / (avg_ms * 1e-3) / 1e9 / peaks["hbm"],
                   peak_source=peaks["src"], step_level=step,
                   kernel_share={k: v["ms"] for k, v in r["prof"].items()}, tile=r["tile"])
        fl = _alg_flops_per_cell(job, fused)
        if precision == fv.FV_FP64 and fl and f64peak:
            # the FP64 form is bound by the FP64 pipe (measured FMA rate)
            peak = f64peak["tflops"]
            tf = fl * job.cells / (avg_ms * 1e-3) / 1e12
            out = dict(bound="alu", achieved=tf, peak=peak, unit="TFLOP/s", frac=tf / peak,
                       traffic=out["traffic"], kernel=out["kernel"], avg_launch_ms=avg_ms,
                       algorithmic_flops_per_launch=fl * job.cells,
                       flops_basis="op-counting build of the oracle (profiles/fp64_opcount.json)",
                       peak_source="measured: " + f64peak["how"], peak_clocks=f64peak["clocks"],
                       hbm=dict(achieved=ach, peak=peaks["hbm"], frac=ach / peaks["hbm"],
                                algorithmic_bytes_per_launch=byt, design_bytes_per_launch=design,
                                step_level=step),
                       kernel_share=out["kernel_share"], tile=r["tile"])
        return out

    head = forms[0]
    hprec = fv.FV_MIXED if head == "mixed" else fv.FV_FP64
    hsteps = args.steps if head == "mixed" else fargs.steps
    if dist:
        from paper_2304_00140_gb300 import replicas
        cells_all = replicas.sum_over_ranks(job.cells, dist, device="cuda")
    else:
        cells_all = job.cells
    val = cells_all * hsteps / (res[head]["ms"] * 1e-3)
    e2e = e2e_form(job, hprec, args, torch) if rank == 0 else None
    if e2e is not None:
        e2e["value"] *= cells_all / job.cells

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ncores = os.cpu_count() or 1
        per_row = job.w.cells // job.w.n[job.w.ndim - 1]
        rows = args.cpu_rows or max(1, min(job.w.n[job.w.ndim - 1], int(1.0e6 / per_row)))
        unit_name = "plane" if job.w.ndim == 3 else "row"
        rate1, cells1, secs1 = cpu_oracle_rate(job, rows, threads=1)
        # all cores: a band sized for about the same seconds
        rows_n = args.cpu_rows or max(1, min(job.w.n[job.w.ndim - 1], rows * max(1, ncores // 2)))
        rate, cells, secs = cpu_oracle_rate(job, rows_n, threads=ncores)
        cpu = dict(value=rate, unit=UNIT, cores=ncores, kind="oracle",
                   sample=f"one LSRK step of a {rows_n}-{unit_name} band of {job.w.name} "
                          f"({cells} cell-updates, {secs:.1f} s, {ncores} threads)",
                   single_thread=dict(value=rate1, cores=1,
                                      sample=f"one LSRK step of a {rows}-{unit_name} band ({cells1} cell-updates, "
                                             f"{secs1:.1f} s)"))

    if rank == 0:
        regbytes = job.nvar * job.cells * 8
        footprint = 3 * regbytes + _nprim(job.w) * job.cells * (4 if head == "mixed" else 8)
        line = dict(
            metric=METRIC, value=val, unit=UNIT, n_gpus=world, steps=hsteps, warmup=args.warmup,
            ms_per_step=res[head]["ms"] / hsteps, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f32+f64" if head == "mixed" else "f64", data="synthetic",
            config=dict(workload=job.name, cases=len(job.cases), grid=w.n[:w.ndim], cells=job.cells, cfl=job.cfl,
                        precision=head,
                        parallelism=(f"batch split over {world} ranks" if len(_workload_cases(args)) > 1 else
                                     f"replicas{world}") if world > 1 else "single GPU",
                        l2=("inputs larger than L2" if footprint > 129e6 else "inputs smaller than L2") +
                        f" (3 FP64 registers of {regbytes / 1e6:.0f} MB each plus primitives)"),
            roofline=roof(res[head], hprec), cpu_baseline=cpu, e2e=e2e,
            gpu_launches=res[head]["launches"], clocks=res[head]["clocks"],
            l1_mixed_vs_fp64=l1, device_errors={k: v["err"] for k, v in res.items()})
        if head == "mixed" and "fp64" in res:
            f64 = res["fp64"]
            line["fp64"] = dict(value=cells_all * fargs.steps / (f64["ms"] * 1e-3), unit=UNIT, dtype="f64",
                                steps=fargs.steps, ms_per_step=f64["ms"] / fargs.steps,
                                roofline=roof(f64, fv.FV_FP64), gpu_launches=f64["launches"],
                                clocks=f64["clocks"])
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
