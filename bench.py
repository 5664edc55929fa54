"""Benchmark of the GB300 GP-MOOD hot path.

Default workload: the Mach-10 double Mach reflection on [0,4] x [0,1] at
4096 x 1024 cells (the largest single-GPU configuration), GP-R3 with the
7->5->3->1 cascade (ell = 12 dx), HLLC, SSP-RK3 at CFL 0.8, MOOD active from
the first step.  One step is one full SSP-RK3 step (three stages, each with
its ghost fill, face sweeps, update + detection and MOOD loop, and the
time-step reduction).  Metric: cell-updates per second.

The default line times the FP64 path and adds, on the same workload, an
`fp32` record (FP32 reconstruction, Riemann solver and detection; FP64 state
and stage accumulation), an `adjoint` record (the 1024^2 periodic shear layer,
GP-R2, 200 steps with checkpoints every 20: reverse / forward time), the
512^2 isentropic vortex in FP64 (`vortex_512`), and the FP64 CPU oracle on a
bounded sample of the workload, single-threaded and on all host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload dmr|vortex]
                    [--precision fp64|fp32] [--only]
    python bench.py --impl reference ...    (the FP64 CPU oracle on the host)

Under torchrun (N > 1) every rank runs its own replica of the workload on its
own GPU (the method has no data exchange between independent problems);
value = all ranks' cell-updates / the slowest rank's time.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D Euler GP-MOOD cell-updates/s"
UNIT = "cell-updates/s"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12  # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 256 * 2.07e9 / 1e12  # 128 FFMA/clk/SM
HLLC_FLOPS = 78  # per pointwise HLLC flux, divisions and square roots counted once
# the oracle's bounded sample of the double Mach reflection: the same problem
# at 1/16 of the cells (it recomputes every face in every MOOD iteration, so
# one full-size step takes minutes on one core)
ORACLE_SAMPLE = (1024, 256)


# --scheme: the default is the benchmark workload (GP-R3 cascade); the others
# time the third-order schemes of Sec. 3.1 on the same problem
SCHEME_DESC = {
    "GP-R3": ("GP-R3 cascade 7->5->3->1", 3),
    "GP-MOOD3": ("GP-MOOD3 (GP-R1 -> FOG)", 1),
    "POL-MOOD3": ("POL-MOOD3 (Poly3 -> FOG)", 1),
}
DEFAULT_SIZE = {"dmr": (4096, 1024), "vortex": (512, 512)}


def workload(kind, nx, ny, scheme="GP-R3"):
    from paper_2110_08683_gb300 import inputs as I

    R = SCHEME_DESC[scheme][1]
    if kind == "dmr":
        p = I.dmr(nx=nx, ny=ny, R=R, cascade=None if scheme == "GP-R3" else [1, 0])
    else:
        p = I.vortex(n=nx, R=R, cascade=None if scheme == "GP-R3" else [1, 0])
    if scheme != "GP-R3":
        p["recon"] = "poly3" if scheme == "POL-MOOD3" else "gp"
    return p


def workload_name(kind, nx, ny, scheme="GP-R3"):
    if kind == "dmr":
        return (f"Mach-10 double Mach reflection {nx}x{ny} on [0,4]x[0,1], "
                f"{SCHEME_DESC[scheme][0]}, ell=12dx, SSP-RK3, CFL 0.8, HLLC")
    return (f"isentropic vortex {nx}^2 periodic [-5,5]^2, {SCHEME_DESC[scheme][0]}, ell=0.5, "
            f"SSP-RK3, CFL 0.8, HLLC")


def faces_flops_per_face(R=3, fused=False):
    """Arithmetic of one first-pass face launch per face: the parity sums of
    the cell (4 variables), the q/2 parity dot products of length N and the
    butterflies, then q HLLC fluxes and the Gauss sum.  The fused kernel's
    block of 8 x 32 cells owns 7 x 31 faces of each direction: it forms the
    sums of its 256 cells once, x states on 224 of them, y states on 256."""
    N = 2 * R * R + 2 * R + 1
    q = R + 1
    sums = 4 * (2 * R * 2 + (R * (R - 1) // 2) * 8)
    pairs, middle = q // 2, q % 2
    dots = 4 * (2 * N * (pairs + middle) + 8 * pairs + 2 * middle)
    riemann = q * (HLLC_FLOPS + 8)
    if not fused:
        return sums + dots + riemann
    return (256 * sums + (224 + 256) * dots) / (2 * 7 * 31) + riemann


FACE_KERNEL_SOURCES = ("gpmood_kernels.cuh", "gpmood_internal.h", "kernels_impl.cuh",
                       "fp_bits.h")


def kernel_source_hash():
    """Hash of the sources that define the first-pass face kernel."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2110_08683_gb300", "csrc")
    for f in FACE_KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def algorithmic_flops_per_face(R=3):
    """The reconstruction and Riemann work of one face as the method states
    it: the left and right states at q Gauss points, 4 variables, each a dot
    product of length N (8 q N FMA, 2 flop each), q HLLC fluxes and the
    Gauss sum of 4 variables (q FMA each)."""
    N = 2 * R * R + 2 * R + 1
    q = R + 1
    return 2 * 8 * q * N + q * HLLC_FLOPS + 2 * 4 * q


def ncu_traffic(precision, kind, scheme="GP-R3"):
    """DRAM bytes per launch of the first-pass face kernel on this workload from the
    committed ncu summary, or None when the kernel sources changed since the
    capture.  Rows are keyed by workload and precision ("dmr fp64"), with the
    scheme appended for the third-order schemes ("vortex fp64 POL-MOOD3")."""
    key = f"{kind} {precision}" + ("" if scheme == "GP-R3" else f" {scheme}")
    path = os.path.join(ROOT, "profiles", "faces_xy_traffic.md")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    # table rows: | workload precision | kernel sources sha256 | DRAM bytes per launch | ...
    for ln in lines:
        cells = [c.strip() for c in ln.strip().strip("|").split("|")]
        if len(cells) >= 3 and cells[0] == key:
            if cells[1] != kernel_source_hash():
                return None
            try:
                return float(cells[2])
            except ValueError:
                return None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = str(index)
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", self.index],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # the timed region starts once the sampler is producing rows
        t0 = time.perf_counter()
        while not self.rows and time.perf_counter() - t0 < 3.0:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        # one GPU per process, selected before any CUDA call
        os.environ["CUDA_VISIBLE_DEVICES"] = str(local)
        import torch.distributed as dist

        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units, ms, world):
    """Whole-job throughput of independent replicas: the units every rank
    processed over the slowest rank's time (max over ranks), per second."""
    total = allreduce_sum(float(units), world)
    ms_max = allreduce_max(float(ms), world)
    return total / (ms_max / 1e3), ms_max


def host_info():
    """Host cores, CPU model and the oracle's compiler flags (for the CPU
    baseline's record)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import oracle as O

    return {"nproc": os.cpu_count(), "cpu_model": model or platform.machine(),
            "machine": platform.machine(), "oracle_flags": " ".join(O.CFLAGS)}


def _oracle_worker(kind, nx, ny, scheme, steps, barrier, queue):
    """One replica of the oracle's bounded sample: `steps` full SSP-RK3 steps
    of the workload from its initial state, timed between two clock reads
    after all replicas have set up."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle as O

    p = workload(kind, nx, ny, scheme)
    o = O.Oracle(p)
    U, t = p["U0"], 0.0
    if barrier is not None:
        barrier.wait()
    t0 = time.monotonic()
    for _ in range(steps):
        U, st, _, _ = o.step(U, t)
        t += st["dt"]
    t1 = time.monotonic()
    o.close()
    queue.put((nx * ny * steps, t0, t1))


def oracle_replicas(kind, nx, ny, scheme, steps, procs):
    """`procs` replicas of the oracle's sample at once, one process each
    (spawned: no CUDA state is inherited): total cell-updates over the span
    from the first start to the last finish."""
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    queue = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(kind, nx, ny, scheme, steps, barrier, queue))
          for _ in range(procs)]
    for q in ps:
        q.start()
    res = [queue.get() for _ in ps]
    for q in ps:
        q.join()
    units = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return units / span, span


def oracle_sample(kind):
    """The oracle's bounded sample of a workload: grid and steps."""
    if kind == "dmr":
        return ORACLE_SAMPLE[0], ORACLE_SAMPLE[1], 1
    return DEFAULT_SIZE[kind][0], DEFAULT_SIZE[kind][1], 2


def sample_text(kind, nx, ny, steps):
    if kind == "dmr":
        return (f"{steps} full SSP-RK3 step(s) from t = 0 of the same double Mach reflection at "
                f"{nx}x{ny} (1/16 of the cells: the oracle recomputes every face in every MOOD "
                f"iteration, so a full-size step takes minutes on one core)")
    return f"{steps} full SSP-RK3 steps from t = 0 of the {nx}^2 vortex"


def cpu_baseline(kind, scheme="GP-R3"):
    """The FP64 CPU oracle as it stands on a bounded sample of the workload:
    one replica on one core, then one replica on every host core at once."""
    nx, ny, steps = oracle_sample(kind)
    one, span1 = oracle_replicas(kind, nx, ny, scheme, steps, 1)
    P = os.cpu_count() or 1
    allv, spanP = oracle_replicas(kind, nx, ny, scheme, steps, P)
    return {"value": allv, "unit": UNIT, "cores": P, "kind": "oracle",
            "sample": sample_text(kind, nx, ny, steps) + f", one replica per core on {P} cores, "
                      f"{spanP:.1f} s",
            "single_thread": {"value": one, "unit": UNIT, "cores": 1, "seconds": round(span1, 2)},
            "host": host_info()}


def measure(kind, nx, ny, precision, scheme, steps, warmup, world, local, eager=False,
            serial=False, profile=True, e2e=True, clocks=True):
    """Time `steps` queued steps of the workload (after `warmup`), then a
    profiled pass for the per-class shares and the x-face kernel's launch
    time, then the end-to-end pass through the public calls with host
    buffers."""
    import torch

    import paper_2110_08683_gb300 as gp

    p = workload(kind, nx, ny, scheme)
    p["serial_launch"] = 1 if serial else 0
    R = SCHEME_DESC[scheme][1]
    g = gp.GPMood(p, precision, eager=eager)
    stream = torch.cuda.Stream()
    g.set_stream(stream.cuda_stream)
    # L2 (129 MB) is flushed between timed steps by writing 256 MB
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    g.set_state(p["U0"])
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            g.step_async()
    g.sync()
    torch.cuda.synchronize()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    sampler = ClockSampler(local) if clocks else None
    # timed region: the steps are queued back to back (the host reads nothing
    # between them), each bracketed by events, an L2 flush between steps
    launches0 = g.launch_count()
    st0 = g.flags(maps=False)[2]
    # the state the timed region starts from: the profiled pass replays the
    # same steps, so its per-class shares describe the timed steps
    U_start = torch.empty((4, ny, nx), dtype=torch.float64, device="cuda")
    g.get_state(U_start)
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    torch.cuda.nvtx.range_push("timed")  # ncu --nvtx-include "timed/" sees these steps
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()
            e0[k].record(stream)
            g.step_async()
            e1[k].record(stream)
    g.sync()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(world)
    if sampler:
        sampler.stop()
    launches = g.launch_count() - launches0
    st1 = g.flags(maps=False)[2]
    ms = sum(a.elapsed_time(b) for a, b in zip(e0, e1))
    value, ms_max = job_rate(nx * ny * steps, ms, world)

    # second timed pass over the same steps for the per-class shares and the
    # dominant kernel's duration: the profiled step graphs carry event nodes
    # around every kernel class (read back after each step).  Captured on
    # first use, so a few steps run before the state is set back and the
    # counters are reset.
    prof = profile and not eager  # per-kernel events exist in the graph mode only
    kt, prof_step_ms, fr = {}, None, []
    if prof:
        g.profile(True)
        g.set_state(U_start)
        g.set_time(st0["t"])
        with torch.cuda.stream(stream):
            for _ in range(3):
                g.step()
        torch.cuda.synchronize()
        g.set_state(U_start)
        g.set_time(st0["t"])
        g.profile(True)
        q0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        q1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.zero_()
                q0[k].record(stream)
                g.step()
                q1[k].record(stream)
                st = g.flags(maps=False)[2]
                fr.append((st["nbad_first"], st["iters"]))
        torch.cuda.synchronize()
        kt = g.kernel_times()
        g.profile(False)
        prof_step_ms = sum(a.elapsed_time(b) for a, b in zip(q0, q1)) / steps

    e2e_rec = None
    if e2e:
        # end to end through the public API with host buffers: every step
        # copies the state in from pinned host memory and reads it back
        Uh = torch.empty((4, ny, nx), dtype=torch.float64, pin_memory=True).numpy()
        Uh[...] = p["U0"]
        Uo = torch.empty((4, ny, nx), dtype=torch.float64, pin_memory=True).numpy()
        f0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        f1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        barrier(world)
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.zero_()
                f0[k].record(stream)
                g.set_state(Uh)
                g.step_async()  # get_state waits for it
                g.get_state(Uo)
                f1[k].record(stream)
                Uh[...] = Uo
        torch.cuda.synchronize()
        barrier(world)
        e2e_value, _ = job_rate(nx * ny * steps,
                                sum(a.elapsed_time(b) for a, b in zip(f0, f1)), world)
        e2e_rec = {"value": e2e_value, "unit": UNIT,
                   "h2d_bytes_per_step": int(Uh.nbytes), "d2h_bytes_per_step": int(Uo.nbytes)}
    g.close()

    # roofline of the dominant kernel: the first-pass x-face kernel
    real64 = precision == "fp64"
    roofline = None
    if prof:
        fx_ms, fx_n = kt["faces_x"]
        per_launch_s = fx_ms / 1e3 / max(fx_n, 1)
        # the fused kernel solves both directions' faces in one launch
        fused = kt["faces_y"][1] == 0
        faces = (nx + 1) * ny + (nx * (ny + 1) if fused else 0)
        peak = FP64_PEAK_TFLOPS if real64 else FP32_PEAK_TFLOPS
        alg = faces * algorithmic_flops_per_face(R)
        exe = faces * faces_flops_per_face(R, fused)
        roofline = {
            "bound": "alu", "achieved": round(alg / per_launch_s / 1e12, 4),
            "peak": round(peak, 4), "unit": "TFLOP/s",
            "frac": round(alg / per_launch_s / 1e12 / peak, 4),
            "traffic": ncu_traffic(precision, kind, scheme),
            "kernel": ("k_faces_xy<R=%d,%s> (x and y faces)" if fused else "k_faces<R=%d,%s,x>")
                      % (R, "double" if real64 else "float"),
            "flops_per_launch": alg,
            "flops_per_face": algorithmic_flops_per_face(R),
            "count": "algorithmic: 8 q N reconstruction FMA (2 flop), q HLLC at %d flop, the "
                     "Gauss sum; per face, x %s faces a launch"
                     % (HLLC_FLOPS, "(nx+1) ny + nx (ny+1)" if fused else "(nx+1) ny"),
            "executed": {"flops_per_face": round(faces_flops_per_face(R, fused), 1),
                         "flops_per_launch": exe,
                         "achieved": round(exe / per_launch_s / 1e12, 4),
                         "frac": round(exe / per_launch_s / 1e12 / peak, 4),
                         "count": "the kernel's own arithmetic after the parity-sum "
                                  "reconstruction (mirror-orbit sums, q/2 dot products, "
                                  "butterflies)"},
            "launch_ms": round(per_launch_s * 1e3, 4),
            "timing": "event nodes around every x-face launch in the step graph, second timed "
                      "pass of the same steps (L2 flushed between steps)",
            "peak_source": "derived: 152 SMs x %s/clk x 2.07 GHz (of nominal; measured DFMA "
                           "1.19 TFLOP/s, FFMA 69.9 TFLOP/s)" % ("4 FP64 flop" if real64
                                                                 else "256 FP32 flop")}
    total_kernel_ms = sum(v[0] for v in kt.values())
    shares = {k: round(v[0] / total_kernel_ms, 4) if total_kernel_ms else None
              for k, v in kt.items()} if prof else None
    ncell = nx * ny
    mood = None
    if fr:
        nb = [b for f in fr for b in f[0]]
        it = [i for f in fr for i in f[1]]
        mood = {"first_pass_flag_fraction_mean": round(sum(nb) / len(nb) / ncell, 6),
                "first_pass_flag_fraction_max": round(max(nb) / ncell, 6),
                "iterations_per_stage_mean": round(sum(it) / len(it), 2),
                "iterations_per_stage_max": max(it)}
    return {
        "value": value, "ms_per_step": ms_max / steps,
        "dtype": "f64" if real64 else "f32+f64",
        "config": {"workload": workload_name(kind, nx, ny, scheme), "cells": ncell,
                   "precision": precision, "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MB write)",
                   "t_start": round(st0["t"], 6), "t_end": round(st1["t"], 6)},
        "roofline": roofline, "kernel_shares": shares,
        # the profiled pass: event-timed kernel classes against the whole step
        # (the difference is the graph's scheduling between kernels, the
        # conditional nodes and the host round trip of the profiled steps)
        "step_anatomy": None if not prof else {
            "kernel_classes_ms_per_step": round(total_kernel_ms / steps, 4),
            "profiled_step_ms": round(prof_step_ms, 4)},
        "mood": mood,
        "launch_mode": ("eager" if eager else "graph, steps queued without host round trips")
                       + (", stream order" if serial else ", programmatic dependent launch"),
        "gpu_launches": int(allreduce_sum(launches, world)),
        "e2e": e2e_rec,
        "clocks": sampler.summary() if sampler else None,
    }


def summary_of(rec):
    """The keys of a sub-record of the default line."""
    keys = ("value", "ms_per_step", "dtype", "config", "roofline", "kernel_shares", "mood",
            "e2e", "gpu_launches", "clocks")
    return {k: rec[k] for k in keys if k in rec}
def run_batch(args, world, rank, local):
    """Many independent four-quadrant problems of uneven sizes in one batch
    (one launch per kernel class, graph-captured MOOD loops)."""
    import torch

    import paper_2110_08683_gb300 as gp
    from paper_2110_08683_gb300 import inputs as I

    torch.cuda.set_device(0 if world > 1 else local)
    probs = I.quadrant_batch(count=args.batch, seed=0)
    cells = sum(q["nx"] * q["ny"] for q in probs)
    b = gp.GPMoodBatch(probs, args.precision, eager=args.eager)
    stream = torch.cuda.Stream()
    b.set_stream(stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    b.set_state([q["U0"] for q in probs])
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            b.step()
    torch.cuda.synchronize()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier(world)
    sampler.start()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            e0[k].record(stream)
            b.step()
            e1[k].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    sampler.stop()
    value, ms = job_rate(cells * args.steps, sum(x.elapsed_time(y) for x, y in zip(e0, e1)), world)
    _, _, _, st = b.info()
    sizes = {}
    for q in probs:
        sizes[q["nx"]] = sizes.get(q["nx"], 0) + 1
    line = {
        "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": f"{args.batch} independent four-quadrant Riemann problems on "
                               f"[0,1]^2, sizes {dict(sorted(sizes.items()))} (n: count), seeded "
                               f"states, GP-R3 cascade 7->5->3->1, ell=12dx, CFL 0.8, one batch",
                   "cells": cells, "precision": args.precision,
                   "parallelism": f"replicas x{world}", "l2": "flushed between timed steps"},
        "autotuned": {"face_kernel": ("fused x+y" if b.tuning()[0] == [0, 0]
                                      else "one sweep per direction"),
                      "warps_xy": b.tuning()[0], "face_items": b.tuning()[1],
                      "update_blocks": b.grids()[0], "mood_blocks": b.grids()[1]},
        "mood_last_step": st,
        "clocks": sampler.summary(),
    }
    b.close()
    return line


def run_adjoint(args, world, rank, local):
    """Forward rollout and its reverse mode on the smooth periodic shear layer
    (GP-R2, MOOD radii frozen from the forward, 200 steps): with checkpoints
    every 20 steps and segments stepped again in the reverse pass, keeping
    their face states (the default) or not, and with every step's tape kept
    resident.  Each reverse pass's time is set against the plain forward
    rollout (steps queued back to back, nothing recorded)."""
    import torch

    import paper_2110_08683_gb300 as gp
    from paper_2110_08683_gb300 import inputs as I
    from paper_2110_08683_gb300.autograd import rollout

    torch.cuda.set_device(0 if world > 1 else local)
    n = args.adjoint_n
    p = I.shear_layer(n=n, R=2, seed=0)
    g = gp.GPMood(p, args.precision, eager=args.eager)
    U0 = torch.tensor(p["U0"], device="cuda")
    c = (torch.arange(n, dtype=torch.float64, device="cuda") + 0.5) / n
    Yc, Xc = torch.meshgrid(c, c, indexing="ij")
    W = torch.zeros((4, n, n), dtype=torch.float64, device="cuda")
    W[0] = ((Xc >= 0.4) & (Xc <= 0.6) & (Yc >= 0.4) & (Yc <= 0.6)).double() / (n * n)
    g.set_state(p["U0"])
    for _ in range(args.warmup):
        g.step()
    # untimed short rollouts and their reverse modes in every tape strategy:
    # capture the recording graphs and allocate the adjoint buffers
    for every, states in ((None, True), (20, True), (20, False)):
        Uw = U0.clone().requires_grad_()
        (rollout(Uw, g, max(args.warmup, 3), every=every, states=states) * W).sum().backward()
    torch.cuda.synchronize()
    steps = args.adjoint_steps
    # the plain forward rollout
    g.set_state(U0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        g.step_async()
    g.sync()
    torch.cuda.synchronize()
    fwd = time.perf_counter() - t0
    modes = {}
    for name, every, states in (("checkpoints_every_20", 20, True),
                                ("checkpoints_every_20_no_state_tape", 20, False),
                                ("resident_tapes", None, True)):
        U0r = U0.clone().requires_grad_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        UN = rollout(U0r, g, steps, every=every, states=states)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        J = (UN * W).sum()
        J.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        modes[name] = {"forward_s": t1 - t0, "backward_s": t2 - t1,
                       "grad_norm": float(U0r.grad.norm()),
                       "backward_over_plain_forward": (t2 - t1) / fwd,
                       "forward_plus_backward_over_plain_forward": (t2 - t0) / fwd}
        del UN, J, U0r
    # finite differences resolve the FP64 map only (FP32: eps_32 / h ~ 6%)
    fd = None
    if args.adjoint_fd and args.precision == "fp64":
        fd = adjoint_fd_check(g, p, U0, W, steps, args.adjoint_fd, torch)
    return {
        "metric": METRIC, "value": n * n * steps / fwd, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": fwd * 1e3 / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": f"periodic double shear layer {n}^2 with a seeded random density "
                               f"field, GP-R2 cascade 5->3->1, ell=12dx, {steps} steps, "
                               "J = integral of rho over [0.4,0.6]^2",
                   "cells": n * n, "precision": args.precision},
        "plain_forward_s": fwd,
        "adjoint": modes,
        "fd_check": fd,
    }


def adjoint_fd_check(g, p, U0, W, steps, ndir, torch):
    """Central finite differences (h = 1e-6) of the frozen-mask map along
    seeded random directions against the adjoint's directional derivative,
    at the full size: the forward records every step's radii and dt once;
    J(U) replays the steps with them held fixed (gpmood_step_frozen)."""
    from paper_2110_08683_gb300.autograd import rollout

    ny, nx = g.ny, g.nx
    U0r = U0.clone().requires_grad_()
    (rollout(U0r, g, steps) * W).sum().backward()
    grad = U0r.grad.detach()
    otape = torch.empty((steps, 3, ny, nx), dtype=torch.uint8, device="cuda")
    tape = torch.empty((3, 4, ny, nx), dtype=torch.float64, device="cuda")
    dts = []
    g.set_state(U0)
    for k in range(steps):
        dts.append(g.step_record(tape.data_ptr(), otape[k].data_ptr()))
    out = torch.empty_like(U0)

    def J(U):
        g.set_state(U.contiguous())
        for k in range(steps):
            g.step_frozen(otape[k].data_ptr(), dts[k])
        g.get_state(out)
        return float(((out * W).sum(dtype=torch.float64)).item())

    gen = torch.Generator(device="cuda").manual_seed(1234)
    h = 1e-6
    errs = []
    t0 = time.perf_counter()
    for _ in range(ndir):
        d = torch.randn(U0.shape, dtype=torch.float64, device="cuda", generator=gen)
        fdv = (J(U0 + h * d) - J(U0 - h * d)) / (2 * h)
        ad = float((grad * d).sum())
        errs.append(abs(ad - fdv) / max(abs(fdv), 1e-300))
    return {"directions": ndir, "h": h, "max_rel_err": max(errs),
            "median_rel_err": sorted(errs)[len(errs) // 2], "seconds": time.perf_counter() - t0,
            "map": "frozen-mask rollout (radii and dt of the forward held fixed)"}


def run_reference(args, world, rank):
    """The FP64 CPU oracle (the reference arm of this tier) on the host
    cores: one replica of the bounded sample per core, all at once, each step
    a full SSP-RK3 step of the sample; the step count is capped so that the
    run stays within a few minutes."""
    kind, scheme = args.workload, args.scheme
    nx, ny, _ = oracle_sample(kind)
    if args.nx:  # a smaller sample (tests)
        nx, ny = args.nx, args.ny or args.nx
    # the cost of one step of the sample on one core sizes the run
    one, span1 = oracle_replicas(kind, nx, ny, scheme, 1, 1)
    budget = 120.0
    k = max(1, min(args.steps, int(budget / max(span1, 1e-3))))
    P = os.cpu_count() or 1
    value, span = oracle_replicas(kind, nx, ny, scheme, k, P)
    sample = (sample_text(kind, nx, ny, k) + f" (of {args.steps} requested), one replica per "
              f"core on {P} cores")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": k, "warmup": 0, "ms_per_step": span * 1e3 / k, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the same configuration keys as the GPU arm's line; how the oracle
        # ran (host processes, the bounded sample) is in cpu_baseline
        "config": {"workload": workload_name(kind, *DEFAULT_SIZE[kind], scheme),
                   "cells": DEFAULT_SIZE[kind][0] * DEFAULT_SIZE[kind][1], "precision": "fp64",
                   "parallelism": f"replicas x{world}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "kind": "oracle",
                         "sample": sample, "sample_cells": nx * ny,
                         "processes": P,
                         "single_thread": {"value": one, "unit": UNIT, "cores": 1,
                                           "seconds": round(span1, 2)},
                         "host": host_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dmr", choices=sorted(DEFAULT_SIZE),
                    help="dmr: the 4096x1024 double Mach reflection (default); vortex: the "
                         "512^2 isentropic vortex")
    ap.add_argument("--nx", type=int, default=0)
    ap.add_argument("--ny", type=int, default=0)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--only", action="store_true",
                    help="the main record alone (no fp32 / vortex / adjoint sub-records, no "
                         "CPU baseline)")
    ap.add_argument("--serial-launch", action="store_true",
                    help="plain stream order between the step's kernels instead of "
                         "programmatic dependent launch")
    ap.add_argument("--scheme", default="GP-R3", choices=sorted(SCHEME_DESC),
                    help="GP-R3: the benchmark workload; GP-MOOD3 / POL-MOOD3: the "
                         "third-order schemes on the same problem")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--eager", action="store_true",
                    help="launch kernels one by one instead of the step graphs (for per-kernel "
                         "profilers; slower, no per-kernel event timing)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time a rollout and its adjoint instead (shear layer, GP-R2)")
    ap.add_argument("--adjoint-n", type=int, default=1024)
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--adjoint-fd", type=int, default=8,
                    help="random directions of the finite-difference check (0: skip)")
    ap.add_argument("--batch", type=int, default=0,
                    help="time a batch of this many uneven four-quadrant problems instead")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, world, rank)), flush=True)
        return
    import torch

    torch.cuda.set_device(0 if world > 1 else local)
    if args.adjoint:
        line = run_adjoint(args, world, rank, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if args.batch > 0:
        line = run_batch(args, world, rank, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    kind = args.workload
    nx = args.nx or DEFAULT_SIZE[kind][0]
    ny = args.ny or DEFAULT_SIZE[kind][1]
    rec = measure(kind, nx, ny, args.precision, args.scheme, args.steps, args.warmup, world,
                  local, eager=args.eager, serial=args.serial_launch)
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": rec["dtype"], "data": "synthetic"}
    for k in ("config", "roofline", "kernel_shares", "step_anatomy", "mood", "launch_mode",
              "gpu_launches", "e2e", "clocks"):
        line[k] = rec[k]
    if not args.only:
        # the metric's other parts on the same workload: the FP32 path
        other = "fp32" if args.precision == "fp64" else "fp64"
        line[other] = summary_of(measure(kind, nx, ny, other, args.scheme, args.steps,
                                         args.warmup, world, local, eager=args.eager,
                                         serial=args.serial_launch, e2e=False))
        if world == 1:
            # the smallest 2D configuration (MOOD idle on the smooth vortex)
            line["vortex_512"] = summary_of(measure("vortex", 512, 512, "fp64", args.scheme,
                                                    args.steps, args.warmup, world, local,
                                                    e2e=False, clocks=False))
            # adjoint / forward time on the shear layer, checkpoints every 20 steps
            a = run_adjoint(argparse.Namespace(**{**vars(args), "adjoint_fd": 0,
                                                  "precision": "fp64"}), world, rank, local)
            ck = a["adjoint"]["checkpoints_every_20"]
            line["adjoint"] = {
                "config": a["config"]["workload"],
                "plain_forward_s": round(a["plain_forward_s"], 4),
                "reverse_over_forward": round(ck["backward_over_plain_forward"], 3),
                "forward_plus_reverse_over_forward": round(
                    ck["forward_plus_backward_over_plain_forward"], 3),
                "checkpoints_every": 20, "face_state_tapes": True,
                "modes": {k: {kk: round(vv, 4) for kk, vv in m.items()}
                          for k, m in a["adjoint"].items()},
                "forward_cell_updates_per_s": a["value"]}
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and not args.only:
            line["cpu_baseline"] = cpu_baseline(kind, args.scheme)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
