#!/usr/bin/env python
"""Throughput of the explicit MHD stage on one GB300 (and N-GPU replicas).

Workload: the 3D stratified low-Mach magnetoconvection box, 256^3 cells, ideal
gas gamma = 5/3, n = 1.5 polytrope under constant g, heating in the bottom 10%,
isobaric density noise 1e-3 (seed 1234), uniform B_x with beta 1e6, periodic
x/y and reflecting z (workloads.stratified_box).  One "step" is one SSP-RK3
step: the CFL reduction plus three stage evaluations (primitives/EOS, shock
flags, PLM, LHLLD/HLL fluxes, Contact-CT, sources, RK update).  The metric is
cell-updates per second per stage: cells x 3 stages x steps / time.  By
default both forms are timed one after the other: the plain FP64 form and the
mixed form (FP32 deviations, FP64 state); the line's value is the mixed form's,
with the FP64 form, their ratio and the per-field L1 of mixed vs FP64 beside it.

  python bench.py [--gpus N --steps K --warmup W] [--form both|fp64|mixed]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Timing: W untimed steps, then K steps bracketed by a barrier and device
synchronisation, CUDA events on the grid's stream; the state (1.07 GB per
copy) is larger than L2, so no flush is needed.  N > 1 (torchrun): every rank
runs its own box (independent replicas, weak scaling), the time is the max over
ranks and the value sums all ranks' work.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MHD cell-updates/s per stage: plain FP64 vs mixed+MLP form at stated L1; % HBM"
UNIT = "cell-updates/s"
WORKLOAD = ("3D stratified low-Mach magnetoconvection box 256^3, ideal gas gamma=5/3, n=1.5 polytrope, "
            "constant g, heating bottom 10%, density noise 1e-3 seed 1234, B_x beta 1e6, periodic x,y / "
            "reflecting z, SSP-RK3, CFL 0.4, LHLLD + HLL flattening, well-balanced")
STAGES = 3
HBM_FALLBACK_GBS = 6800.0
FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64 (profiling recipe's nominal table)

# Algorithmic work per unit.
# Bytes of one stage per cell that any implementation must move: read the stage
# input (5 cell + 3 face doubles), read U^n for stages 2-3, write the output.
BYTES_PER_CELL_STAGE = {1: 128.0, 2: 192.0, 3: 192.0}
# FP64 flux kernel: FP64 operations per face (DADD + DMUL + 2 DFMA counted from
# the ncu SASS counters of k_flux on the stratified box at 64^3, mean of the
# three directions).
FP64_FLOP_PER_FACE = 637.7
# Mixed flux kernel: FP32 operations per face (FADD + FMUL + 2 FFMA from the ncu
# SASS counters of k_flux<0/1/2, float> on the stratified box at 160^3, per sweep
# direction), and its DRAM bytes per face (dram__bytes_read + write, same capture;
# W is larger than L2 at 160^3, so the per-face traffic carries over to 256^3);
# peak = 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (measured FFMA probe:
# 73.2 TFLOP/s).
FP32_FLOP_PER_FACE = {"flux_x": 381.1, "flux_y": 381.1, "flux_z": 380.1}
FP32_DRAM_BYTES_PER_FACE = {"flux_x": 74.4, "flux_y": 75.8, "flux_z": 76.1}
FP32_NOMINAL_TFLOPS = 80.5
# Fused tile kernel (k_flux_update_mx): from the ncu counters of the
# stratified box at 160^3 (W larger than L2), one launch of stage 1 and one of
# stage 2 of the scalar launch shape (2): FP32 operations (FADD + FMUL + 2 FFMA)
# 1398 per cell as executed, i.e. 414 per face over the 3.375 faces per cell
# an 8^3 tile evaluates; the algorithmic count is 3 faces per cell x 414 =
# 1243.  The default shape evaluates the same operations, partly as packed
# FP32x2 instructions that those per-opcode counters do not include.  DRAM
# bytes per cell of the current default shape: 111.8 (stage 1, no increment
# to read), 144.6 (stage 2) and 205.3 (stage 3, which also reads and writes
# the FP64 state), 153.9 on average over an RK3 step.
FUSED_FLOP_PER_CELL = 3.0 * 414.3
FUSED_DRAM_BYTES_PER_CELL = (111.8 + 144.6 + 205.3) / 3.0


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,clocks.mem")

    def __init__(self, gpu_id):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_id)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, mem, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
            if len(parts) > 8:
                try:
                    mem.append(float(parts[8]))
                except ValueError:
                    pass
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "mem_mhz": statistics.median(mem) if mem else None}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, ws):
    """Maximum of x over the ranks (the slowest rank's time)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ms_local, ws):
    """Whole-job throughput: every rank's units over the slowest rank's time
    (independent replicas, weak scaling).  Returns (rate, ms_max)."""
    ms_max = allreduce_max(ms_local, ws)
    return units_per_rank * ws / (ms_max * 1e-3), ms_max


def make_problem(n):
    import workloads as W
    return W.stratified_box(n, n, n)


def time_form(P, pr, form, steps, warmup, stream, ws, fused=-1):
    """Device-timed K steps of one precision form; returns dict of measurements.
    fused >= 0 picks the mixed stage's kernel decomposition (phl_set_fused)."""
    import torch
    g = P.Grid(pr, precision=form, stream=stream.cuda_stream)
    if form == "mixed" and fused >= 0:
        g.set_fused(fused)
    g.load()
    for _ in range(warmup):
        g.step(1)
    g.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(ws)
    with torch.cuda.stream(stream):
        e0.record(stream)
        g.step(steps)
        e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    g.check()
    # per-kernel breakdown: the same number of steps again with an event pair
    # around every launch (kept out of the timed region above)
    g.set_timing(True)
    g.kernel_times(reset=True)
    g.step(steps)
    kt = g.kernel_times(reset=True)
    g.set_timing(False)
    g.check()
    st = g.stats()
    return g, ms, kt, st


def roofline(kt, pr, form, hbm_peak, peak_kind, alu):
    """Dominant kernel (largest summed device time) against its bound.  alu:
    the FMA throughputs measured on this GPU by the library's probe
    (phl_probe_alu) in TFLOP/s, {"fp32": .., "fp64": ..}."""
    name, (launches, ms) = max(kt.items(), key=lambda kv: kv[1][1])
    avg_ms = ms / max(launches, 1)
    ncells = pr.ncells
    fp32_peak, fp64_peak = alu["fp32"], alu["fp64"]
    if name == "stage_mixed":
        per_launch = ncells * sum(BYTES_PER_CELL_STAGE.values()) / 3.0
        achieved = per_launch / (avg_ms * 1e-3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "peak_kind": f"{peak_kind} HBM copy",
                "avg_launch_ms": avg_ms, "launches": launches}
    if name == "flux_update":
        # fused tile kernel: the faces of all three directions + the cell update;
        # algorithmic work = 3 faces per cell x the FP32 operations per face
        flop = FUSED_FLOP_PER_CELL
        achieved = ncells * flop / (avg_ms * 1e-3) / 1e12
        traffic = ncells * FUSED_DRAM_BYTES_PER_CELL
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                "traffic_note": "bytes per launch: ncu DRAM bytes per cell at 160^3 (RK3 mean) x cells",
                "peak_kind": "measured FP32 FFMA rate (phl_probe_alu, this run)",
                "nominal_peak": FP32_NOMINAL_TFLOPS, "frac_of_nominal": achieved / FP32_NOMINAL_TFLOPS,
                "flop_per_cell": flop, "avg_launch_ms": avg_ms, "launches": launches}
    if name.startswith("flux"):
        n = pr.n[0]
        faces = (n + 1) * (n + 2) * (n + 2)
        fp64 = form == "fp64"
        flop = FP64_FLOP_PER_FACE if fp64 else FP32_FLOP_PER_FACE[name]
        peak = fp64_peak if fp64 else fp32_peak
        achieved = faces * flop / (avg_ms * 1e-3) / 1e12
        traffic = None if fp64 else faces * FP32_DRAM_BYTES_PER_FACE[name]
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_note": None if fp64 else "bytes per launch: ncu DRAM bytes per face at 160^3 x faces",
                "peak_kind": "measured FP64 DFMA rate (phl_probe_alu)" if fp64 else "measured FP32 FFMA rate (phl_probe_alu)",
                "flop_per_face": flop, "avg_launch_ms": avg_ms, "launches": launches}
    # HBM view of the whole stage for any other dominant kernel
    stage_ms = sum(v[1] for v in kt.values()) / max(kt.get("update_cells", (1, 0))[0], 1)
    per_stage = ncells * sum(BYTES_PER_CELL_STAGE.values()) / 3.0
    achieved = per_stage / (stage_ms * 1e-3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": None, "peak_kind": f"{peak_kind} HBM copy",
            "avg_launch_ms": avg_ms, "launches": launches, "note": "whole-stage algorithmic bytes / stage time"}


def kernel_hbm(kt, pr, hbm_peak, peak_kind):
    """The dominant kernel against HBM: the stage's algorithmic bytes (170.7 B
    per cell-stage: read the FP64 stage input and U^n, write the output) for
    the cells one launch updates, over its average launch time."""
    name, (launches, ms) = max(kt.items(), key=lambda kv: kv[1][1])
    avg_ms = ms / max(launches, 1)
    b = sum(BYTES_PER_CELL_STAGE.values()) / 3.0
    gbs = pr.ncells * b / (avg_ms * 1e-3) / 1e9
    return {"kernel": name, "bound": "hbm", "bytes_per_cell_stage": b, "achieved": gbs, "peak": hbm_peak,
            "unit": "GB/s", "frac": gbs / hbm_peak, "peak_kind": f"{peak_kind} HBM copy",
            "avg_launch_ms": avg_ms}


def stage_hbm(rate, form, hbm_peak, peak_kind):
    """Whole stage against HBM: algorithmic bytes per cell-stage x rate, 170.7 B
    (read the stage input, 5 cell + 3 face doubles, read U^n in stages 2-3,
    write the output; the state is FP64 in both forms).  The mixed form keeps
    its stage increments in FP32, so its own layout moves 128 B (U^n read,
    increment read and written): reported beside it."""
    b = sum(BYTES_PER_CELL_STAGE.values()) / 3.0
    gbs = rate * b / 1e9
    out = {"bytes_per_cell_stage": b, "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "peak_kind": f"{peak_kind} HBM copy", "frac_of_8tbs": gbs / 8000.0}
    if form == "mixed":
        out["mixed_layout_bytes_per_cell_stage"] = 128.0
        out["mixed_layout_frac"] = rate * 128.0 / 1e9 / hbm_peak
    return out


def e2e_measure(P, g, pr, steps, form="mixed", fused=-1, inflight=3):
    """Same metric through the public API with pinned host buffers each step:
    phl_set_state from host memory, phl_step, phl_get_state into host memory.
    Several grids are in flight (three: measured 2.39 / 3.9 / 4.4e9
    cell-updates/s with one / two / three at 256^3), each on its own stream and
    driven by its own host thread (the ctypes calls release the GIL): while
    one grid's state crosses the host link, the others compute, and the two
    link directions run together.  Every step still copies its full input in
    and its result out.  Value: cell-updates of all steps of all grids over
    the wall time."""
    import threading
    import torch
    grids = [g]
    for _ in range(inflight - 1):
        gx = P.Grid(pr, precision=form, stream=torch.cuda.Stream().cuda_stream)
        if form == "mixed" and fused >= 0:
            gx.set_fused(fused)
        grids.append(gx)
    bufs = []
    for _ in grids:
        host = {k: torch.from_numpy(getattr(pr, k).copy()).pin_memory() for k in ("cons", "bx", "by", "bz")}
        out = {k: torch.empty_like(v).pin_memory() for k, v in host.items()}
        bufs.append((host, out))
    nbytes = sum(v.numel() * 8 for v in bufs[0][0].values())

    dev = torch.cuda.current_device()
    errors = []

    def run(gi, n):
        try:
            torch.cuda.set_device(dev)   # a new host thread starts on device 0
            gr, (host, out) = grids[gi], bufs[gi]
            for _ in range(n):
                gr.set_state(host["cons"], host["bx"], host["by"], host["bz"])
                gr.step(1)
                gr.get_state_into(out["cons"], out["bx"], out["by"], out["bz"])
        except Exception as exc:   # re-raised on the main thread
            errors.append(exc)

    for gi in range(inflight):   # one untimed round each (first touch of the pinned buffers and staging)
        run(gi, 1)
    torch.cuda.synchronize()
    th = [threading.Thread(target=run, args=(gi, steps)) for gi in range(inflight)]
    t0 = time.perf_counter()
    for t in th:
        t.start()
    for t in th:
        t.join()
    t1 = time.perf_counter()
    if errors:
        raise errors[0]
    for gr in grids:
        gr.check()
    for gr in grids[1:]:
        gr.close()
    val = pr.ncells * STAGES * inflight * steps / (t1 - t0)
    return {"value": val, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "steps": inflight * steps, "pipeline": f"{inflight} grids in flight (own stream and host thread each)"}


def host_info():
    """Core count and CPU model of the host the oracle runs on."""
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Architecture", "CPU(s)", "Thread(s) per core", "Socket(s)"):
                info[k.strip()] = v.strip()
    except Exception:
        pass
    return info


# The paper's own CPU figure (context only, other hardware): 1.03 us per cell
# per time step for the Godunov MHD update on one AMD EPYC 9554 core at 3.8 GHz
# (32^3, PPH + LHLLD + SSP-RK3, EOS excluded): 3 stages per step.
PAPER_CPU = {"value": 3.0 / 1.03e-6, "unit": UNIT, "cores": 1,
             "hardware": "AMD EPYC 9554 @3.8 GHz, one core (the paper's figure: 1.03 us per cell per step)",
             "note": "context only: another machine, PPH reconstruction, EOS excluded"}


def oracle_sample(steps=2, nxy=64, nz=256):
    """The CPU oracle as it stands, on a sample of the workload (the same box
    physics on nxy x nxy x nz cells): single-threaded, and the same sources
    built with OpenMP over all host cores (bit-identical results)."""
    import workloads as W
    import oracle as O
    pr = W.stratified_box(nxy, nxy, nz)
    legs = {}
    for par in (False, True):
        O.set_parallel(par)
        o = O.Oracle(pr)
        t0 = time.perf_counter()
        o.run(steps)
        legs[par] = time.perf_counter() - t0
    O.set_parallel(False)
    ncores = os.cpu_count()
    one, allc = legs[False], legs[True]
    return {"value": pr.ncells * STAGES * steps / allc, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": f"{nxy}x{nxy}x{nz} cells of the same box physics, {steps} SSP-RK3 steps: "
                      f"{allc:.1f} s on all {ncores} host cores (OpenMP build of the same C), "
                      f"{one:.1f} s single-threaded",
            "single_thread": {"value": pr.ncells * STAGES * steps / one, "unit": UNIT, "cores": 1},
            "host": host_info(), "paper_cpu_context": PAPER_CPU}


def run_reference(args):
    """The reference arm of this workload: the CPU oracle as it stands (the
    OpenMP build of its C over all host cores), on a sample of the box (64 x 64
    columns of the full height) per step."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import workloads as W
    import oracle as O
    O.set_parallel(True)
    nxy = 64
    pr = W.stratified_box(nxy, nxy, args.n)
    o = O.Oracle(pr)
    st = None
    for _ in range(args.warmup):
        st, _, _ = o.run(1, st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st, _, _ = o.run(1, st)
    dt = time.perf_counter() - t0
    val = pr.ncells * STAGES * args.steps / dt
    ncores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_cells": [nxy, nxy, args.n], "form": "oracle"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": f"{nxy}x{nxy}x{args.n} cells per step of the same box physics, "
                                   f"OpenMP over {ncores} host cores", "host": host_info()},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def l1_mixed_vs_fp64(P, pr, steps=3):
    """Per-field L1 of the mixed form against the FP64 form on the benchmark
    box after a few steps at the same fixed dt (deviations from the initial
    state for rho, m, E and the face field): ||q_mix - q_64||_1 / ||q_64 - q_0||_1."""
    import numpy as np
    g64 = P.Grid(pr, precision="fp64")
    g64.load()
    dt = g64.compute_dt()
    g64.step(steps, dt)
    a = g64.get_state()
    g64.close()
    gm = P.Grid(pr, precision="mixed")
    gm.load()
    gm.step(steps, dt)
    b = gm.get_state()
    gm.close()
    out = {}
    names = {0: "rho", 1: "mx", 2: "my", 3: "mz", 4: "E"}
    for v, nm in names.items():
        d0 = np.abs(a["cons"][v] - pr.cons[v]).sum()
        out[nm] = float(np.abs(b["cons"][v] - a["cons"][v]).sum() / max(d0, 1e-300))
    for k in ("bx", "by", "bz"):
        d0 = np.abs(a[k] - getattr(pr, k)).sum()
        out[k] = float(np.abs(b[k] - a[k]).sum() / max(d0, 1e-300)) if d0 > 0 else 0.0
    return {"steps": steps, "dt": dt, "l1_rel_of_change": out,
            "note": "||mixed - fp64||_1 / ||fp64 - initial||_1 per field at the same fixed dt"}


# the stellar box's mixed inversion (k_eos_cells<float> from each cell's record): FP64 operations
# per cell-stage, ncu on the 128^3 box (DADD + DMUL + 2 DFMA)
EOS_FP64_FLOP_PER_CELL = 721.0


def stellar_c3(P, n, steps, warmup, stream, ws, alu=None):
    """The same box with the stellar EOS (ions + radiation + e-/e+ pairs, 16O/28Si
    0.5/0.5, rho 1e5-1e7 g/cc): plain FP64 form (Newton from the previous T)
    vs the mixed form with the network's first guess, trained here on 1e7
    seeded EOS samples by the project's own kernels."""
    import numpy as np
    import workloads as W
    table = P.EosTable(nrho=321, nT=241)   # 80 nodes per decade: interpolation error ~1e-8 (P, e), ~4e-7 (c_v, gamma_c)
    net = P.Mlp(seed=7)
    train = net.train(table, nsamples=10_000_000, epochs=8, batch=4096, lr=1e-2, seed=2026)
    pr = W.stellar_box(n, n, n)
    out = {"workload": f"stellar box {n}^3 (ions + radiation + e-/e+ table EOS, 16O/28Si 0.5/0.5, "
                       f"rho 1e7 -> 1e5 g/cc polytrope, CGS), SSP-RK3",
           "mlp_training": train, "forms": {}}
    runs = (("fp64", "fp64", None, 0), ("mixed", "mixed", None, 0), ("mixed+mlp", "mixed", net, 1),
            ("mixed+mlp_cold_only", "mixed", net, 2))
    for name, prec, mlp, mode in runs:
        import torch
        g = P.Grid(pr, precision=prec, stream=stream.cuda_stream, eos_table=table, mlp=mlp, mlp_mode=mode)
        g.load()
        for _ in range(warmup):
            g.step(1)
        g.check()
        it0 = g.stats()["newton_iters"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(ws)
        with torch.cuda.stream(stream):
            e0.record(stream)
            g.step(steps)
            e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        ms = allreduce_max(e0.elapsed_time(e1), ws)
        g.check()
        it = g.stats()["newton_iters"] - it0
        kt = None
        if name == "mixed+mlp_cold_only":   # one more step with per-kernel events: the inversion's roofline
            g.set_timing(True)
            g.step(1)
            kt = g.kernel_times(reset=True)
            g.set_timing(False)
        g.close()
        out["forms"][name] = {"value": pr.ncells * STAGES * steps * ws / (ms * 1e-3), "unit": UNIT,
                              "ms_per_step": ms / steps,
                              "newton_iters_per_cell_stage": it / (pr.ncells * STAGES * steps)}
        if kt and "prim" in kt and alu:
            # the class holds the inversion and the ghost fill of each stage: per stage of the one timed step
            launches, kms = kt["prim"]
            avg = kms / STAGES
            tf = pr.ncells * EOS_FP64_FLOP_PER_CELL / (avg * 1e-3) / 1e12
            out["forms"][name]["kernels"] = {k: {"launches": v[0], "ms": v[1]} for k, v in kt.items()}
            out["roofline"] = {"kernel": "k_eos_cells (inversion, class prim: with the stage's ghost fill)",
                               "avg_stage_ms": avg,
                               "bound": "fp64", "achieved": tf, "peak": alu["fp64"], "unit": "TFLOP/s",
                               "frac": tf / alu["fp64"], "flop_per_cell": EOS_FP64_FLOP_PER_CELL,
                               "traffic": None,
                               "note": "DADD + DMUL + 2 DFMA per cell from ncu at 128^3 (recorded path); the class "
                                       "also holds the ghost fill",
                               "peak_kind": "measured FP64 DFMA rate (phl_probe_alu)"}
    f = out["forms"]
    out["mixed_mlp_over_fp64"] = f["mixed+mlp"]["value"] / f["fp64"]["value"]
    out["mixed_mlp_cold_only_over_fp64"] = f["mixed+mlp_cold_only"]["value"] / f["fp64"]["value"]
    out["network_mode"] = ("default use_mlp = 2: the network guesses T only where no previous T exists; "
                           "use_mlp = 1 (network first at every stage) loses in time stepping: its guess "
                           "needs more Newton steps than the previous step's T")
    # per-field L1 of the mixed + network form against the FP64 form, 3 steps at a fixed dt
    g64 = P.Grid(pr, precision="fp64", eos_table=table)
    g64.load()
    dt = g64.compute_dt()
    g64.step(3, dt)
    a = g64.get_state()
    g64.close()
    gm = P.Grid(pr, precision="mixed", eos_table=table, mlp=net, mlp_mode=2)
    gm.load()
    gm.step(3, dt)
    b = gm.get_state()
    gm.close()
    l1 = {}
    ref0 = P.Grid(pr, precision="fp64", eos_table=table)
    ref0.load()
    s0 = ref0.get_state()
    ref0.close()
    for v, nm in {0: "rho", 1: "mx", 2: "my", 3: "mz", 4: "E"}.items():
        d0 = np.abs(a["cons"][v] - s0["cons"][v]).sum()
        l1[nm] = float(np.abs(b["cons"][v] - a["cons"][v]).sum() / max(d0, 1e-300))
    l1["T"] = float(np.abs(b["T"] - a["T"]).sum() / max(np.abs(a["T"] - s0["T"]).sum(), 1e-300))
    out["l1_mixed_mlp_vs_fp64"] = {"steps": 3, "l1_rel_of_change": l1}
    net.close()
    table.close()
    return out


def diffusion_sts(P, n, stream, hbm_peak, peak_kind, reps=3):
    """Thermal diffusion by RKL2 super-time-stepping (phl_diffuse) on the same
    box: radiative conductivity K = k0 T^3 / rho sized so that the box's MHD
    step is ~100 parabolic limits (CFL_p ~ 100: ~20 stages, the paper's middle
    case).  Times whole super steps (one read-back of the parabolic rate, the
    set-up kernels, the stage kernels) with CUDA events, in the mixed form
    (float stages on the change of e_int) on the mixed grid and in the FP64
    form.  Algorithmic bytes per cell-stage of the stage kernel: mixed, it
    reads d^(m-1), d^(m-2), y0, the conductivity factor, 1/(rho c_v), the
    operator at d = 0 and three face differences and writes d^(m): 10 x 4 =
    40 B; FP64, it reads e_int^(m-1), e_int^(m-2), e_int^(0), the operator at
    e_int^(0), 1/rho and k0/rho^nR and writes e_int^(m): 7 x 8 = 56 B."""
    import torch
    pr = make_problem(n)
    cv = 1.0 / (pr.gamma - 1.0)
    g = P.Grid(pr, precision="mixed", stream=stream.cuda_stream)
    g.load()
    dt_h = g.compute_dt()
    # parabolic rate of K = k0 T^3/rho at the hottest, thinnest cell: D / dx^2 summed over 3 axes
    rho = pr.cons[0]
    T = (pr.cons[4] - 0.5 * (pr.cons[1] ** 2 + pr.cons[2] ** 2 + pr.cons[3] ** 2) / rho) / rho / cv
    rate1 = (T ** 3 / rho / (rho * cv)).max() * 3 * n * n     # for k0 = 1
    k0 = 100.0 / (2.0 * rate1 * dt_h)                          # dt_h / dt_p = 100
    def timed(form, dt):
        g.load()
        g.diffuse(dt, k0, nT=3, nR=1, cv=cv, precision=form)    # warm-up
        g.load()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                ns = g.diffuse(dt, k0, nT=3, nR=1, cv=cv, precision=form)
            e1.record(stream)
        torch.cuda.synchronize()
        g.check()
        return ns, e0.elapsed_time(e1) / reps

    out = {}
    for form, nbytes in (("mixed", 40.0), ("fp64", 56.0)):
        ns, ms = timed(form, dt_h)
        # the stage kernel alone: two super steps with different stage counts
        ns2, ms2 = timed(form, dt_h / 8.0)
        ms_stage = (ms - ms2) / (ns - ns2)
        rate = pr.ncells * ns / (ms * 1e-3)
        gbs = rate * nbytes / 1e9
        gbs_k = pr.ncells * nbytes / (ms_stage * 1e-3) / 1e9
        out[form] = {"stages": ns, "ms_per_super_step": ms, "value": rate, "unit": "cell-stages/s",
                     "bytes_per_cell_stage": nbytes,
                     "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                             "peak_kind": f"{peak_kind} HBM copy", "note": "whole super step incl. set-up"},
                     "stage_kernel": {"ms": ms_stage, "set_up_ms": ms - ns * ms_stage,
                                      "achieved": gbs_k, "peak": hbm_peak, "unit": "GB/s",
                                      "frac": gbs_k / hbm_peak,
                                      "method": f"(t({ns} stages) - t({ns2} stages)) / {ns - ns2}"}}
    g.close()
    res = {"workload": f"RKL2 thermal diffusion on the {n}^3 box, K = k0 T^3 / rho, dt = the MHD CFL step, "
                       f"CFL_p = 100"}
    res.update(out["mixed"])
    res["form"] = "mixed"
    res["fp64"] = out["fp64"]
    return res


POISSON_FLOP_PER_CELL_IT = 62.0     # FP64 flops per cell and BiCGSTAB iteration (FMA = 2), absolute criterion
POISSON_BYTES_PER_CELL_IT = 200.0   # algorithmic bytes per cell and iteration (25 vector reads/writes of 8 B)
FP64_NOMINAL_TFLOPS = 1.25          # GB300 dense FP64 (nominal)


def poisson_sphere(P, n, stream, hbm_peak, peak_kind, reps=2):
    """The paper's Poisson accuracy test at n^3: the (1 - r^2/r0^2)^2 sphere
    (r0 = 1/4, rho0 = 1, G = 1) on the (eta + eta^5)/4 stretched grid,
    monopole boundary values, absolute RMS residual below 1e-10, zero
    initial guess; FP64 BiCGSTAB with the Jacobi preconditioner
    (phl_poisson_solve).  Inputs resident on the device; CUDA-event time per
    solve, iterations, and the iteration against the FP64 and HBM rooflines
    (62 FP64 flops and 200 algorithmic bytes per cell and iteration)."""
    import torch
    import workloads as W
    xf = [W.stretched_faces(n)] * 3
    rho = torch.from_numpy(W.sphere_density(xf)).cuda()
    S = P.Poisson(xf, G=1.0, lmax=0, criterion="absolute", tol=1e-10, max_iter=20000,
                  stream=stream.cuda_stream)
    phi = torch.zeros_like(rho)
    with torch.cuda.stream(stream):
        S.solve(rho, phi)                                   # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            phi.zero_()
            _, it, res = S.solve(rho, phi)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    S.close()
    cells = n ** 3
    ms_it = ms / it
    tfl = cells * POISSON_FLOP_PER_CELL_IT / (ms_it * 1e-3) / 1e12
    gbs = cells * POISSON_BYTES_PER_CELL_IT / (ms_it * 1e-3) / 1e9
    return {"workload": f"Poisson sphere test on the stretched {n}^3 grid (monopole, |r| < 1e-10, phi0 = 0)",
            "iterations": it, "residual": res, "ms_per_solve": ms, "ms_per_iteration": ms_it,
            "value": cells * it / (ms * 1e-3), "unit": "cell-iterations/s",
            "fp64": {"achieved": tfl, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                     "frac": tfl / FP64_NOMINAL_TFLOPS, "peak_kind": "nominal FP64"},
            "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "peak_kind": f"{peak_kind} HBM copy"}}


def ensemble_c4(P, steps, warmup, stream, ws):
    """24 independent boxes of the stratified-box physics with edges drawn
    from {64, 96, 128, 160, 192} per axis (seed 2024), mixed form: one
    persistent launch per stage over all boxes, graph-captured step, launch
    shape from the autotuner.  Beside it, the same boxes stepped one after
    another with the per-kernel path."""
    import torch
    import workloads as W
    probs = W.ensemble()
    cells = sum(p.ncells for p in probs)
    E = P.Ensemble(probs, use_graph=True)
    E.load()
    tune = E.autotune(trial_steps=1)
    E.load()
    for _ in range(warmup):
        E.step(1)
    E.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(ws)
    e0.record()
    E.step(steps)
    e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    ms = allreduce_max(e0.elapsed_time(e1), ws)
    E.check()
    info = E.info()
    E.close()
    # the same boxes, one grid after another (per-kernel launches, no graph)
    grids = [P.Grid(p, precision="mixed") for p in probs]
    for g in grids:
        g.load()
        g.step(1)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        for g in grids:
            g.step(1)
    e1.record()
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    launches_seq = sum(g.stats()["kernels_per_step"] for g in grids)
    for g in grids:
        g.close()
    return {"workload": "24 stratified boxes (C2 physics), edges from {64,96,128,160,192} per axis, seed 2024, "
                        "mixed form", "boxes": [list(p.n) for p in probs], "cells": cells,
            "value": cells * STAGES * steps * ws / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "launch_shape": {"mode": ["persistent stage kernel", "one launch per phase",
                                      "per-box kernel chains on concurrent streams",
                                      "persistent stage kernel on the fused tiles"][info["mode"]],
                             "block": info["block"], "blocks_per_sm": info["blocks_per_sm"],
                             "streams": info["streams"]},
            "graph": info["graph"], "launches_per_step": info["launches_per_step"],
            "autotune": tune,
            "sequential_grids": {"value": cells * STAGES * steps / (ms_seq * 1e-3), "ms_per_step": ms_seq / steps,
                                 "launches_per_step": launches_seq}}


# Cubed-sphere shell (FP64): the flux kernel's FP64 operations per face
# (DADD + DMUL + 2 DFMA from the ncu SASS counters of k_sph_flux on the
# 6 x 64 x 64 x 64 shell: 4690.3 M over 4.743 M faces) and its DRAM bytes
# per face in the same capture (517.4 MB; the work arrays exceed L2 there).
SPH_FP64_FLOP_PER_FACE = 988.9
SPH_FLUX_DRAM_BYTES_PER_FACE = 109.1
# the mixed form's flux kernel: FP32 operations per face, FADD + FMUL + 2 FFMA
# of the scalar solver on the same shell (2533.6 M over 4.743 M faces; the
# packed-lane solver the kernel runs does the same arithmetic, partly as
# f32x2 instructions those counters leave out), and its DRAM bytes per face
# (241.0 MB in the capture of the packed-lane kernel)
SPH_FP32_FLOP_PER_FACE = 534.2
# the stellar shell's mixed inversion (k_sph_prims_st<float>, recorded path): FP64 operations and
# FP64-pipe instructions per cell-stage, ncu on the 6 x 64^3 stellar shell
SPH_ST_FP64_FLOP_PER_CELL = 722.0
SPH_ST_FP64_INST_PER_CELL = 507.1
SPH_MX_FLUX_DRAM_BYTES_PER_FACE = 50.8


def cubed_sphere_c5(P, steps, warmup, stream, alu, hbm_peak, peak_kind, N=256, Nr=384, precision="fp64",
                    eos="stellar", table=None, mlp=None):
    """The cubed-sphere shell 6 x N x N x Nr (phl_sphere_*): the n = 1.5
    polytrope between r = 0.2 and 1 under its own radial gravity, density
    noise 1e-3, a poloidal seed field at beta 1e5, heating in the inner 30%,
    LHLLD, CFL 0.4, reflecting radial walls, well-balanced, in the FP64 or
    the mixed form; eos "stellar": the stellar EOS (ions + radiation + e-/e+
    table, 16O/28Si 0.5/0.5, 1e7 -> 6.1e5 g/cm^3 across the shell), loaded
    from primitives and then reloaded without temperatures, so that the first
    (warm-up) inversion starts from the network's guess (a cold start) and
    every later one from the previous stage's T.  State resident on the
    device; CUDA events on the sphere's stream around K steps after W warm-up
    steps; then one more step with per-kernel timing."""
    import torch
    import workloads as W
    torch.cuda.empty_cache()
    pr = W.shell_problem(N, Nr, device="cuda", eos=eos)
    S = P.Sphere.from_problem(pr, stream=stream.cuda_stream, precision=precision, eos_table=table, mlp=mlp)
    torch.cuda.synchronize()          # the inputs were written on torch's stream
    S.load(pr)
    counts = S.counts()
    S.check()                         # synchronises the sphere's stream before the inputs go
    if eos == "stellar":              # the same state without temperatures: a cold start
        st = {k: torch.empty_like(getattr(pr, k)) for k in ("pa", "pb", "pr")}
        st["cons"] = torch.empty_like(pr.cons)
        S.get_state(st)
        S.set_state(st["cons"], st["pa"], st["pb"], st["pr"])
        S.check()
        del st
    del pr
    torch.cuda.empty_cache()
    S.set_graph(True)                 # each step one captured CUDA graph
    S.step(warmup)
    S.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    S.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    S.check()
    S.set_timing(True)
    S.step(1)
    kt = S.kernel_times(reset=True)
    S.set_timing(False)
    S.check()
    S.close()
    cells, faces = counts["cells"], counts["faces"]
    name, (launches, kms) = max(kt.items(), key=lambda kv: kv[1][1])
    avg = kms / max(launches, 1)
    eos_txt = ("stellar EOS (ions + radiation + e-/e+ table, 16O/28Si 0.5/0.5, rho 1e7 -> 6.1e5 g/cc; "
               "temperature guesses: the network on the cold start, then the previous stage's T)"
               if eos == "stellar" else "ideal gas gamma 5/3")
    out = {"workload": f"cubed-sphere shell 6 x {N} x {N} x {Nr} (r 0.2..1), n=1.5 polytrope, radial g, "
                       "density noise 1e-3 seed 1234, poloidal field beta 1e5, heating inner 30%, LHLLD, "
                       f"CFL 0.4, reflecting walls, well-balanced, {eos_txt}, {precision}",
           "cells": cells, "faces": faces, "edges": counts["edges"],
           "value": cells * STAGES * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
           "steps": steps, "warmup": warmup, "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kt.items()},
           "launches_per_step": sum(v[0] for v in kt.values()), "graph": True}
    roof = {"kernel": name, "avg_launch_ms": avg, "launches": launches}
    if eos == "stellar" and name == "sph_prim" and precision == "mixed":
        # the inversion: FP64-pipe bound; operation counts per cell from ncu (recorded path)
        tf = cells * SPH_ST_FP64_FLOP_PER_CELL / (avg * 1e-3) / 1e12
        inst = cells * SPH_ST_FP64_INST_PER_CELL / (avg * 1e-3) / 1e12
        roof.update({"bound": "fp64", "achieved": tf, "peak": alu["fp64"], "unit": "TFLOP/s",
                     "frac": tf / alu["fp64"], "flop_per_cell": SPH_ST_FP64_FLOP_PER_CELL,
                     "fp64_pipe_inst_per_cell": SPH_ST_FP64_INST_PER_CELL,
                     "fp64_pipe_inst_rate_frac": inst / (alu["fp64"] / 2.0),
                     "traffic": None,
                     "note": "DADD + DMUL + 2 DFMA per cell from ncu on the 6 x 64^3 stellar shell; the "
                             "instruction rate against the DFMA probe's (one FP64-pipe instruction per DFMA)",
                     "peak_kind": "measured FP64 DFMA rate (phl_probe_alu)"})
    elif eos == "stellar":
        roof["note"] = ("stellar EOS: the inversion (sph_prim) and the general-EOS solver (sph_flux) run FP64 "
                        "table work bound by the FP64 pipe; no per-cell operation count is taken for the FP64 form")
    elif name == "sph_flux" and precision == "fp64":
        # HBM view: W read once per cell, phi read and F, E, contact sign
        # written once per face
        b = cells * 64.0 + faces * (8.0 + 40.0 + 24.0 + 1.0)
        gbs = b / (avg * 1e-3) / 1e9
        roof["hbm"] = {"bytes_per_launch": b, "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                       "frac": gbs / hbm_peak, "peak_kind": f"{peak_kind} HBM copy"}
        tf = faces * SPH_FP64_FLOP_PER_FACE / (avg * 1e-3) / 1e12
        roof.update({"bound": "alu", "achieved": tf, "peak": alu["fp64"], "unit": "TFLOP/s",
                     "frac": tf / alu["fp64"], "flop_per_face": SPH_FP64_FLOP_PER_FACE,
                     "traffic": faces * SPH_FLUX_DRAM_BYTES_PER_FACE,
                     "traffic_note": "ncu DRAM bytes per face on the 6 x 64^3 shell x faces",
                     "peak_kind": "measured FP64 DFMA rate (phl_probe_alu)"})
    elif name == "sph_flux":
        # mixed: FP32 work arrays; W read once per cell, phi (FP64) and dPhi
        # (FP32) read, F, E (FP32) and the contact sign written once per face
        b = cells * 32.0 + faces * (8.0 + 4.0 + 20.0 + 12.0 + 1.0)
        gbs = b / (avg * 1e-3) / 1e9
        roof["hbm"] = {"bytes_per_launch": b, "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                       "frac": gbs / hbm_peak, "peak_kind": f"{peak_kind} HBM copy"}
        tf = faces * SPH_FP32_FLOP_PER_FACE / (avg * 1e-3) / 1e12
        roof.update({"bound": "alu", "achieved": tf, "peak": alu["fp32"], "unit": "TFLOP/s",
                     "frac": tf / alu["fp32"], "flop_per_face": SPH_FP32_FLOP_PER_FACE,
                     "traffic": faces * SPH_MX_FLUX_DRAM_BYTES_PER_FACE,
                     "traffic_note": "ncu DRAM bytes per face on the 6 x 64^3 shell x faces",
                     "peak_kind": "measured FP32 FFMA rate (phl_probe_alu)"})
    out["roofline"] = roof
    return out


def cubed_sphere_forms(P, args, stream, alu, hbm_peak, peak_kind):
    """The stellar shell in the mixed form (the value) and in the FP64 form
    beside it; the ideal-gas shell's mixed form for reference."""
    import time
    table = P.EosTable(nrho=321, nT=241)
    mlp = P.Mlp(seed=7)
    t0 = time.perf_counter()
    mlp.train(table, nsamples=2_000_000, epochs=4, batch=1024, lr=1e-2, seed=2026)
    t_train = time.perf_counter() - t0
    mx = cubed_sphere_c5(P, args.c5_steps_mixed, 2, stream, alu, hbm_peak, peak_kind, args.c5_n, args.c5_nr,
                         "mixed", "stellar", table, mlp)
    f64 = cubed_sphere_c5(P, args.c5_steps, 1, stream, alu, hbm_peak, peak_kind, args.c5_n, args.c5_nr, "fp64",
                          "stellar", table, mlp)
    mx["fp64"] = f64
    mx["mixed_over_fp64"] = mx["value"] / f64["value"]
    mx["mlp_training_s"] = t_train
    ideal = cubed_sphere_c5(P, args.c5_steps_mixed, 2, stream, alu, hbm_peak, peak_kind, args.c5_n, args.c5_nr,
                            "mixed", "ideal")
    mx["ideal_gas_mixed"] = {k: ideal[k] for k in ("workload", "value", "unit", "ms_per_step", "kernels", "roofline")}
    mlp.close()
    table.close()
    return mx


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="both", choices=["fp64", "mixed", "both"],
                    help="both: time the plain FP64 form and the mixed form; the value is the mixed form's")
    ap.add_argument("--n", type=int, default=256, help="box edge (256 is the benchmark workload)")
    ap.add_argument("--fused", type=int, default=-1,
                    help="mixed stage: 0 = per-direction face kernels, 1..4 = fused tile kernel launch shape "
                         "(default: the library's choice)")
    ap.add_argument("--no-pph", action="store_true", help="skip the mixed form with PPH reconstruction")
    ap.add_argument("--no-sts", action="store_true", help="skip the RKL2 thermal-diffusion super step")
    ap.add_argument("--sts-only", action="store_true",
                    help="time only the RKL2 thermal-diffusion super step (print its object; for profiling)")
    ap.add_argument("--no-poisson", action="store_true", help="skip the Poisson solve")
    ap.add_argument("--poisson-only", action="store_true",
                    help="time only the Poisson solve (print its object; for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-l1", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-c3", action="store_true", help="skip the stellar-EOS box (mixed + network vs FP64)")
    ap.add_argument("--c3-steps", type=int, default=4)
    ap.add_argument("--c3-only", action="store_true",
                    help="only the stellar-EOS box (its JSON object alone, for profiling)")
    ap.add_argument("--no-c4", action="store_true", help="skip the 24-box ensemble")
    ap.add_argument("--c4-steps", type=int, default=5)
    ap.add_argument("--c4-only", action="store_true", help="only the 24-box ensemble (its JSON object alone)")
    ap.add_argument("--no-c5", action="store_true", help="skip the cubed-sphere shell")
    ap.add_argument("--c5-steps", type=int, default=2, help="cubed sphere: timed FP64 steps")
    ap.add_argument("--c5-steps-mixed", type=int, default=5, help="cubed sphere: timed mixed steps")
    ap.add_argument("--c5-precision", default="both", choices=["fp64", "mixed", "both"])
    ap.add_argument("--c5-eos", default="stellar", choices=["stellar", "ideal"],
                    help="cubed sphere with one precision: the EOS (both precisions: stellar, plus the ideal gas's "
                         "mixed form for reference)")
    ap.add_argument("--c5-only", action="store_true", help="only the cubed-sphere shell (its JSON object alone)")
    ap.add_argument("--c5-n", type=int, default=256, help="cubed sphere: angular cells per patch side")
    ap.add_argument("--c5-nr", type=int, default=384, help="cubed sphere: radial cells")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P

    hbm_peak, peak_kind = read_peaks()
    stream = torch.cuda.Stream()
    alu = {k: P.probe_alu(k) for k in ("fp32", "fp64")}
    if args.sts_only:
        if rank == 0:
            print(json.dumps(diffusion_sts(P, args.n, stream, hbm_peak, peak_kind)))
        return 0
    if args.poisson_only:
        if rank == 0:
            print(json.dumps(poisson_sphere(P, args.n, stream, hbm_peak, peak_kind)))
        return 0
    if args.c4_only:
        c4 = ensemble_c4(P, args.c4_steps, 2, stream, ws)
        if rank == 0:
            print(json.dumps(c4))
        return 0
    if args.c5_only:
        if rank == 0:
            if args.c5_precision == "both":
                print(json.dumps(cubed_sphere_forms(P, args, stream, alu, hbm_peak, peak_kind)))
            else:
                steps = args.c5_steps if args.c5_precision == "fp64" else args.c5_steps_mixed
                table = mlp = None
                if args.c5_eos == "stellar":
                    table = P.EosTable(nrho=321, nT=241)
                    mlp = P.Mlp(seed=7)
                    mlp.train(table, nsamples=2_000_000, epochs=4, batch=1024, lr=1e-2, seed=2026)
                print(json.dumps(cubed_sphere_c5(P, steps, 1, stream, alu, hbm_peak, peak_kind, args.c5_n,
                                                 args.c5_nr, args.c5_precision, args.c5_eos, table, mlp)))
        return 0
    if args.c3_only:
        c3 = stellar_c3(P, args.n, args.c3_steps, 2, stream, ws, alu)
        if rank == 0:
            print(json.dumps(c3))
        return 0
    pr = make_problem(args.n)
    props = torch.cuda.get_device_properties(local)
    gpu_id = getattr(props, "uuid", None)
    gpu_id = f"GPU-{gpu_id}" if gpu_id is not None and not str(gpu_id).startswith("GPU-") else (gpu_id or local)
    forms = ["fp64", "mixed"] if args.form == "both" else [args.form]
    head = forms[-1]
    res = {}
    clk = None
    for form in forms:
        clocks = Clocks(gpu_id) if form == head else None
        g, ms, kt, st = time_form(P, pr, form, args.steps, args.warmup, stream, ws, args.fused)
        if clocks is not None:
            clk = clocks.stop()
        value, ms_max = whole_job_rate(pr.ncells * STAGES * args.steps, ms, ws)
        res[form] = dict(g=g, ms=ms_max, kt=kt, value=value)
        if form != head:
            g.close()
    h = res[head]
    g = h["g"]
    roof = roofline(h["kt"], pr, head, hbm_peak, peak_kind, alu)
    roof_hbm = kernel_hbm(h["kt"], pr, hbm_peak, peak_kind)
    e2e = e2e_measure(P, g, pr, args.e2e_steps, head, args.fused)
    g.close()
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample()
    l1 = None
    if rank == 0 and len(forms) == 2 and not args.no_l1:
        l1 = l1_mixed_vs_fp64(P, pr)
    c3 = None
    if not args.no_c3 and len(forms) == 2:
        c3 = stellar_c3(P, args.n, args.c3_steps, 2, stream, ws, alu)
    c4 = None
    if not args.no_c4 and len(forms) == 2:
        c4 = ensemble_c4(P, args.c4_steps, 2, stream, ws)
    sts = None
    if not args.no_sts and len(forms) == 2:
        sts = diffusion_sts(P, args.n, stream, hbm_peak, peak_kind)
    poisson = None
    if not args.no_poisson and len(forms) == 2:
        poisson = poisson_sphere(P, args.n, stream, hbm_peak, peak_kind)
    c5 = None
    if not args.no_c5 and len(forms) == 2:
        c5 = cubed_sphere_forms(P, args, stream, alu, hbm_peak, peak_kind)
    launches = sum(v[0] for v in h["kt"].values())
    forms_out = {f: {"value": r["value"], "ms_per_step": r["ms"] / args.steps,
                     "stage_hbm": stage_hbm(r["value"] / max(ws, 1), f, hbm_peak, peak_kind),
                     "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in r["kt"].items()}}
                 for f, r in res.items()}
    if len(forms) == 2:
        forms_out["mixed_over_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
    if "mixed" in forms and not args.no_pph:
        # the same box with the PPH reconstruction (Sect. 2.5, item ii), the
        # paper's production choice: the mixed form, same steps
        q = pr.copy()
        q.recon = "pph"
        gp, msp, _, _ = time_form(P, q, "mixed", args.steps, args.warmup, stream, ws, args.fused)
        gp.close()
        vp, msp = whole_job_rate(pr.ncells * STAGES * args.steps, msp, ws)
        forms_out["mixed_pph"] = {"value": vp, "ms_per_step": msp / args.steps}
        # the limited fifth-order reconstruction (item iii): per-direction mixed
        # kernels (the fused tile stages two ghost layers; PQH needs three)
        q = pr.copy()
        q.recon = "pqh"
        gq, msq, _, _ = time_form(P, q, "mixed", args.steps, args.warmup, stream, ws, 0)
        gq.close()
        vq, msq = whole_job_rate(pr.ncells * STAGES * args.steps, msq, ws)
        forms_out["mixed_pqh"] = {"value": vq, "ms_per_step": msq / args.steps, "path": "per-direction kernels"}
    line = {
        "metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": h["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": pr.ncells, "n": list(pr.n), "form": head,
                   "forms_timed": forms, "stages_per_step": STAGES, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (state 1.07 GB per copy, no flush)"},
        "roofline": roof,
        "roofline_hbm": roof_hbm,
        "alu_peaks_measured": alu,
        "forms": forms_out,
        "l1_mixed_vs_fp64": l1,
        "stellar_eos_box": c3,
        "ensemble_24_boxes": c4,
        "thermal_diffusion_sts": sts,
        "poisson_sphere": poisson,
        "cubed_sphere_shell": c5,
        "gpu_launches": launches,
        "e2e": e2e,
        "clocks": clk,
        "cpu_baseline": cpu,
        "stage_hbm": stage_hbm(h["value"] / max(ws, 1), head, hbm_peak, peak_kind),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
