#!/usr/bin/env python
"""Throughput of the GB300 CT-MHD step: cell-updates/s (FP64) on the 256^3 decaying-turbulence
workload, with the live roofline of the dominant kernel, an end-to-end number through the C ABI
with host buffers, clocks sampled during the timed region, and the CPU oracle as baseline.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

One step = one mhd_step_cfl of the whole box: the CFL time step (CFL 0.3, computed on the device)
and a full RK2-SSP step (two stages, first-order flux correction on). N > 1 (torchrun) runs one independent box per
GPU (replicas; the path is not sharded) and reports the aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per GB300 (FP64, plain vs batched vs fwd+adjoint), % HBM roofline"
UNIT = "cell-updates/s"

# Roofline constants: GB300 FP64 = 152 SMs x 2 DFMA/clk x 2 flops at 2070 MHz (the recipe's SM
# count and maximum clock; the DFMA rate per SM per clock is measured by mhd_fp64_rate, which the
# bench runs and reports). Algorithmic FP64 flops (one per +, -, *, /, sqrt) counted by the
# oracle's op-counting scalar (python -m oracle.count_flops): per face of the face sweep
# (reconstruction of 7 primitives + Riemann solve + Joule flux) and per cell-update of the whole
# step, HLLD counted one-sided (the states of the fan region the face lies in; the full count, with
# both sides' star states formed everywhere, is beside it). Turbulence: four 48^3 cuts of the timed
# 256^3 state; the others on 32^3 (fast wave, Alfven wave) and 64 x 64 x 4 (Harris sheet) samples.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FLOPS_PER_FACE = {"turbulence": 286.0, "turbulence_full_hlld": 303.7, "alfven_ppm_ep": 455.2,
                  "fast_wave": 249.0, "harris": 361.3}
FLOPS_PER_CELL_UPDATE = {"turbulence": 2746.0, "turbulence_full_hlld": 2852.6, "alfven_ppm_ep": 3628.6,
                         "fast_wave": 2325.3, "harris": 2968.1}
HBM_PEAK_GBS = 6759.6  # measured copy bandwidth of this GPU model (STREAM-style copy)
ALG_BYTES_PER_CELL_UPDATE = 320  # stage 1: 64 B in + 64 B out; stage 2: 128 B in + 64 B out
# DRAM traffic of one face-sweep launch (the x, y and z sweeps of a stage; mean of a stage-1 and a
# stage-2 launch) from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), valid only for the kernel sources it was taken on.
TRAFFIC = {"face": {"bytes_per_launch": 2305.9e6, "cells": 160**3, "src": "cf90455b07c49ff7"}}


# what the face sweep's machine code is compiled from: its kernel, the numerics and indexing
# headers, and the layout of the parameter struct it receives
FACE_SOURCES = ("mhd_face.cu", "mhd_face.cuh", "mhd_device.cuh", "mhd_index.cuh")


def kernel_src_hash(files=FACE_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2609_10816_gb300", "csrc")
    for f in sorted(files):
        h.update(open(os.path.join(csrc, f), "rb").read())
    internal = open(os.path.join(csrc, "mhd_internal.cuh")).read()
    i0 = internal.index("struct Dev {")
    h.update(internal[i0:internal.index("};", i0)].encode())
    return h.hexdigest()[:16]


def max_over_ranks(x, dist, dev):
    """The largest of the ranks' values of x (the slowest rank's time); x itself at N = 1."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second, timed by the slowest rank (replicas: every rank
    advances its own box of the same size)."""
    return world * units_per_rank / (ms / 1e3)


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(n):
    from paper_2609_10816_gb300 import inputs

    cons, b, info = inputs.turbulence((n, n, n), seed=2, v_rms=5.0)
    return cons, b, info


WORKLOAD_NAME = ("{n}^3 periodic FP64 ideal decaying MHD turbulence: rho=1, B0=(0,0,0.5), p=rho/gamma, "
                 "seeded solenoidal velocity, E(k)~k^-2 on 1<=|k|<=3, rms Mach 5; PPM+HLLD, Q26 EMF "
                 "compute + LD04 averaging, RK2-SSP with first-order flux correction, CFL 0.3")


# the CPU oracle's workloads: recipe -> (inputs, scheme)
ORACLE_RECIPES = {
    "turbulence": dict(recon="ppm", riemann="hlld", emf="q26", eta=0.0),
    "fast_wave": dict(recon="plm_mc", riemann="hll", emf="q26", eta=0.0),
    "harris": dict(recon="plm_mc", riemann="hlld", emf="q26", eta=1e-4),
}


_W = None  # the oracle worker's box (set in each spawned process)


def _oracle_worker_init(recipe, shape):
    """Spawned process: the oracle and one box of a workload's recipe."""
    global _W
    import oracle
    from paper_2609_10816_gb300 import inputs

    if recipe == "turbulence":
        cons, b, info = inputs.turbulence(shape, seed=2, v_rms=5.0)
    elif recipe == "fast_wave":
        cons, b, info = inputs.fast_wave(shape)
    else:
        cons, b, info = inputs.harris_sheet(shape)
    sch = ORACLE_RECIPES[recipe]
    _W = {"cfg": oracle.Config(shape=shape, h=info["h"], **sch), "cons": cons, "b": b}


def _oracle_worker_steps(arg):
    """Advance this process's box by CFL steps for budget_s seconds (or `steps` steps): (steps, s)."""
    import oracle

    budget_s, steps = arg
    w = _W
    k, t0 = 0, time.perf_counter()
    while (steps is None and time.perf_counter() - t0 < budget_s) or (steps is not None and k < steps):
        dt = oracle.max_dt(w["cfg"], w["cons"], w["b"], 0.3)
        w["cons"], w["b"], _ = oracle.step(w["cfg"], w["cons"], w["b"], dt)
        k += 1
    return k, time.perf_counter() - t0


def _oracle_pool(n, procs, recipe="turbulence", shape=None):
    import multiprocessing as mp

    shape = shape or (n, n, n)
    return mp.get_context("spawn").Pool(procs, initializer=_oracle_worker_init, initargs=(recipe, shape))


def oracle_rate(recipe, shape, budget_s, procs):
    """Cell-updates/s of the oracle on `procs` processes, each advancing its own box for budget_s."""
    with _oracle_pool(0, procs, recipe, shape) as pool:
        pool.map(_oracle_worker_steps, [(0.0, 1)] * procs)
        res = pool.map(_oracle_worker_steps, [(budget_s, None)] * procs)
    ncell = shape[0] * shape[1] * shape[2]
    return sum(ncell * k / el for k, el in res), sum(k for k, _ in res)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(budget_s=12.0, n=48):
    """The oracle as it stands, single-threaded per process, on every host core at once: one
    spawned process per core advances its own box of the workload's recipe for budget_s seconds;
    the rate is the sum over processes."""
    procs = host_cores()
    rate, steps = oracle_rate("turbulence", (n, n, n), budget_s, procs)
    one, _ = oracle_rate("turbulence", (n, n, n), budget_s / 3, 1)
    fw, _ = oracle_rate("fast_wave", (32, 32, 32), budget_s / 3, procs)
    hs, _ = oracle_rate("harris", (128, 128, 4), budget_s / 3, procs)
    return {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes (one per host core), each advancing its own {n}^3 box of the same recipe "
                      f"(PPM+HLLD+Q26+LD04, CFL dt + RK2/FOFC step) for {budget_s:.0f} s: {steps} steps in all",
            "one_core": one,
            "other_configs_all_cores": {"fast_wave_32cubed_plm_hll": fw,
                                        "harris_128x128x4_plm_hlld_eta1e-4": hs}}


def run_reference(args):
    """--impl reference: the CPU oracle timed on every host core (one process per core, each
    advancing its own 32^3 box of the workload's recipe), one step per process per timed step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = 32
    procs = host_cores()
    with _oracle_pool(n, procs) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_worker_steps, [(0.0, 1)] * procs)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_oracle_worker_steps, [(0.0, 1)] * procs)
        el = time.perf_counter() - t0
    v = procs * n**3 * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME.format(n=256),
                   "sample": f"{procs} boxes of {n}^3 per step, one per host core"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": f"{args.steps} timed steps; each advances {procs} independent {n}^3 boxes of "
                                   f"the same recipe, one oracle process per host core"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_batched(args, dev, stream, barrier, dist, world, same_state=None):
    """1024 patches, edges uniform from {16, 24, 32, 48, 64} (seed 4), cell width 1/64, smooth
    random states; PPM + HLLD + Q26 + LD04; schedule from the autotuner; one CUDA-graph replay per
    step (CFL reduction + dt + the persistent stage launches); then FS18 and B25a from the same
    state with the same schedule."""
    import numpy as np
    import torch

    from paper_2609_10816_gb300 import inputs, mhd

    dims = [tuple(int(x) for x in d) for d in inputs.patch_dims(args.npatch, seed=4)]
    rng = np.random.default_rng(4)
    h = 1.0 / 64
    bt = mhd.Batch(dims, h, stream=stream)
    pats = [inputs.random_patch(d, rng, h=h)[:2] for d in dims]
    cons, b = bt.pack(pats, dev)
    del pats
    sch = mhd.scheme("ppm", "hlld", "q26")
    sched = bt.tune(cons, b, 0.3, sch)
    # the initial state again for the comparisons below (the other launch form; FS18 / B25a)
    start = (cons.clone(), b.clone())

    def timed(scheme):
        for _ in range(3):
            bt.step(cons, b, 0.3, scheme)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            bt.step(cons, b, 0.3, scheme)
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), dist, dev)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = timed(sch)
    dt = bt.last_dt()  # also raises on a barrier timeout
    flagged = bt.stats()
    phases = {f"stage{st + 1}": {k: round(v, 3) for k, v in ph.items()} for st, ph in bt.phase_ms().items()}
    nl = sched["launches_per_stage"]
    form = {1: "one persistent launch per stage", 3: "per stage 3 persistent launches (faces; edges, update, "
            "flags; first-order correction, which exits at once when nothing is flagged)"}
    out = {"batched": whole_job_rate(bt.ncell * args.steps, world, ms),
           "batched_config": {"patches": len(dims), "cells_per_gpu": bt.ncell, "schedule": sched,
                              "ms_per_step": ms / args.steps, "last_dt": dt,
                              "fofc_flagged_last_step": list(flagged),
                              "phase_ms_last_step": phases,
                              "launches_per_step": f"1 graph: maxspeed, set_dt, {form[nl]}"}}
    # the launch form the tuner did not pick, same schedule otherwise
    cons.copy_(start[0])
    b.copy_(start[1])
    bt.set_launches(4 - nl)
    out[f"batched_{4 - nl}_launches_per_stage"] = whole_job_rate(bt.ncell * args.steps, world, timed(sch))
    bt.set_launches(nl)
    if not args.q26_only:
        # the other EMF compute schemes on the same patches from the same state, same schedule
        for emf in ("fs18", "b25a"):
            cons.copy_(start[0])
            b.copy_(start[1])
            ms_e = timed(mhd.scheme("ppm", "hlld", emf))
            bt.last_dt()
            out[f"batched_{emf}"] = whole_job_rate(bt.ncell * args.steps, world, ms_e)
    del start
    bt.close()
    del cons, b
    if same_state is not None:
        # the batch machinery on the plain form's own state (one box, same cells, same physics):
        # separates the cost of the batched kernel from that of the patches' different flow
        c0, b0, h0 = same_state
        n0 = c0.shape[1]
        bt = mhd.Batch([(n0, n0, n0)], h0, stream=stream)
        cons, b = bt.pack([(c0, b0)], dev)
        bt.set_schedule(seg=64, order=1, blocks_per_sm=0, use_graph=True)
        c_start, b_start = cons.clone(), b.clone()
        for nl_s in (3, 1):  # three launches per stage, then one
            cons.copy_(c_start)
            b.copy_(b_start)
            bt.set_launches(nl_s)
            ms = timed(sch)
            bt.last_dt()
            key = f"batched_1x{n0}cubed_same_state" + ("" if nl_s == 3 else "_one_launch_per_stage")
            out[key] = whole_job_rate(n0**3 * args.steps, world, ms)
            out["batched_config"]["same_state_phase_ms_last_step" + ("" if nl_s == 3 else "_one_launch")] = {
                f"stage{st + 1}": {k: round(v, 3) for k, v in ph.items()} for st, ph in bt.phase_ms().items()}
        del c_start, b_start
        bt.close()
    return out


def run_alfven(args, dev, stream, barrier, dist, world):
    """The paper's throughput problem (Sec. 5.2): linearly polarised Alfven wave, k L / 2 pi =
    (1, 2, 3), theta = pi/4, rho = b_bg = 1, p = 1/gamma, at its per-GPU size (128^3 by default)
    for 100 CFL steps, PPM-EP + HLLD with each EMF compute scheme and LD04 averaging (the paper's
    B25b averaging is not defined in it), and Q26 with plain PPM beside them."""
    import torch

    from paper_2609_10816_gb300 import inputs, mhd

    n, steps = args.alfven_n, args.alfven_steps
    cons, b, info = inputs.alfven_oblique((n, n, n))
    ctx = mhd.Context((n, n, n), info["h"], stream=stream)
    out = {}
    for recon, emf in (("ppm_ep", "q26"), ("ppm_ep", "fs18"), ("ppm_ep", "b25a"), ("ppm", "q26")):
        sch = mhd.scheme(recon, "hlld", emf)
        st = mhd.to_device(cons, b, dev)
        for _ in range(3):
            ctx.step_cfl(st, 0.3, sch)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.step_cfl(st, 0.3, sch)
        e1.record(stream)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        out[f"alfven{n}_{emf}" + ("" if recon == "ppm_ep" else "_plain_ppm")] = whole_job_rate(n**3 * steps, world, ms)
        del st
    ctx.close()
    out[f"alfven{n}_config"] = {"cells": n**3, "steps": steps,
                                "scheme": "PPM-EP + HLLD + {Q26, FS18, B25a} + LD04 (and Q26 with PPM)",
                                "q26_fp64_frac_of_nominal_peak": out[f"alfven{n}_q26"] / world * FLOPS_PER_CELL_UPDATE[
                                    "alfven_ppm_ep"] / 1e12 / FP64_PEAK_TFLOPS,
                                "q26_speedup_vs_fs18": out[f"alfven{n}_q26"] / out[f"alfven{n}_fs18"] - 1,
                                "q26_speedup_vs_b25a": out[f"alfven{n}_q26"] / out[f"alfven{n}_b25a"] - 1}
    return out


def _timed_steps(ctx, st, sch, eta, steps, stream, barrier, dist, dev, graph=False):
    """ms of `steps` mhd_step_cfl calls (CFL 0.3) after three warm-up steps; with graph, the steps
    are recorded once as a CUDA graph and the graph is replayed."""
    import torch

    for _ in range(3):
        ctx.step_cfl(st, 0.3, sch, eta)
    g = None
    if graph:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(steps):
                ctx.step_cfl(st, 0.3, sch, eta)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    if graph:
        g.replay()
    else:
        for _ in range(steps):
            ctx.step_cfl(st, 0.3, sch, eta)
    e1.record(stream)
    barrier()
    ctx.last_dt()  # raises on a non-finite signal speed
    return max_over_ranks(e0.elapsed_time(e1), dist, dev)


def run_c1(args, dev, stream, barrier, dist, world):
    """The 32^3 fast eigenmode along the box diagonal (rho0 = 1, p0 = 1/gamma, b0 oblique, amplitude
    1e-6), PLM-MC + HLL + Q26 + LD04, CFL 0.3, 100 steps of mhd_step_cfl, called eagerly and, timed
    beside it, recorded once as a CUDA graph and replayed (no host launch cost)."""
    from paper_2609_10816_gb300 import inputs, mhd

    shape, steps = (32, 32, 32), 100
    cons, b, info = inputs.fast_wave(shape)
    ctx = mhd.Context(shape, info["h"], stream=stream)
    sch = mhd.scheme("plm_mc", "hll", "q26")
    out = {}
    for graph in (False, True):
        st = mhd.to_device(cons, b, dev)
        ms = _timed_steps(ctx, st, sch, 0.0, steps, stream, barrier, dist, dev, graph=graph)
        out["c1_fast_wave_32cubed" + ("_in_graph" if graph else "")] = whole_job_rate(32**3 * steps, world, ms)
    md, mb = ctx.divb(st)
    ctx.close()
    r = out["c1_fast_wave_32cubed"] / world
    out["c1_config"] = {"cells": 32**3, "steps": steps, "scheme": "PLM-MC + HLL + Q26 + LD04",
                        "fp64_frac_of_nominal_peak": r * FLOPS_PER_CELL_UPDATE["fast_wave"] / 1e12 / FP64_PEAK_TFLOPS,
                        "hbm_frac": r * ALG_BYTES_PER_CELL_UPDATE / 1e9 / HBM_PEAK_GBS,
                        "max_divb_dx_over_b": md * info["h"][0] / mb}
    return out


def run_c3(args, dev, stream, barrier, dist, world):
    """512 x 512 x 4 resistive reconnection (periodic double Harris sheet, beta 0.2, seeded 1e-3
    velocity noise), eta = 1e-4, PLM-MC + HLLD + Q26 + LD04, CFL 0.3, 200 steps."""
    from paper_2609_10816_gb300 import inputs, mhd

    shape, steps, eta = (512, 512, 4), 200, 1e-4
    cons, b, info = inputs.harris_sheet(shape)
    ctx = mhd.Context(shape, info["h"], stream=stream)
    sch = mhd.scheme("plm_mc", "hlld", "q26")
    st = mhd.to_device(cons, b, dev)
    ms = _timed_steps(ctx, st, sch, eta, steps, stream, barrier, dist, dev)
    # the kernel split from 20 more steps with the library's per-class events on
    ctx.profile(True)
    ctx.profile_read(reset=True)
    for _ in range(20):
        ctx.step_cfl(st, 0.3, sch, eta)
    barrier()
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    N = 512 * 512 * 4
    md, mb = ctx.divb(st)
    s1, s2 = ctx.stats()
    ctx.close()
    r = N * steps / (ms / 1e3)
    return {"c3_reconnection_512x512x4": whole_job_rate(N * steps, world, ms),
            "c3_config": {"cells": N, "steps": steps, "eta": eta, "scheme": "PLM-MC + HLLD + Q26 + LD04",
                          "ms_per_step": ms / steps,
                          "fp64_frac_of_nominal_peak": r * FLOPS_PER_CELL_UPDATE["harris"] / 1e12 / FP64_PEAK_TFLOPS,
                          "hbm_frac": r * ALG_BYTES_PER_CELL_UPDATE / 1e9 / HBM_PEAK_GBS,
                          "max_divb_dx_over_b": md * info["h"][0] / mb, "fofc_flagged_last_step": [s1, s2],
                          "kernels_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]}}}


def run_adjoint_step(args, dev, stream, barrier, dist, world):
    """The adjoint step alone: 64^3 turbulence at Mach 2 (the differentiation workload's state),
    PPM + HLLD + Q26 + LD04, eta = 1e-3, mhd_step_adjoint called `adj_reps` times with a seeded
    random adjoint state (each call reruns the forward stages it needs); ms per adjoint step."""
    import numpy as np
    import torch

    from paper_2609_10816_gb300 import inputs, mhd

    n, eta = args.adj_n, 1e-3
    cons, b, info = inputs.turbulence((n, n, n), seed=2, v_rms=2.0)
    ctx = mhd.Context((n, n, n), info["h"], stream=stream)
    sch = mhd.scheme("ppm", "hlld", "q26")
    st = mhd.to_device(cons, b, dev)
    dt = ctx.max_dt(st, 0.3, eta)
    rng = np.random.default_rng(8)
    lam = mhd.to_device(rng.normal(size=cons.shape), rng.normal(size=b.shape), dev)
    ctx.step_adjoint(st, lam, dt, sch, eta)  # warm-up (allocates the adjoint scratch)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.adj_reps):
        ctx.step_adjoint(st, lam, dt, sch, eta)
    e1.record(stream)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev) / args.adj_reps
    ctx.close()
    return {"adjoint_step_ms": ms, "adjoint_step_config": {"cells": n**3, "calls": args.adj_reps, "eta": eta}}


def run_fwd_adjoint(args, dev, stream, barrier, dist, world):
    """64^3 turbulence at Mach 2 (rho = 1, B0 = (0,0,0.5), p = rho/gamma), eta = 1e-3, PPM + HLLD
    + Q26 + LD04, 20 steps with the dt sequence frozen from a first forward pass, checkpoints
    every 5 steps; loss = sum of b^2 at the final time; gradients in the initial velocity field
    (rho and p held) and eta. Throughput counts cell-updates of the forward pass per second of
    forward + backward time. Central differences (h = 1e-6) on 16 random directions check it."""
    import numpy as np
    import torch

    from paper_2609_10816_gb300 import adjoint, inputs, mhd

    n, nsteps, eta0 = args.adj_n, 20, 1e-3
    cons, b, info = inputs.turbulence((n, n, n), seed=2, v_rms=2.0)
    ctx = mhd.Context((n, n, n), info["h"], stream=stream)
    sch = mhd.scheme("ppm", "hlld", "q26")
    st = mhd.to_device(cons, b, dev)
    dts = []
    for _ in range(nsteps):  # freeze the dt sequence
        dts.append(ctx.max_dt(st, 0.3, eta0))
        ctx.step(st, dts[-1], sch, eta0)
    rho = torch.tensor(cons[0], device=dev)
    p = rho / (5.0 / 3.0)
    bt = torch.tensor(b, device=dev)
    u_init = torch.tensor(cons[1:4] / cons[0], device=dev)

    def init(u):
        bc = 0.5 * (bt + torch.stack([torch.roll(bt[d], -1, dims=2 - d) for d in range(3)]))
        e = p / (5.0 / 3.0 - 1.0) + 0.5 * rho * (u * u).sum(0) + 0.5 * (bc * bc).sum(0)
        return torch.cat([rho[None], rho * u, e[None]], 0).contiguous()

    def loss(u, e):
        cf, bf = adjoint.evolve(init(u), bt, e, ctx, dts, sch, every=5)
        return (bf * bf).sum()

    def one():
        u = u_init.clone().requires_grad_(True)
        e = torch.tensor(eta0, dtype=torch.float64, requires_grad=True)
        L = loss(u, e)
        L.backward()
        return u.grad, e.grad

    one()  # warm-up (allocates the adjoint scratch)
    barrier()
    t0 = time.perf_counter()
    reps = 2
    for _ in range(reps):
        gu, ge = one()
    torch.cuda.synchronize(dev)
    el = (time.perf_counter() - t0) / reps
    el = max_over_ranks(el, dist, dev)
    # central differences on 16 random directions
    rng = np.random.default_rng(16)
    worst = 0.0
    with torch.no_grad():
        for _ in range(16):
            vu = torch.tensor(rng.normal(size=u_init.shape), device=dev)
            ve = float(rng.normal())
            h = 1e-6
            fd = (float(loss(u_init + h * vu, torch.tensor(eta0 + h * ve, dtype=torch.float64)))
                  - float(loss(u_init - h * vu, torch.tensor(eta0 - h * ve, dtype=torch.float64)))) / (2 * h)
            got = float((gu * vu).sum()) + float(ge) * ve
            worst = max(worst, abs(got - fd) / max(abs(fd), 1e-300))
    ctx.close()
    return {"fwd_adjoint": whole_job_rate(n**3 * nsteps, world, 1e3 * el),
            "fwd_adjoint_config": {"cells": n**3, "steps": nsteps, "checkpoint_every": 5, "eta": eta0,
                                   "seconds_fwd_plus_bwd": el, "dL_deta": float(ge),
                                   "fd_16_directions_max_rel_err": worst}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=256, help="box edge of the timed workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--q26-only", action="store_true", help="skip the FS18 / B25a comparison runs")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-patches form")
    ap.add_argument("--npatch", type=int, default=1024)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the forward + adjoint form")
    ap.add_argument("--adj-n", type=int, default=64)
    ap.add_argument("--adj-reps", type=int, default=8, help="calls of the adjoint-step form")
    ap.add_argument("--no-alfven", action="store_true", help="skip the oblique Alfven-wave throughput runs")
    ap.add_argument("--alfven-n", type=int, default=128)
    ap.add_argument("--alfven-steps", type=int, default=100)
    ap.add_argument("--no-c1", action="store_true", help="skip the 32^3 fast-eigenmode form")
    ap.add_argument("--no-c3", action="store_true", help="skip the 512x512x4 reconnection form")
    ap.add_argument("--only", default=None,
                    help="comma-separated forms to run besides the headline step (emf, batch, alfven, adjoint, "
                         "adjoint_step, c1, c3, e2e, cpu); the rest are skipped (adjoint_step runs only when named)")
    args = ap.parse_args()
    args.adjoint_step = False
    if args.only is not None:
        keep = set(x.strip() for x in args.only.split(",") if x.strip())
        args.q26_only = "emf" not in keep
        args.no_batch = "batch" not in keep
        args.no_alfven = "alfven" not in keep
        args.no_adjoint = "adjoint" not in keep
        args.no_c1 = "c1" not in keep
        args.no_c3 = "c3" not in keep
        args.no_cpu_baseline = "cpu" not in keep
        args.adjoint_step = "adjoint_step" in keep
        if "e2e" not in keep:
            args.e2e_steps = 0
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_2609_10816_gb300 import build, mhd

    build.build()
    n = args.n
    cons, b, info = workload(n)
    N = n**3
    # one stream of its own for the library and torch's work on the state (on the legacy default
    # stream, the end-to-end leg's copies overlapped the steps less)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = mhd.Context((n, n, n), info["h"], stream=stream)
    st = mhd.to_device(cons, b, dev)
    sch = mhd.scheme("ppm", "hlld", "q26")

    def one_step():
        ctx.step_cfl(st, 0.3, sch)

    for _ in range(max(3, args.warmup)):
        one_step()
    torch.cuda.synchronize(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # the FP64 pipe's measured rate on this GPU (DFMA, DADD, DMUL), the roofline's denominator
    fp64_probe = {k: mhd.fp64_rate(k, 1 << 14, stream) for k in ("dfma", "dadd", "dmul")}
    # what a binary64 multiply on the integer pipe adds (not used by the step's kernels)
    fp64_probe.update({k: mhd.fp64_rate(k, 1 << 13, stream) for k in ("int_mul", "dfma_int_mul",
                                                                      "dfma_int_mul_2x128")})
    # DFMA on 16 and 8 lanes of each warp: what FP64 work in a divergent branch costs
    fp64_probe.update({k: mhd.fp64_rate(k, 1 << 13, stream) for k in ("dfma_16_lanes", "dfma_8_lanes")})
    fp64_peak_tflops = 2.0 * fp64_probe["dfma"] / 1e12

    # ---- device-resident timed region ------------------------------------------------------
    ctx.profile(True)
    ctx.profile_read(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            one_step()
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    s1, s2 = ctx.stats()
    md, mb = ctx.divb(st)
    t_max = max_over_ranks(ms, dist, dev)
    value = whole_job_rate(N * args.steps, world, t_max)

    # dominant kernel and its live roofline
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_launches = prof[dom]
    per_launch_s = dom_ms / 1e3 / dom_launches if dom_launches else float("nan")
    key = "turbulence"
    # one face launch covers the x, y and z sweeps of a stage: 3 N faces
    faces_per_launch = 3 * N
    if dom == "face":
        flops_per_launch = FLOPS_PER_FACE[key] * faces_per_launch
    else:
        flops_per_launch = float("nan")

    achieved = flops_per_launch / per_launch_s / 1e12
    tr = TRAFFIC.get(dom)
    traffic = tr["bytes_per_launch"] * (N / tr["cells"]) if tr and tr.get("src") == kernel_src_hash() else None
    launches_timed = sum(v[1] for v in prof.values())

    # ---- the comparison EMF compute schemes on the same workload (Sec. 3.6) -----------------
    forms = {"plain_q26": value}
    if not args.q26_only:
        for emf in ("fs18", "b25a"):
            sch_e = mhd.scheme("ppm", "hlld", emf)
            st_e = mhd.to_device(cons, b, dev)
            for _ in range(2):
                ctx.step_cfl(st_e, 0.3, sch_e)
            barrier()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(args.steps):
                ctx.step_cfl(st_e, 0.3, sch_e)
            g1.record(stream)
            barrier()
            ms_e = max_over_ranks(g0.elapsed_time(g1), dist, dev)
            forms[f"plain_{emf}"] = whole_job_rate(N * args.steps, world, ms_e)
            del st_e

    # ---- batched form: 1024 uneven periodic patches, one persistent launch per stage ---------
    if not args.no_batch:
        forms.update(run_batched(args, dev, stream, barrier, dist, world, same_state=(cons, b, info["h"][0])))

    if not args.no_alfven:
        forms.update(run_alfven(args, dev, stream, barrier, dist, world))

    if args.adjoint_step:
        forms.update(run_adjoint_step(args, dev, stream, barrier, dist, world))

    if not args.no_adjoint:
        forms.update(run_fwd_adjoint(args, dev, stream, barrier, dist, world))

    if not args.no_c1:
        forms.update(run_c1(args, dev, stream, barrier, dist, world))

    if not args.no_c3:
        forms.update(run_c3(args, dev, stream, barrier, dist, world))

    # ---- end to end through the C ABI with host buffers --------------------------------------
    # Every step copies its input state from pinned host memory and its result back. Two device
    # states and two copy streams pipeline it: the upload of step k+1 and the download of step
    # k-1 run while step k computes (the C2C link is full duplex).
    cons_h = torch.from_numpy(cons).pin_memory()
    b_h = torch.from_numpy(b).pin_memory()
    outs = [(torch.empty_like(cons_h).pin_memory(), torch.empty_like(b_h).pin_memory()) for _ in range(2)]
    sts = [st, mhd.to_device(cons, b, dev)]
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def e2e_run():
        barrier()
        f0.record(stream)
        up.wait_event(f0)
        for k in range(args.e2e_steps):
            i = k % 2
            s_k = sts[i]
            if k >= 2:
                up.wait_event(ev_out[i])  # buffer i's previous result has been read back
            with torch.cuda.stream(up):
                s_k.cons.copy_(cons_h, non_blocking=True)
                s_k.b.copy_(b_h, non_blocking=True)
            ev_in[i].record(up)
            stream.wait_event(ev_in[i])
            ctx.step_cfl(s_k, 0.3, sch)
            ev_done[i].record(stream)
            down.wait_event(ev_done[i])
            with torch.cuda.stream(down):
                outs[i][0].copy_(s_k.cons, non_blocking=True)
                outs[i][1].copy_(s_k.b, non_blocking=True)
            ev_out[i].record(down)
        for i in range(min(2, args.e2e_steps)):
            stream.wait_event(ev_out[i])
        f1.record(stream)
        barrier()
        return max_over_ranks(f0.elapsed_time(f1), dist, dev)

    # the copies share the host's memory with other jobs on the machine: the pipeline is timed
    # three times and the median reported (all three beside it)
    e2e_runs = sorted(e2e_run() for _ in range(3)) if args.e2e_steps > 0 else []
    e2e_ms = e2e_runs[1] if e2e_runs else float("nan")
    e2e_value = whole_job_rate(N * args.e2e_steps, world, e2e_ms) if args.e2e_steps > 0 else None
    del sts[1]

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    clocks = clk.summary()
    clk_mhz = clocks.get("sm_mhz")
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(3, args.warmup),
        "ms_per_step": t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD_NAME.format(n=n),
            "cells_per_gpu": N,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (state 64 B/cell = %.2f GB per GPU)" % (64 * N / 1e9),
        },
        "roofline": {
            "kernel": dom,
            "bound": "alu",
            "achieved": achieved,
            "peak": fp64_peak_tflops,
            "unit": "TFLOP/s",
            "frac": achieved / fp64_peak_tflops,
            "traffic": traffic,
            "peak_source": "FP64 measured on this GPU in this run: 2 flops x the DFMA rate of mhd_fp64_rate "
                           "(independent chains on every SM)",
            "frac_of_nominal": achieved / FP64_PEAK_TFLOPS,
            "nominal_peak": FP64_PEAK_TFLOPS,
            "nominal_source": "152 SMs x 2 DFMA/clk x 2 flops x 2070 MHz (recipe SM count and maximum clock)",
            "algorithmic_flops_per_launch": flops_per_launch,
            "flops_per_unit": f"{FLOPS_PER_FACE[key]} per face (HLLD one-sided; {FLOPS_PER_FACE['turbulence_full_hlld']} "
                              f"with both sides' star states), x {faces_per_launch} faces per launch (the x, y "
                              f"and z sweeps of one stage)",
            "frac_full_hlld_count": (FLOPS_PER_FACE["turbulence_full_hlld"] * faces_per_launch / per_launch_s / 1e12
                                     / fp64_peak_tflops) if dom == "face" else None,
            "avg_launch_ms": per_launch_s * 1e3,
        },
        "fp64_probe": {
            "ops_per_s": fp64_probe,
            "per_sm_per_clock": {k: v / 152 / ((clk_mhz or 2070.0) * 1e6) for k, v in fp64_probe.items()},
            "how": "mhd_fp64_rate: 8 independent chains per thread, 8 x 256 threads per SM, CUDA events; "
                   "int_mul: chains of the integer-pipe binary64 multiply; dfma_int_mul: 4 DFMA + 4 of those "
                   "chains (operations of both counted); _2x128: at 2 blocks of 128 threads per SM",
        },
        "hbm_roofline": {
            "algorithmic_bytes_per_cell_update": ALG_BYTES_PER_CELL_UPDATE,
            "achieved_GBps": value / world * ALG_BYTES_PER_CELL_UPDATE / 1e9,
            "peak_GBps": HBM_PEAK_GBS,
            "frac": value / world * ALG_BYTES_PER_CELL_UPDATE / 1e9 / HBM_PEAK_GBS,
        },
        "fp64_whole_step": {
            "algorithmic_flops_per_cell_update": FLOPS_PER_CELL_UPDATE[key],
            "achieved_TFLOPs": value / world * FLOPS_PER_CELL_UPDATE[key] / 1e12,
            "frac": value / world * FLOPS_PER_CELL_UPDATE[key] / 1e12 / fp64_peak_tflops,
            "frac_of_nominal": value / world * FLOPS_PER_CELL_UPDATE[key] / 1e12 / FP64_PEAK_TFLOPS,
        },
        "kernels_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]},
        "e2e": {
            "value": e2e_value,
            "unit": UNIT,
            "h2d_bytes_per_step": int(cons_h.numel() * 8 + b_h.numel() * 8),
            "d2h_bytes_per_step": int(outs[0][0].numel() * 8 + outs[0][1].numel() * 8),
            "steps": args.e2e_steps,
            "runs_ms": e2e_runs,
            "timing": "median of 3 timed runs of the pipeline",
            "pipeline": "2 device states; upload of step k+1 and download of step k-1 overlap step k",
        },
        "gpu_launches": launches_timed,
        "clocks": clocks,
        "checks": {"fofc_flagged_last_step": [s1, s2], "max_divb_dx_over_b": md * info["h"][0] / mb},
        "forms": forms,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
