#!/usr/bin/env python
"""Throughput of the GB300 QED step: particle-steps/s and QED events/s.

Default workload: the rotating-field cascade (1e5 electrons at rest in a
0.1-wavelength ball, E = a0 (cos t, sin t, 0) with a0 = 1000, dt = T/100,
3 periods = 300 steps, Compton + Breit-Wheeler, leveling cap 5e7 per
species).  One bench "step" is one PIC step of the whole ensemble through the
library (push with sub-stepping, avalanche passes, dead-photon removal,
leveling).

Timed window (cascades with a cap): the last W + K steps of the run, where
the photons are leveled at their cap every step.  The steps before the window
run untimed, then W warm-up steps, then K timed steps.  Each timed step is
enqueued with qed_push_async (one CUDA graph launch; the host never waits
inside the loop) between an L2 flush and CUDA events on the library's
stream; qed_push_wait after the loop reads the counts back.  A second pass
over the same window through the host-driven launches (cfg.profile) times
each kernel for the breakdown and the roofline of the dominant kernel.
Extra keys: the same K steps at the start of the cascade (early_window), the
whole run, the FP64 mode, the network sampler, the optical-depth method, the
end-to-end path through pinned host buffers, and the FP64 oracle timed on
the host cores.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload and window on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2409_17299_gb300 import workloads as W  # noqa: E402  (no CUDA, no method arithmetic)

# algorithmic bytes per particle-step of the lepton pass (read x,y,z,px,py,pz,w + id;
# write x,y,z,px,py,pz) and per emission (nevents update + photon record + birth clock)
LEPTON_BYTES = {"fp32": 7 * 4 + 8 + 6 * 4, "fp64": 7 * 8 + 8 + 6 * 8}
EMIT_BYTES = {"fp32": 8 + 7 * 4 + 8 + 4 + 8, "fp64": 8 + 7 * 8 + 8 + 4 + 8}
# photon step: read w, x, k, id; write x.  Pair: photon weight cleared, two
# lepton records (x, p, w, id, nevents, birth clock)
PHOTON_BYTES = {"fp32": 4 + 3 * 4 + 3 * 4 + 8 + 3 * 4, "fp64": 8 + 3 * 8 + 3 * 8 + 8 + 3 * 8}
PAIR_BYTES = {"fp32": 4 + 2 * (7 * 4 + 8 + 4 + 8), "fp64": 8 + 2 * (7 * 8 + 8 + 4 + 8)}
# optical-depth scheme, per particle-step: the same records plus the optical
# depth (working precision) read and written
OD_LEPTON_BYTES = {"fp32": LEPTON_BYTES["fp32"] + 8, "fp64": LEPTON_BYTES["fp64"] + 16}
OD_PHOTON_BYTES = {"fp32": PHOTON_BYTES["fp32"] + 8, "fp64": PHOTON_BYTES["fp64"] + 16}
# DRAM bytes (read + write) per particle-step of the step-start passes, from
# one ncu capture of the current kernels at the first step of the timed
# window of the default workload (dram__bytes_read.sum + dram__bytes_write.sum
# over the particles at the step start; the lepton figure includes the
# photon records of its 0.3 emissions per lepton-step):
# profiles/k_photon_pass_fp32_rotating_e_cascade.md and
# profiles/k_lepton_pass_fp32_rotating_e_cascade.md.  None when the kernel
# changed since its capture.
NCU_PHOTON_BYTES_PER_STEP = {"fp32": 47.6, "fp64": None}
NCU_LEPTON_BYTES_PER_STEP = {"fp32": 80.1, "fp64": None}
# FP64 FLOPs (2 DFMA + DADD + DMUL thread instructions) per particle-step of
# the FP64 step-start passes at the rotating-E cascade's cap (0.3 emissions
# per lepton-step): the launch's count over the particles it pushed, from one
# ncu capture of the current kernels (profiles/fp64_passes_rotating_e_cascade.md)
NCU_FP64_FLOP_PER_STEP = {"k_lepton_pass": 481.7, "k_photon_pass": 206.0}
# algorithmic FLOPs per training sample of the 2-64-64-64-1 network: forward
# 2 x (2*64 + 64*64 + 64*64 + 64) multiply-adds, backward the two 64x64 input
# gradients, the two 64x64 weight gradients, W1's and W4's gradients
MLP_TRAIN_FLOP_PER_SAMPLE = 2 * (2 * 64 + 64 * 64 + 64 * 64 + 64) + 2 * (4 * 64 * 64 + 2 * 64 + 64)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="rotating_e_cascade",
                    choices=["rotating_e_cascade", "uniform_b_emission", "standing_wave_cascade", "standing_wave_grid",
                             "batched_uniform_b"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--compare-fp64", type=int, default=1, help="also time the FP64 mode (extra key)")
    ap.add_argument("--compare-mlp", type=int, default=1,
                    help="also train the surrogate sampler (1e8 table draws) and time the cascade with it")
    ap.add_argument("--mlp-samples", type=float, default=1e8)
    ap.add_argument("--mlp-batch", type=int, default=8192,
                    help="--train-only: samples per optimizer step (a multiple of 128)")
    ap.add_argument("--train-only", action="store_true",
                    help="only train the surrogate on --mlp-samples draws and print the training line")
    ap.add_argument("--compare-od", type=int, default=1,
                    help="also time the accumulated optical-depth scheme on the same workload (extra key)")
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--growth", type=int, default=1,
                    help="also run the paper's test problem (Sec. 5.1, 5 seeds x FP64, FP32, network sampler) "
                         "and report the growth rate and density profile (extra key)")
    ap.add_argument("--e2e", type=int, default=1)
    ap.add_argument("--scale", type=float, default=1.0, help="scale the seed count (tests only)")
    ap.add_argument("--batch-threads", type=int, default=0, choices=[0, 128, 256, 512],
                    help="batched workload: fixed block shape instead of the autotuner's (0)")
    ap.add_argument("--ncu-window", action="store_true",
                    help="profiling run for ncu --profile-from-start off: only the host-driven pass over the timed "
                         "window, its K steps inside cudaProfilerStart/Stop; prints the window's statistics")
    ap.add_argument("--profile-step", type=int, default=None,
                    help="profiling run for ncu --profile-from-start off: drive the workload (--scale) to this "
                         "step, then one host-driven step inside cudaProfilerStart/Stop")
    ap.add_argument("--profile-sampler", default="table", choices=["table", "mlp"],
                    help="--profile-step: emission sampler (mlp: a network trained on --mlp-samples draws first)")
    ap.add_argument("--profile-method", default="waiting-time", choices=["waiting-time", "optical-depth"],
                    help="--profile-step: event method")
    return ap.parse_args()


def make_workload(name, scale=1.0, rank=0):
    if name == "rotating_e_cascade":
        w = W.rotating_e_cascade(n=int(100000 * scale), seed=1 + 1000 * rank,
                                 thin_cap=int(50_000_000 * scale))
    elif name == "standing_wave_cascade":
        w = W.standing_wave_cascade(n=int(1_000_000 * scale), seed=4 + 1000 * rank,
                                    thin_cap=int(200_000_000 * scale))
    elif name == "standing_wave_grid":
        w = W.standing_wave_grid(n=int(1_000_000 * scale), seed=4 + 1000 * rank,
                                 thin_cap=int(200_000_000 * scale))
    elif name == "batched_uniform_b":
        w = W.batched_uniform_b(seed=2 + 1000 * rank, size_scale=scale)
    else:
        w = W.uniform_b_emission(n=int(16384 * scale), seed=1000 * rank)
    return w


def default_steps(w):
    if isinstance(w, list):
        return 3, w[0].nsteps
    if w.thin_cap:
        return 5, 20
    return 3, w.nsteps - 3


def window_start(w, warm, steps):
    """First step of the warm-up: cascades with a cap end their window at the
    last step of the run (leveled at the cap); otherwise the run's start."""
    if isinstance(w, list) or not w.thin_cap:
        return 0
    return max(0, w.nsteps - warm - steps)


def capacities(w, nsteps=None):
    """Buffer sizes for a run of nsteps steps (cascades: bounded by the cap)."""
    nsteps = w.nsteps if nsteps is None else nsteps
    n0 = sum(len(s["id"]) for s in w.species)
    if w.thin_cap:
        # each species is leveled at the cap after a step: room for the cap
        # plus one step's growth (photons grow fastest)
        return [int(1.3 * w.thin_cap) + 4 * n0, int(1.3 * w.thin_cap) + 4 * n0, int(1.6 * w.thin_cap) + 4 * n0]
    return [n0, 16, int(n0 * (1 + 0.15 * nsteps)) + 1024]


# ---------------------------------------------------------------------------
# CPU oracle legs (spawned processes; never touch CUDA)
# ---------------------------------------------------------------------------
def _oracle_shard(args):
    name, scale_seed, lo, hi, warm, steps = args     # warm: steps run untimed first
    sys.path.insert(0, ROOT)
    import oracle
    w = make_workload(name, 1.0)
    if isinstance(w, list):                       # batched: shard k samples ensemble k
        w = w[scale_seed % len(w)]
        hi = lo + min(hi - lo, len(w.species[0]["id"]))
        lo, hi = 0, hi - lo
    total = len(w.species[0]["id"])
    frac = (hi - lo) / total
    ws = W.subset(w, 0, slice(lo, hi))
    tabs = oracle.build_tables()
    cap = [max(1024, int(c * frac * 1.2)) for c in capacities(w)]
    ens = oracle.Ensemble.from_arrays(ws.species, cap)
    cfg = oracle.make_cfg(seed=w.seed, push_photons=w.push_photons, thin_cap=int(w.thin_cap * frac),
                          field_kind=w.field_kind, field_prm=w.field_prm)
    if w.field_kind == W.FIELD_GRID:              # the caller refills the grid every step
        def run(s0, k):
            tot = {"particle_steps": 0, "emit_events": 0, "pair_events": 0}
            for s in range(s0, s0 + k):
                oracle.set_field_grid(W.grid_values(w.notes["a0"], s * w.dt))
                st1 = oracle.push_and_generate(ens, tabs, cfg, w.dt, 1, s)
                for key in tot:
                    tot[key] += st1[key]
            return tot
    else:
        def run(s0, k):
            return oracle.push_and_generate(ens, tabs, cfg, w.dt, k, s0)
    if warm:
        run(0, warm)
    t0 = time.perf_counter()
    st = run(warm, steps)
    dt = time.perf_counter() - t0
    return st["particle_steps"], st["emit_events"] + st["pair_events"], dt


def oracle_run(name, warm, steps, target_s=15.0, procs=None):
    """Time the oracle on disjoint seed subsets of the workload, one process
    per host core: steps 0..warm-1 untimed (a cascade's cap scaled to the
    subset), then steps warm..warm+steps-1 timed.  Returns particle-steps/s,
    events/s, cores, sample text."""
    import multiprocessing as mp
    procs = procs or min(16, os.cpu_count() or 1)
    w = make_workload(name, 1.0)
    total = sum(len(x.species[0]["id"]) for x in w) if isinstance(w, list) else len(w.species[0]["id"])
    # seeds per shard sized from a nominal oracle rate of ~3e6 particle-steps/s
    if name == "rotating_e_cascade":
        per = 250
    elif name in ("standing_wave_cascade", "standing_wave_grid"):
        per = 60
    elif name == "batched_uniform_b":
        per = 400
    else:
        per = 2000
    per = max(1, min(per, total // procs))
    if isinstance(w, list):
        jobs = [(name, k, 0, per, warm, steps) for k in range(procs)]
    else:
        jobs = [(name, 0, k * per, (k + 1) * per, warm, steps) for k in range(procs)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_shard, jobs)
    wall = time.perf_counter() - t0
    ps = sum(r[0] for r in res)
    ev = sum(r[1] for r in res)
    tmax = max(r[2] for r in res)
    sample = ("%d disjoint subsets of %d seed electrons each (%d of %d) of %s (leveling cap scaled to the "
              "subset), steps 0..%d untimed, %d..%d timed, FP64 oracle, one process per core"
              % (procs, per, procs * per, total, name, warm - 1, warm, warm + steps - 1))
    return ps / tmax, ev / tmax, procs, sample, wall


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, index=0):
        self.p = None
        # raw samples: QED_CLOCKS_CSV if set, else a temporary file (the JSON
        # line carries the summary)
        self.path = os.environ.get("QED_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), "qed_clocks_%d_%d.csv" % (os.getpid(), index))
        self.index = index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except ValueError:
                continue
            for k, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(k)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


class GridFeed:
    """The caller's side of a gridded field: the node values of step s are
    written to a device buffer the library reads (outside the timed pushes)."""

    def __init__(self, w, gen, prec):
        import torch
        import paper_2409_17299_gb300 as q
        self.w = w
        self.dev = None
        if w.field_kind != W.FIELD_GRID:
            return
        nx, ny, nz = (int(v) for v in w.field_prm[:3])
        self.dev = torch.empty((6, nz, ny, nx), device="cuda",
                               dtype=torch.float32 if prec == q.QED_FP32 else torch.float64)
        q.qed_set_field_grid(gen.ctx, self.dev.data_ptr())

    def feed(self, step):
        if self.dev is not None:
            import torch
            self.dev.copy_(torch.from_numpy(W.grid_values(self.w.notes["a0"], step * self.w.dt)))

    def nbytes(self):
        return 0 if self.dev is None else self.dev.numel() * self.dev.element_size()


def size_cascade(w, nsteps, precision, method=0):
    """Buffer capacities that hold every step of the run: one untimed pass
    over the whole cascade, growing a species by 5% beyond the demand
    whenever a step overflows (the step is replayed identically)."""
    import torch
    import paper_2409_17299_gb300 as q
    prec = q.QED_FP32 if precision == "fp32" else q.QED_FP64
    cfg = q.make_config(precision=prec, seed=w.seed, push_photons=w.push_photons, thin_cap=w.thin_cap,
                        restore_on_overflow=1, event_method=method)
    gen = q.Generator(cfg)
    ens = q.DeviceEnsemble.from_host(w.species, capacities(w, nsteps), prec, optical_depth=method != 0)
    field = q.make_field(w.field_kind, w.field_prm)
    grid = GridFeed(w, gen, prec)
    for s in range(nsteps):
        grid.feed(s)
        while True:
            gen._bind(ens)
            P = ens.struct()
            rc, st = q.qed_push_and_generate(gen.ctx, P, field, w.dt, 1, s)
            ens.pull_counts(P)
            if rc == q.QED_OK:
                break
            if rc != q.QED_ERR_CAPACITY:
                raise q.QedError(rc, "qed_push_and_generate", st)
            ens.grow([max(ens.capacity[k], int(1.05 * st["needed_capacity"][k]) + 1024) for k in range(3)])
    caps = list(ens.capacity)
    gen.close()
    del ens
    torch.cuda.empty_cache()
    return caps


def gpu_run(args, w, precision, start, warm, steps, profile=False, mlp_params=None, caps=None, method=0,
            profiler_range=False):
    """Steps 0..start+warm-1 untimed (one batch, one wait), then `steps`
    timed steps: per step an L2 flush, then the step enqueued between two
    CUDA events (qed_push_async; no host wait inside the loop); one
    qed_push_wait after the loop.  Returns the summed device time of the
    timed steps, their statistics, the counts at the window's start and end,
    the GPU time between steps not spent flushing (host-induced idling), and
    the host's waits inside and after the loop."""
    import torch
    import paper_2409_17299_gb300 as q
    prec = q.QED_FP32 if precision == "fp32" else q.QED_FP64
    # capacities are sized for the whole run, so no overflow snapshot
    cfg = q.make_config(precision=prec, seed=w.seed, push_photons=w.push_photons, thin_cap=w.thin_cap,
                        profile=int(profile), restore_on_overflow=0, event_method=method,
                        sampler=q.QED_SAMPLER_MLP if mlp_params is not None else q.QED_SAMPLER_TABLE)
    gen = q.Generator(cfg)
    if mlp_params is not None:
        q.qed_mlp_set_params(gen.ctx, mlp_params)
    s0 = start + warm
    ens = q.DeviceEnsemble.from_host(w.species, caps or capacities(w, s0 + steps), prec,
                                     optical_depth=method != 0)
    field = q.make_field(w.field_kind, w.field_prm)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    grid = GridFeed(w, gen, prec)
    if grid.dev is None:
        if s0:
            gen.push_async(ens, field, w.dt, s0, 0)
            gen.wait(ens)
    else:                                  # the caller refills the grid every step
        for s in range(s0):
            grid.feed(s)
            gen.push(ens, field, w.dt, 1, s, auto_grow=False)
    torch.cuda.synchronize()
    counts0 = list(ens.count)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    if profiler_range:
        torch.cuda.profiler.start()
    t0 = time.perf_counter()
    host_in_loop = 0.0
    for k, s in enumerate(range(s0, s0 + steps)):
        grid.feed(s)
        f, a, b = ev[k]
        f.record(stream)
        flush.fill_(float(s))
        a.record(stream)
        th = time.perf_counter()
        gen.push_async(ens, field, w.dt, 1, s)
        host_in_loop += time.perf_counter() - th
        b.record(stream)
    # qed_push_wait removes the dead entries the steps left in place (moves are
    # deferred while few): timed apart, between an event before the call and
    # one after it (an upper bound: it includes the call's return)
    c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c.record(stream)
    tw = time.perf_counter()
    st = gen.wait(ens)
    drain = time.perf_counter() - tw
    d.record(stream)
    torch.cuda.synchronize()
    if profiler_range:
        torch.cuda.profiler.stop()
    wall = time.perf_counter() - t0
    ms = sum(a.elapsed_time(b) for _, a, b in ev)
    # device time between the end of a step and the next flush: the GPU
    # waiting for the host
    idle = sum(ev[k - 1][2].elapsed_time(ev[k][0]) for k in range(1, steps))
    counts = list(ens.count)
    gen.close()
    del ens, flush
    torch.cuda.empty_cache()
    st["lepton_launches"] = steps + st["passes"]
    st["counts_start"] = counts0
    st["gpu_idle_ms"] = idle
    st["host_enqueue_ms"] = host_in_loop * 1e3
    st["drain_wait_ms"] = drain * 1e3
    st["window"] = [s0, s0 + steps - 1]
    st["final_compaction_ms"] = c.elapsed_time(d)
    return ms, wall, st, counts


def batch_run(ws, precision, warm, steps, threads=0):
    """64 ensembles through qed_batch_push: one persistent launch per call.
    A sizing pass on copies fixes the photon buffers; W warm-up steps run as
    one call, then the K timed steps as one call."""
    import torch
    import paper_2409_17299_gb300 as q
    prec = q.QED_FP32 if precision == "fp32" else q.QED_FP64
    cfg = q.make_config(precision=prec, seed=ws[0].seed, push_photons=0, profile=1, block_threads=threads)
    gen = q.Generator(cfg)
    fields = (q.QedFieldDesc * len(ws))()
    for k, w in enumerate(ws):
        fields[k] = q.make_field(w.field_kind, w.field_prm)

    def fresh(ph_caps):
        ens = [q.DeviceEnsemble.from_host(w.species, [len(w.species[0]["id"]), 1, int(c)], prec)
               for w, c in zip(ws, ph_caps)]
        arr = (q.QedParticles * len(ens))()
        for k, e in enumerate(ens):
            arr[k] = e.struct()
        return ens, arr

    # sizing pass: photon demand of the whole run, ensemble by ensemble
    caps = [len(w.species[0]["id"]) * 2 + 1024 for w in ws]
    while True:
        ens, arr = fresh(caps)
        rc, st = q.qed_batch_push(gen.ctx, arr, fields, ws[0].dt, warm + steps, 0)
        if rc == q.QED_OK:
            need = [int(arr[k].s[2].count) for k in range(len(ws))]
            break
        caps = [c * 4 for c in caps]
        del ens, arr
        torch.cuda.empty_cache()
    del ens, arr
    torch.cuda.empty_cache()
    caps = [int(n * 1.05) + 1024 for n in need]
    tuned = None
    if not threads:                         # else the block shape is fixed by the caller
        ens, arr = fresh(caps)
        tuned = q.qed_autotune_batch(gen.ctx, arr, fields, ws[0].dt, 2)
        tuned = (tuned[0], tuned[1], q.qed_batch_shape(gen.ctx)[1])
        del ens, arr
    ens, arr = fresh(caps)
    if warm:
        q.qed_batch_push(gen.ctx, arr, fields, ws[0].dt, warm, 0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush.fill_(1.0)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    rc, st = q.qed_batch_push(gen.ctx, arr, fields, ws[0].dt, steps, warm)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    counts = [[int(arr[k].s[s].count) for s in range(3)] for k in range(len(ws))]
    gen.close()
    return ms, st, counts, tuned


def e2e_run(w, precision, start, warm, steps, caps=None):
    """Same steps through the C ABI with the ensemble in pinned host memory:
    every step copies it to the device, pushes one step, and copies it back.
    Steps before the window (0..start-1) run on the device untimed, and their
    result is copied to the host buffers first."""
    import numpy as np
    import torch
    import paper_2409_17299_gb300 as q
    prec = q.QED_FP32 if precision == "fp32" else q.QED_FP64
    cfg = q.make_config(precision=prec, seed=w.seed, push_photons=w.push_photons, thin_cap=w.thin_cap,
                        restore_on_overflow=0)
    gen = q.Generator(cfg)
    caps = caps or capacities(w, start + warm + steps)
    dev = q.DeviceEnsemble(caps, prec)
    fd = dev.fdtype
    host = []
    for s in range(3):
        d = {f: torch.zeros(caps[s], dtype=fd).pin_memory() for f in ("x", "y", "z", "px", "py", "pz", "w")}
        d["id"] = torch.zeros(caps[s], dtype=torch.int64).pin_memory()
        d["nevents"] = torch.zeros(caps[s], dtype=torch.int32).pin_memory()
        sp = w.species[s]
        n = len(sp["id"])
        for f in ("x", "y", "z", "px", "py", "pz", "w"):
            d[f][:n].copy_(torch.from_numpy(np.asarray(sp[f], dtype=np.float64)).to(fd))
        d["id"][:n].copy_(torch.from_numpy(np.asarray(sp["id"], dtype=np.uint64).view(np.int64)))
        host.append(d)
    count = [len(sp["id"]) for sp in w.species]
    field = q.make_field(w.field_kind, w.field_prm)
    stream = torch.cuda.current_stream()
    grid = GridFeed(w, gen, prec)

    def one_step(s, nb):
        grid.feed(s)                              # the step's field is an input too
        nb[0] += grid.nbytes()
        for k in range(3):
            n = count[k]
            for f in host[k]:
                dev.arr[k][f][:n].copy_(host[k][f][:n], non_blocking=True)
                nb[0] += n * host[k][f].element_size()
        dev.count = list(count)
        gen.push(dev, field, w.dt, 1, s, auto_grow=False)
        for k in range(3):
            n = dev.count[k]
            for f in host[k]:
                host[k][f][:n].copy_(dev.arr[k][f][:n], non_blocking=True)
                nb[1] += n * host[k][f].element_size()
            count[k] = n
        stream.synchronize()

    if start:
        for k in range(3):
            n = count[k]
            for f in host[k]:
                dev.arr[k][f][:n].copy_(host[k][f][:n])
        dev.count = list(count)
        gen.push_async(dev, field, w.dt, start, 0) if grid.dev is None else None
        if grid.dev is None:
            gen.wait(dev)
        else:
            for s in range(start):
                grid.feed(s)
                gen.push(dev, field, w.dt, 1, s, auto_grow=False)
        for k in range(3):
            n = dev.count[k]
            for f in host[k]:
                host[k][f][:n].copy_(dev.arr[k][f][:n])
            count[k] = n
    nbw = [0, 0]
    for s in range(start, start + warm):
        one_step(s, nbw)
    torch.cuda.synchronize()
    nb = [0, 0]
    ps = 0
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    t0 = time.perf_counter()
    for s in range(start + warm, start + warm + steps):
        before = q.qed_get_stats(gen.ctx)["particle_steps"]
        one_step(s, nb)
        ps += q.qed_get_stats(gen.ctx)["particle_steps"] - before
    b.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    gen.close()
    return ps, a.elapsed_time(b), wall, nb


def reduce_over_ranks(particle_steps, events, secs, world):
    """Whole-job totals: work summed over the ranks, time the slowest rank's
    (each rank runs its own replica; no data-path exchange)."""
    if world <= 1:
        return particle_steps, events, secs
    import torch
    import torch.distributed as dist
    s = torch.tensor([particle_steps, events], dtype=torch.float64)
    t = torch.tensor([secs], dtype=torch.float64)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(s[0]), float(s[1]), float(t[0])


def main():
    args = parse()
    if args.ncu_window or args.profile_step is not None or args.train_only:
        args.cpu_baseline = 0                     # a profiling run times nothing on the host
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    w0 = make_workload(args.workload, args.scale)
    dw, ds = default_steps(w0)
    warm = args.warmup if args.warmup is not None else dw
    steps = args.steps if args.steps is not None else ds
    start = window_start(w0, warm, steps)

    if args.impl == "reference":
        if rank != 0:
            return
        ps_rate, ev_rate, cores, sample, wall = oracle_run(args.workload, start + warm, steps)
        line = {"impl": "reference", "metric": "particle-steps/s", "value": ps_rate, "unit": "particle-steps/s",
                "n_gpus": args.gpus, "steps": steps, "warmup": warm, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "precision": "fp64", "l2": "n/a (CPU)",
                           "window": [start + warm, start + warm + steps - 1]},
                "events_per_s": ev_rate,
                "cpu_baseline": {"value": ps_rate, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": ps_rate, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    # CPU baseline first: its process pool is spawned before CUDA is initialised
    cpu = None
    if args.cpu_baseline and rank == 0 and world == 1:
        cpu = oracle_run(args.workload, start + warm, steps)

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("gloo")
    from paper_2409_17299_gb300 import build
    build.build()
    import paper_2409_17299_gb300 as q  # noqa: F401

    w = make_workload(args.workload, args.scale, rank)
    if args.workload == "batched_uniform_b":
        return batched_main(args, w, warm, steps, rank, world, cpu)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0

    n_total = start + warm + steps
    if args.train_only:
        _, train = train_surrogate_timed(int(args.mlp_samples), peaks, args.mlp_batch)
        print(json.dumps(train), flush=True)
        return
    if args.profile_step is not None:
        mlp_params = None
        if args.profile_sampler == "mlp":
            mlp_params, _ = train_surrogate_timed(int(args.mlp_samples), peaks)
        return profile_step(w, args.precision, args.profile_step, mlp_params,
                            1 if args.profile_method == "optical-depth" else 0)
    caps = size_cascade(w, n_total, args.precision) if w.push_photons else None
    if args.ncu_window:
        _, _, t, _ = gpu_run(args, w, args.precision, start, warm, steps, caps=caps, profile=True,
                             profiler_range=True)
        print(json.dumps({"ncu_window": t["window"], "particle_steps": t["particle_steps"],
                          "lepton_steps": t["lepton_steps"], "photon_steps": t["photon_steps"],
                          "emit_events": t["emit_events"], "pair_events": t["pair_events"],
                          "counts_at_start": t["counts_start"], "kernel_ms": t["kernel_ms"],
                          "thinned": t["thinned"], "moved": t["moved"]}), flush=True)
        return
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # the headline without per-kernel events; then the same steps again with
    # the library's per-kernel CUDA events for the breakdown and the roofline
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms, wall, tot_plain, counts = gpu_run(args, w, args.precision, start, warm, steps, caps=caps)
    torch.cuda.synchronize()
    ms_prof, _, tot, _ = gpu_run(args, w, args.precision, start, warm, steps, caps=caps, profile=True)
    # the same work, instrumented (FP32 leveling sums depend on the array
    # order, so a rare keep/drop decision may differ between the two passes)
    assert abs(tot["particle_steps"] / tot_plain["particle_steps"] - 1) < 1e-3
    torch.cuda.synchronize()
    secs = ms / 1e3
    ps_total, ev_total, tmax = reduce_over_ranks(float(tot_plain["particle_steps"]),
                                                 float(tot_plain["emit_events"] + tot_plain["pair_events"]), secs,
                                                 world)

    def host_side(t, dev_ms):
        # waits inside the timed loop: the library's stream waits minus the
        # one wait after the loop (the graph path issues no other)
        inside = max(0.0, t["sync_ms"] - t["drain_wait_ms"])
        return {"host_sync_wait_in_loop_ms": inside, "drain_wait_after_loop_ms": t["drain_wait_ms"],
                "final_compaction_ms": t["final_compaction_ms"],
                "host_enqueue_ms": t["host_enqueue_ms"], "gpu_idle_between_steps_ms": t["gpu_idle_ms"],
                "device_ms": dev_ms, "host_sync_wait_frac_of_device": inside / dev_ms if dev_ms > 0 else None}

    other_windows = {}
    if start > 0 and world == 1:
        # the same K steps at the start of the cascade (about 1e5 leptons), and
        # the whole run step by step
        ms_e, _, tot_e, _ = gpu_run(args, w, args.precision, 0, warm, steps, caps=caps)
        other_windows["early_window"] = {
            "value": tot_e["particle_steps"] / (ms_e / 1e3), "ms_per_step": ms_e / steps,
            "steps": tot_e["window"], "counts_at_start": tot_e["counts_start"],
            "events_per_s": (tot_e["emit_events"] + tot_e["pair_events"]) / (ms_e / 1e3),
            "host": host_side(tot_e, ms_e)}
        ms_w, _, tot_w, _ = gpu_run(args, w, args.precision, 0, 0, n_total, caps=caps)
        other_windows["whole_run"] = {
            "value": tot_w["particle_steps"] / (ms_w / 1e3), "ms_per_step": ms_w / n_total,
            "steps": tot_w["window"], "events_per_s": (tot_w["emit_events"] + tot_w["pair_events"]) / (ms_w / 1e3),
            "host": host_side(tot_w, ms_w)}

    fp64 = None
    if args.compare_fp64 and args.precision == "fp32" and world == 1:
        ms64, wall64, tot64, _ = gpu_run(args, w, "fp64", start, warm, steps, caps=caps)
        _, _, tot64p, _ = gpu_run(args, w, "fp64", start, warm, steps, caps=caps, profile=True)
        fp64 = {"value": tot64["particle_steps"] / (ms64 / 1e3), "events_per_s":
                (tot64["emit_events"] + tot64["pair_events"]) / (ms64 / 1e3), "ms_per_step": ms64 / steps,
                "roofline": fp64_roofline(tot64p, hbm_peak)}

    mlp = None
    if args.compare_mlp and world == 1 and args.workload == "rotating_e_cascade":
        import paper_2409_17299_gb300 as q
        P, train = train_surrogate_timed(int(args.mlp_samples), peaks)
        ms_m, _, tot_m, _ = gpu_run(args, w, args.precision, start, warm, steps, mlp_params=P, caps=caps)
        mlp = {"value": tot_m["particle_steps"] / (ms_m / 1e3),
               "events_per_s": (tot_m["emit_events"] + tot_m["pair_events"]) / (ms_m / 1e3),
               "ms_per_step": ms_m / steps, **train}
        # the pass kernels' HBM fractions with the network sampler (a second,
        # instrumented pass over the same steps)
        _, _, tot_mp, _ = gpu_run(args, w, args.precision, start, warm, steps, mlp_params=P, caps=caps,
                                  profile=True)
        pr = args.precision
        lb = LEPTON_BYTES[pr] * tot_mp["lepton_steps"] + EMIT_BYTES[pr] * tot_mp["emit_events"]
        pb = PHOTON_BYTES[pr] * tot_mp["photon_steps"] + PAIR_BYTES[pr] * tot_mp["pair_events"]
        lk, pk = tot_mp["kernel_ms"][0], tot_mp["kernel_ms"][1]
        mlp["roofline"] = {
            "k_lepton_pass (network sampler)": {"kernel_ms": lk, "achieved_gbs": lb / (lk / 1e3) / 1e9 if lk > 0 else None,
                                                "frac": lb / (lk / 1e3) / 1e9 / hbm_peak if lk > 0 else None},
            "k_photon_pass": {"kernel_ms": pk, "achieved_gbs": pb / (pk / 1e3) / 1e9 if pk > 0 else None,
                              "frac": pb / (pk / 1e3) / 1e9 / hbm_peak if pk > 0 else None},
            "peak": hbm_peak, "unit": "GB/s", "peak_source": peak_src + " hbm_gbs"}
        # the same training at larger batches: more tiles per Adam step
        # amortise the step's barriers, but fewer steps leave a higher loss
        runs = []
        for b in (19456, 38912, 77824):
            _, tb = train_surrogate_timed(int(args.mlp_samples), peaks, b)
            runs.append({"batch": b, "seconds": tb["train_seconds"], "final_mse": tb["train_final_mse"],
                         "achieved_tflops": tb["train_roofline"]["achieved"], "frac": tb["train_roofline"]["frac"]})
        mlp["train_batch_sweep"] = {
            "note": "same samples and learning rate as the headline training (batch 8192, the setting the "
                    "tests validate); a larger batch means fewer Adam steps and a higher final loss",
            "runs": runs}

    growth = None
    if args.growth and world == 1 and args.workload == "rotating_e_cascade":
        import numpy as np
        modes = {"fp64": [growth_run("fp64", sd) for sd in GROWTH_SEEDS],
                 "fp32": [growth_run("fp32", sd) for sd in GROWTH_SEEDS]}
        if mlp:
            modes["surrogate_fp32"] = [growth_run("fp32", sd, mlp_params=P) for sd in GROWTH_SEEDS]
        growth = {k: growth_summary(v) for k, v in modes.items()}
        ref = growth["fp64"]
        for k, v in growth.items():
            v["eta_gamma_vs_fp64"] = v["gamma_mean"] / ref["gamma_mean"] - 1
            v["profile_l1_vs_fp64"] = float(np.abs(np.array(v["profile_mean"]) - np.array(ref["profile_mean"])).sum())
        # one seed per mode over 20 T (the paper's long runs): Gamma fitted
        # from 3.5 T to 20 T
        s20 = GROWTH_SEEDS[:4]
        t20 = {"fp64": [growth_run("fp64", sd, periods=20, fit=GROWTH_FIT_20T) for sd in s20],
               "fp32": [growth_run("fp32", sd, periods=20, fit=GROWTH_FIT_20T) for sd in s20]}
        if mlp:
            t20["surrogate_fp32"] = [growth_run("fp32", sd, mlp_params=P, periods=20, fit=GROWTH_FIT_20T)
                                     for sd in s20[:2]]
        growth["t20"] = {k: growth_summary(v) for k, v in t20.items()}
        for k, v in growth["t20"].items():
            v["eta_gamma_vs_fp64"] = v["gamma_mean"] / growth["t20"]["fp64"]["gamma_mean"] - 1
            v["profile_l1_vs_fp64"] = float(np.abs(np.array(v["profile_mean"]) -
                                                   np.array(growth["t20"]["fp64"]["profile_mean"])).sum())
            v["seeds"] = list(s20[:len(t20[k])])
        growth["setup"] = ("paper test problem: 2.5e5 e-/e+ at rest filling the 1-wavelength box, standing CP wave "
                           "a0 = 1557, dt = T/200, 5 T, leveling cap %d per species; Gamma fitted over steps %d-%d "
                           "from the leptons' total weight; density profile of lepton weight along x, %d bins; "
                           "seeds %s" % (GROWTH_CAP, GROWTH_FIT[0], GROWTH_FIT[1], GROWTH_BINS, list(GROWTH_SEEDS)))

    od = None
    if args.compare_od and world == 1 and args.workload != "batched_uniform_b":
        import paper_2409_17299_gb300 as q
        M = q.QED_METHOD_OPTICAL_DEPTH
        caps_od = size_cascade(w, n_total, args.precision, M) if w.push_photons else None
        ms_o, _, tot_op, counts_o = gpu_run(args, w, args.precision, start, warm, steps, caps=caps_od, method=M)
        _, _, tot_o, _ = gpu_run(args, w, args.precision, start, warm, steps, caps=caps_od, method=M, profile=True)
        prec = args.precision
        lep_b = OD_LEPTON_BYTES[prec] * tot_o["lepton_steps"] + EMIT_BYTES[prec] * tot_o["emit_events"]
        ph_b = OD_PHOTON_BYTES[prec] * tot_o["photon_steps"] + PAIR_BYTES[prec] * tot_o["pair_events"]
        lk, pk = tot_o["kernel_ms"][0], tot_o["kernel_ms"][1]
        od = {"value": tot_op["particle_steps"] / (ms_o / 1e3),
              "events_per_s": (tot_op["emit_events"] + tot_op["pair_events"]) / (ms_o / 1e3),
              "ms_per_step": ms_o / steps, "final_counts": counts_o,
              "kernels": {"k_lepton_od": {"kernel_ms": lk, "bytes_per_particle_step": OD_LEPTON_BYTES[prec],
                                          "achieved_gbs": lep_b / (lk / 1e3) / 1e9 if lk > 0 else None},
                          "k_photon_od": {"kernel_ms": pk, "bytes_per_particle_step": OD_PHOTON_BYTES[prec],
                                          "achieved_gbs": ph_b / (pk / 1e3) / 1e9 if pk > 0 else None}},
              "method": "accumulated optical depth: rate once per step, at most one event per step"}
        for k in od["kernels"].values():
            k["frac"] = k["achieved_gbs"] / hbm_peak if k["achieved_gbs"] else None

    e2e = None
    if args.e2e:
        ps_e, ms_e2, wall_e, nb = e2e_run(w, args.precision, start, warm, steps, caps=caps)
        e2e = {"value": ps_e / (ms_e2 / 1e3) * world, "unit": "particle-steps/s",
               "h2d_bytes_per_step": nb[0] // max(1, steps), "d2h_bytes_per_step": nb[1] // max(1, steps)}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    prec = args.precision
    lep_bytes = LEPTON_BYTES[prec] * tot["lepton_steps"] + EMIT_BYTES[prec] * tot["emit_events"]
    ph_bytes = PHOTON_BYTES[prec] * tot["photon_steps"] + PAIR_BYTES[prec] * tot["pair_events"]
    lep_ms, ph_ms = tot["kernel_ms"][0], tot["kernel_ms"][1]
    launches = max(1, tot["lepton_launches"])
    kernels = {
        "k_lepton_pass": {"achieved": lep_bytes / (lep_ms / 1e3) / 1e9 if lep_ms > 0 else None,
                          "kernel_ms": lep_ms, "launches": launches,
                          "bytes_per_particle_step": LEPTON_BYTES[prec], "bytes_per_emission": EMIT_BYTES[prec],
                          "units": "lepton particle-steps %d, emissions %d" % (tot["lepton_steps"],
                                                                             tot["emit_events"]),
                          "algorithmic_bytes_per_step": lep_bytes / steps,
                          "traffic": (NCU_LEPTON_BYTES_PER_STEP[prec] * tot["lepton_steps"] / steps
                                      if NCU_LEPTON_BYTES_PER_STEP[prec] else None)},
        "k_photon_pass": {"achieved": ph_bytes / (ph_ms / 1e3) / 1e9 if ph_ms > 0 else None,
                          "kernel_ms": ph_ms, "launches": launches if w.push_photons else 0,
                          "bytes_per_photon_step": PHOTON_BYTES[prec], "bytes_per_pair": PAIR_BYTES[prec],
                          "units": "photon-steps %d, pairs %d" % (tot["photon_steps"], tot["pair_events"]),
                          "algorithmic_bytes_per_step": ph_bytes / steps,
                          "traffic": (NCU_PHOTON_BYTES_PER_STEP[prec] * tot["photon_steps"] / steps
                                      if NCU_PHOTON_BYTES_PER_STEP[prec] and w.push_photons else None)},
    }
    for k in kernels.values():
        k["frac"] = k["achieved"] / hbm_peak if k["achieved"] else None
    dom = max(kernels, key=lambda k: kernels[k]["kernel_ms"])
    achieved = kernels[dom]["achieved"]
    line = {
        "metric": "particle-steps/s", "value": ps_total / tmax, "unit": "particle-steps/s",
        "n_gpus": world, "steps": steps, "warmup": warm, "ms_per_step": tmax * 1e3 / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "precision": prec + (" (fp64 sub-step clock, fp64 chi fallback)" if prec == "fp32" else ""),
                   "seed_electrons": len(w.species[0]["id"]), "thin_cap": w.thin_cap,
                   "steps_total": w.nsteps, "dt": "T/%d" % round(2 * math.pi / w.dt),
                   "step_range": tot_plain["window"], "warmup_range": [start, start + warm - 1] if warm else None,
                   "counts_at_window_start": tot_plain["counts_start"],
                   "window": ("the last %d steps of the run: the photons are leveled at the cap every step "
                              "(steps before it run untimed)" % (warm + steps)) if start > 0 else "the run's start",
                   "l2": "flushed between timed steps (256 MB write)",
                   "launch": "one CUDA graph per step (qed_push_async); one wait after the timed steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "events_per_s": ev_total / tmax,
        "final_counts": counts,
        "gpu_launches": tot_plain["launches"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": (achieved / hbm_peak) if achieved else None,
                     "traffic": kernels[dom]["traffic"],
                     "kernel": "%s<%s>" % (dom, "float" if prec == "fp32" else "double"),
                     "peak_source": peak_src + " hbm_gbs",
                     "achieved_is": "algorithmic bytes of all launches / summed CUDA-event time of the launches",
                     "traffic_is": "ncu DRAM bytes per particle-step (step-start launch at the cap) x the "
                                   "kernel's particle-steps per step: bytes per step, all launches",
                     "kernels": kernels},
        "breakdown_ms": {"lepton": tot["kernel_ms"][0], "photon": tot["kernel_ms"][1],
                         "compaction": tot["kernel_ms"][2], "leveling": tot["kernel_ms"][3],
                         "device_total": ms_prof, "device_total_uninstrumented": ms,
                         "note": "kernel times from a second pass over the same steps with per-kernel events "
                                 "(host-driven launches)"},
        "host": host_side(tot_plain, ms),
        "chi_fp64_fallbacks": tot["chi_fp64"],
        "paper_context": ("context only: the paper's QED module takes 2.19 s for 2.5e5 particles x 100 steps "
                          "on 2x Xeon Silver 4310T (20 cores, AVX-512), i.e. >= 1.1e7 particle-steps/s "
                          "(a lower bound derived here; the paper quotes no particle-steps/s)"),
        "clocks": clk.summary(),
    }
    line.update(other_windows)
    if fp64:
        line["fp64"] = fp64
        line["fp32_speedup_over_fp64"] = line["value"] / fp64["value"]
    if mlp:
        line["surrogate"] = mlp
        line["surrogate_speedup_over_table_fp32"] = mlp["value"] / line["value"]
        if fp64:
            line["surrogate_speedup_over_fp64_table"] = mlp["value"] / fp64["value"]
    if od:
        line["optical_depth_method"] = od
    if growth:
        line["test_problem_growth"] = growth
    if e2e:
        line["e2e"] = e2e
    if cpu:
        line["cpu_baseline"] = {"value": cpu[0], "unit": "particle-steps/s", "cores": cpu[2], "kind": "oracle",
                                "sample": cpu[3], "events_per_s": cpu[1]}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Instruction issue peak of one GB300: 152 SMs x 4 schedulers x 2.07 GHz,
# one warp instruction per scheduler per clock.
ISSUE_PEAK_WARP_INSTR = 152 * 4 * 2.07e9
# Warp instructions per lepton-step of the step-fused batch kernel (128
# threads) from one ncu capture of the current kernel: the 10-step call's
# count over its 4.02e7 lepton-steps
# (profiles/k_emission_fused_batched_uniform_b.md); None when not captured
NCU_FUSED_WARP_INSTR_PER_STEP = {"fp32": 40.8, "fp64": None}


# The paper's test problem (Sec. 5.1-5.2): growth rate of the cascade in its
# exponential stage and the lepton density profile, per mode and seed
GROWTH_SEEDS = (11, 12, 13, 14, 15)
GROWTH_CAP = 2_000_000          # leveling cap per species (the paper does not print its own)
GROWTH_FIT = (700, 1000)        # steps fitted: 3.5 T to 5 T (the paper: exponential after ~3.5 T)
GROWTH_FIT_20T = (700, 4000)    # the 20 T runs: 3.5 T to 20 T
GROWTH_BINS = 64


def growth_run(precision, seed, mlp_params=None, n=250_000, cap=GROWTH_CAP, hook=None, periods=5, fit=GROWTH_FIT):
    """One run of the test problem over `periods` periods (5 T by default;
    one step per call): Gamma (per period) from the slope of ln W, W the
    leptons' total weight (leveling keeps its expectation), over the steps
    `fit`; the weighted lepton density along x (wrapped to the box) at the
    end, normalised.  hook(step, gen, ens) runs before each step."""
    import numpy as np
    import torch
    import paper_2409_17299_gb300 as q
    w = W.paper_test_problem(n=n, seed=seed, thin_cap=cap, periods=periods)
    prec = q.QED_FP32 if precision == "fp32" else q.QED_FP64
    gen = q.Generator(q.make_config(precision=prec, seed=w.seed, push_photons=1, thin_cap=cap,
                                    sampler=q.QED_SAMPLER_MLP if mlp_params is not None else q.QED_SAMPLER_TABLE))
    if mlp_params is not None:
        q.qed_mlp_set_params(gen.ctx, mlp_params)
    ens = q.DeviceEnsemble.from_host(w.species, [int(1.3 * cap) + n, int(1.3 * cap) + n, int(1.8 * cap) + n], prec)
    field = q.make_field(w.field_kind, w.field_prm)
    lnw = []
    t0 = time.perf_counter()
    for s in range(w.nsteps):
        if hook is not None:
            hook(s, gen, ens, w, field)
        gen.push(ens, field, w.dt, 1, s)
        tot = sum(ens.arr[k]["w"][:ens.count[k]].double().sum() for k in (0, 1))
        lnw.append(math.log(float(tot)))
    secs = time.perf_counter() - t0
    t = (np.arange(w.nsteps) + 1) * w.dt
    a, b = fit
    gamma = float(np.polyfit(t[a:b], np.array(lnw[a:b]), 1)[0] * 2 * math.pi)
    xs, ws = [], []
    for k in (0, 1):
        m = ens.count[k]
        xs.append(ens.arr[k]["x"][:m].double().cpu().numpy())
        ws.append(ens.arr[k]["w"][:m].double().cpu().numpy())
    x = (np.concatenate(xs) + math.pi) % (2 * math.pi) - math.pi
    h, _ = np.histogram(x, bins=GROWTH_BINS, range=(-math.pi, math.pi), weights=np.concatenate(ws))
    counts = list(ens.count)
    gen.close()
    del ens
    torch.cuda.empty_cache()
    return {"gamma": gamma, "profile": (h / h.sum()).tolist(), "counts": counts, "seconds": secs}


def growth_summary(runs):
    """Gamma mean, standard deviation, 3-sigma envelope of the mean and the
    mean profile of a mode's runs."""
    import numpy as np
    g = np.array([r["gamma"] for r in runs])
    sd = float(g.std(ddof=1)) if len(g) > 1 else 0.0
    m = float(g.mean())
    env = 3 * sd / math.sqrt(len(g))
    return {"gamma_per_period": g.tolist(), "gamma_mean": m, "gamma_std": sd, "gamma_mean_3sigma": [m - env, m + env],
            "profile_mean": np.mean([r["profile"] for r in runs], axis=0).tolist(),
            "seconds": float(sum(r["seconds"] for r in runs))}


def profile_step(w, precision, step, mlp_params=None, method=0):
    """Drive the workload to `step` (captured steps), then run one step
    through the host-driven launches inside cudaProfilerStart/Stop: the small
    case an ncu capture of single kernels is taken on.  mlp_params: network
    sampler with these parameters; method: event method."""
    import torch
    import paper_2409_17299_gb300 as q
    prec = q.QED_FP32 if precision == "fp32" else q.QED_FP64
    caps = [int(c * 1.1) for c in capacities(w, w.nsteps)]
    sampler = q.QED_SAMPLER_MLP if mlp_params is not None else q.QED_SAMPLER_TABLE

    def generator(profile):
        g = q.Generator(q.make_config(precision=prec, seed=w.seed, push_photons=w.push_photons,
                                      thin_cap=w.thin_cap, profile=profile, sampler=sampler, event_method=method))
        if mlp_params is not None:
            q.qed_mlp_set_params(g.ctx, mlp_params)
        return g
    gen = generator(0)
    ens = q.DeviceEnsemble.from_host(w.species, caps, prec, optical_depth=method != 0)
    field = q.make_field(w.field_kind, w.field_prm)
    for s in range(0, step, 10):
        gen.push(ens, field, w.dt, min(10, step - s), s)
    genp = generator(1)
    counts0 = list(ens.count)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    st = genp.push(ens, field, w.dt, 1, step)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profiled_step": step, "counts_at_start": counts0, "counts_after": list(ens.count),
                      **{k: st[k] for k in ("particle_steps", "lepton_steps", "photon_steps", "emit_events",
                                            "pair_events", "passes", "thinned", "moved")}}), flush=True)
    gen.close()
    genp.close()


def train_surrogate_timed(samples, peaks, batch=8192):
    """Train the surrogate on `samples` table draws (batch 8192 and lr 4e-3
    are the settings the tests use) after a short warm-up training; wall time
    of the call and the training roofline against the measured BF16 peak."""
    import torch
    import paper_2409_17299_gb300 as q
    tg = q.Generator(q.make_config(precision=q.QED_FP32))
    q.qed_train_surrogate(tg.ctx, batch * 16, batch, 4e-3, 7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = q.qed_train_surrogate(tg.ctx, samples, batch, 4e-3, 7)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    P = q.qed_mlp_get_params(tg.ctx)
    tg.close()
    bf16_peak = peaks.get("bf16_tflops")
    ach = MLP_TRAIN_FLOP_PER_SAMPLE * samples / train_s / 1e12
    return P, {
        "train_samples": samples, "train_batch": batch, "train_seconds": train_s, "train_final_mse": loss,
        "network": "2-64-64-64-1 SiLU, BF16 weights, FP32 accumulation; training on tcgen05.mma with "
                   "tensor-memory accumulators (one cooperative launch), inference inside the lepton "
                   "pass on mma.sync",
        "train_roofline": {
            "bound": "tensor", "achieved": ach, "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": ach / bf16_peak if bf16_peak else None,
            "peak_source": "measured bf16_tflops (burst)" if bf16_peak else None,
            "flop_per_sample": MLP_TRAIN_FLOP_PER_SAMPLE,
            "achieved_is": "algorithmic FLOPs of the matrix products x samples / wall time of the training call"}}


def fp64_roofline(tot, hbm_peak):
    """The FP64 mode's pass kernels against the measured FP64 arithmetic peak
    (qed_measure_fp64_peak, timed live) and against HBM."""
    import paper_2409_17299_gb300 as q
    peak, _ = q.qed_measure_fp64_peak(1 << 16)
    out = {"bound": "fp64", "unit": "FLOP/s", "peak": peak,
           "peak_source": "measured: qed_measure_fp64_peak (FP64 FMA chains, one wave of resident blocks)",
           "flop_is": "2 DFMA + DADD + DMUL thread instructions per particle-step (ncu) x particle-steps / "
                      "summed CUDA-event time of the launches", "kernels": {}}
    for k, ms, units, nbytes in (("k_lepton_pass", tot["kernel_ms"][0], tot["lepton_steps"],
                                  LEPTON_BYTES["fp64"] * tot["lepton_steps"] + EMIT_BYTES["fp64"] * tot["emit_events"]),
                                 ("k_photon_pass", tot["kernel_ms"][1], tot["photon_steps"],
                                  PHOTON_BYTES["fp64"] * tot["photon_steps"] + PAIR_BYTES["fp64"] * tot["pair_events"])):
        if ms <= 0:
            continue
        fl = NCU_FP64_FLOP_PER_STEP[k] * units / (ms / 1e3)
        gbs = nbytes / (ms / 1e3) / 1e9
        out["kernels"][k] = {"kernel_ms": ms, "achieved": fl, "frac": fl / peak,
                             "flop_per_particle_step": NCU_FP64_FLOP_PER_STEP[k],
                             "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak}
    dom = max(out["kernels"], key=lambda k: out["kernels"][k]["kernel_ms"]) if out["kernels"] else None
    if dom:
        out.update({"kernel": dom + "<double>", "achieved": out["kernels"][dom]["achieved"],
                    "frac": out["kernels"][dom]["frac"], "hbm_frac": out["kernels"][dom]["hbm_frac"]})
    return out


def batch_roofline(st, precision):
    """The step-fused kernel reads and writes each lepton once per call, so
    it is bound by instruction issue, not HBM: achieved = warp instructions
    per lepton-step (ncu) x lepton-steps / kernel time, against the issue
    peak."""
    ms = st["kernel_ms"][0]
    per = NCU_FUSED_WARP_INSTR_PER_STEP.get(precision)
    ach = per * st["lepton_steps"] / (ms / 1e3) if (per and ms > 0) else None
    return {"bound": "alu", "unit": "warp instructions/s", "achieved": ach, "peak": ISSUE_PEAK_WARP_INSTR,
            "frac": ach / ISSUE_PEAK_WARP_INSTR if ach else None, "traffic": None,
            "peak_source": "152 SMs x 4 schedulers x 2.07 GHz (one warp instruction per scheduler per clock)",
            "warp_instr_per_lepton_step": per, "kernel": "k_emission_fused<%s>" % (
                "float" if precision == "fp32" else "double"), "kernel_ms": ms,
            "note": "step-fused: leptons stay in registers across steps; HBM traffic is per call, not per step"}


def batched_main(args, ws, warm, steps, rank, world, cpu):
    import torch
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms, st, counts, tuned = batch_run(ws, args.precision, warm, steps, args.batch_threads)
    ps, ev, secs = reduce_over_ranks(float(st["particle_steps"]), float(st["emit_events"]), ms / 1e3, world)
    if rank != 0:
        return
    n_lep = sum(len(w.species[0]["id"]) for w in ws)
    line = {
        "metric": "particle-steps/s", "value": ps / secs, "unit": "particle-steps/s", "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": "batched_uniform_b", "ensembles": len(ws), "leptons": n_lep,
                   "precision": args.precision, "launch": "one persistent kernel per call (CUDA graph)",
                   "l2": "inputs larger than L2 (%d MB of leptons)" % (n_lep * 40 // 2 ** 20)},
        "events_per_s": ev / secs,
        "gpu_launches": st["launches"],
        "autotune": ({"chosen_threads": tuned[0], "chosen_step_budget": tuned[2],
                      "ms_128_256_512_at_best_budget": tuned[1]} if tuned else None),
        "roofline": batch_roofline(st, args.precision),
        "clocks": clk.summary(),
    }
    if cpu:
        line["cpu_baseline"] = {"value": cpu[0], "unit": "particle-steps/s", "cores": cpu[2], "kind": "oracle",
                                "sample": cpu[3], "events_per_s": cpu[1]}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
