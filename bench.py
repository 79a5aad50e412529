#!/usr/bin/env python3
"""Throughput benchmark of the GB300 Yee FDTD step (one JSON line on rank 0).

Workload (default): a 512^3-cell PEC cavity, FP32 storage, background eps_r = 1
plus 32 seeded dielectric spheres (radius 8-40 cells, eps_r in {2.25, 4.0}),
mu_r = 1, dt = 0.5/sqrt(3), uniform[-1, 1) random initial fields.  One bench
step is one solve of 200 leapfrog steps followed by the FP64 energy check.

  value       Gcell-updates/s = cells * 200 * steps * ranks / time, inputs resident in HBM
  e2e         the same, with the host->device load of the fields (pinned memory) and the
              device->host read of the energy inside every timed step
  roofline    the dominant kernel (two-step temporal-blocking launch): algorithmic bytes per launch
              (one read + one write of every field per launch) / mean launch time vs the measured
              HBM copy peak
  cpu_baseline  the FP64 oracle (OpenMP, all host cores) on a bounded sample of the workload

Multi-GPU (torchrun): each rank solves its own cavity (independent replicas, no
collective on the data path); value sums all ranks over the max-over-ranks time.
`--impl reference` times the oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import cavity_inputs as ci  # noqa: E402

WORKLOADS = {
    # name: (nx, ny, nz, leapfrog steps per bench step, storage, sphere seed, field seed)
    "single512": dict(n=(512, 512, 512), steps=200, storage=0, sphere_seed=1, field_seed=2, spheres=32),
    # the same cavity with 16-bit storage (FP32 arithmetic)
    "single512_f16": dict(n=(512, 512, 512), steps=200, storage=1, sphere_seed=1, field_seed=2, spheres=32),
    "single512_bf16": dict(n=(512, 512, 512), steps=200, storage=2, sphere_seed=1, field_seed=2, spheres=32),
    # small case for ncu captures (fields 0.8 GB > L2, a few launches)
    "single256": dict(n=(256, 256, 256), steps=20, storage=0, sphere_seed=1, field_seed=2, spheres=8),
    "single256_f16": dict(n=(256, 256, 256), steps=20, storage=1, sphere_seed=1, field_seed=2, spheres=8),
    # DRAM-counter case of single512: the same 512 x 512 tiles over 64 planes (0.8 GB of fields > L2), whose
    # traffic per plane is that of the full cavity (scaled by 512 / 64 for its launches)
    "single512_z64": dict(n=(512, 512, 64), steps=20, storage=0, sphere_seed=1, field_seed=2, spheres=32),
    "precision384_f16": dict(n=(384, 384, 384), steps=1000, storage=1, sphere_seed=3, field_seed=4, spheres=32),
    "precision384_bf16": dict(n=(384, 384, 384), steps=1000, storage=2, sphere_seed=3, field_seed=4, spheres=32),
    # 256 independent cavities, sides iid U{16..96}, vacuum or spheres (p = 1/2), 500 steps per bench step
    "batch256": dict(kind="batch", count=256, lo=16, hi=96, steps=500, seed=5, storage=0),
    # Poisson stream: 200 req/s, sides log-uniform 16-256, steps U{100..2000}, BF16 flag Bernoulli(1/2)
    "serve": dict(kind="serve", rate=200.0, seed=6, budget_gb=120),
    # error study: 384^3 spheres, 1000 steps, FP32 / FP16 / BF16 storage against the FP64 oracle
    "precision": dict(kind="precision", n=(384, 384, 384), steps=1000, sphere_seed=3, field_seed=4, spheres=32),
    # the single512 cavity as 4 z-slabs on this GPU: two ghost planes per side, one two-step launch per exchange
    "slab512": dict(kind="slab", n=(512, 512, 512), steps=200, storage=0, sphere_seed=1, field_seed=2, spheres=32,
                    nslabs=4, ghost=2),
    # the fourth-order (2,4) scheme on the single512 cavity (fused fourth-order kernel, one step per launch)
    "order4_512": dict(n=(512, 512, 512), steps=200, storage=0, sphere_seed=1, field_seed=2, spheres=32, order=4,
                       tuning=dict(kernel=2, tile_y=12, stages=5, zchunk=0, ctas_per_sm=0, use_graph=1)),
    "order4_512_f16": dict(n=(512, 512, 512), steps=200, storage=1, sphere_seed=1, field_seed=2, spheres=32, order=4,
                           tuning=dict(kernel=2, tile_y=12, stages=5, zchunk=0, ctas_per_sm=0, use_graph=1)),
    # small case of the same for ncu captures (FP32 and FP16 storage)
    "order4_256": dict(n=(256, 256, 256), steps=20, storage=0, sphere_seed=1, field_seed=2, spheres=8, order=4,
                       tuning=dict(kernel=2, tile_y=12, stages=5, zchunk=0, ctas_per_sm=0, use_graph=1)),
    "order4_256_f16": dict(n=(256, 256, 256), steps=20, storage=1, sphere_seed=1, field_seed=2, spheres=8, order=4,
                           tuning=dict(kernel=2, tile_y=12, stages=5, zchunk=0, ctas_per_sm=0, use_graph=1)),
}
# Launch configuration the bench times (the full-size parity test uses the same): the two-step
# temporal-blocking kernel, 60 x 16-cell tiles (FP32), 4-slot TMA ring (what fits beside 16-row
# planes), graphs of 8 launches.
BENCH_TUNING = dict(kernel=3, tile_y=16, stages=4, zchunk=0, ctas_per_sm=0, use_graph=1)
# Batches of the serving loop: two-step launches, 16-row tiles (what fdtd_batch_autotune picks for the
# batch workload, and measured best on the serving stream; the mix changes every chunk, so it is fixed
# rather than re-tuned).
SERVE_TUNING = dict(kernel=3, tile_y=16, stages=4)
STEPS_PER_LAUNCH = {1: 0.5, 2: 1, 3: 2, 4: 2, 5: 3}   # leapfrog steps per launch of each kernel kind (SIMPLE: H and E launches)
DOMINANT_KERNEL = {1: "simple_h_kernel/simple_e_kernel", 2: "fused_step_kernel", 3: "fused2_step_kernel",
                   4: "fused2r_step_kernel", 5: "fused3_step_kernel"}
ID_BYTES = 1  # material id per cell
NOMINAL_HBM_GBS = 8000.0   # GB300 HBM3e nominal bandwidth (context beside the measured copy peak)

# DRAM traffic per fused launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the
# SHA-256 of the kernel source and the device headers it includes, as measured; ignored (reported null)
# once any of them changes.
MEASURED_TRAFFIC = {
    # ncu (one-pass metric set), 512^3 bench configuration, mean of three launches of the two-step kernel
    # (6.84 / 6.94 / 6.89 GB)
    ("single512", "810efbd94e2c72f5"): 6.889e9,
}


TUNING_OVERRIDE: dict | None = None   # --tuning: fields of the single-cavity launch configuration to replace


def tuning_of(w) -> dict:
    base = w.get("tuning", BENCH_TUNING)
    if TUNING_OVERRIDE is not None:
        return dict(base, **TUNING_OVERRIDE)
    return base


def dominant_kernel(w) -> str:
    k = tuning_of(w)["kernel"]
    if w.get("order", 2) == 4:
        return {1: "simple4_h_kernel/simple4_e_kernel"}.get(k, "fused4_step_kernel")
    return DOMINANT_KERNEL[k]


def kernel_source_hash(w=None) -> str:
    k = tuning_of(w or {})["kernel"]
    if (w or {}).get("order", 2) == 4:
        src = "k_order4.cu" if k == 1 else "k_fused4.cu"
    else:
        src = {2: "k_fused.cu", 3: "k_fused2.cu", 4: "k_fused2r.cu", 5: "k_fused3.cu"}.get(k, "k_simple.cu")
    headers = ["fdtd_internal.cuh", "fused_common.cuh"] + (["order4.cuh"] if (w or {}).get("order", 2) == 4 else [])
    h = hashlib.sha256()
    for name in [src] + headers:
        h.update(code_only(open(os.path.join(ROOT, "paper_2504_09118_gb300", "csrc", name)).read()).encode())
    return h.hexdigest()[:16]


def code_only(text: str) -> str:
    """CUDA source without comments and whitespace runs: what the compiler sees, so that a comment edit
    keeps a measured traffic figure attached to the unchanged kernel."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def sphere_coefs(w):
    nx, ny, nz = w["n"]
    sph = ci.sphere_list(w["sphere_seed"], w["spheres"], (nx, ny, nz), 8.0, 40.0)
    return ci.sphere_coefficients(sph, nx, ny, nz, ci.COURANT_HALF_DT)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None):
        self.proc = None
        self.path = path or os.path.join("/tmp", f"fdtd_clocks_{os.getpid()}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        try:
            self.fh.close()
        except Exception:
            pass

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except Exception:
            rows = []
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's); x itself for one rank."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ws: int, seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time (weak scaling)."""
    return units_per_rank * ws / seconds


def cpu_baseline(w, budget_s: float = 12.0):
    """Time the FP64 oracle (OpenMP build, all host cores) on a bounded z-slab of the workload."""
    import oracle
    nx, ny, _ = w["n"]
    nzs = 16
    ce, ch = (None, None)
    sph = ci.sphere_list(w["sphere_seed"], w["spheres"], w["n"], 8.0, 40.0)
    ce_s, ch_s = ci.sphere_coefficients(sph, nx, ny, nzs, ci.COURANT_HALF_DT)
    f = oracle.as_f64(ci.random_fields(w["field_seed"], nx, ny, nzs))
    ce64 = [c.astype(np.float64) for c in ce_s]
    step = oracle.step4 if w.get("order", 2) == 4 else oracle.step
    t0 = time.perf_counter()
    step(f, ce64, ch_s, 1, omp=True)
    one = time.perf_counter() - t0
    steps = max(1, min(200, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    step(f, ce64, ch_s, steps, omp=True)
    dt = time.perf_counter() - t0
    rate = nx * ny * nzs * steps / dt / 1e9
    # the same oracle on one thread (the paper's single-thread setting), 128^3 vacuum, a few steps
    g = oracle.as_f64(ci.random_fields(w["field_seed"], 128, 128, 128))
    t0 = time.perf_counter()
    step(g, ci.COURANT_HALF_DT, ci.COURANT_HALF_DT, 1, omp=False)
    one = time.perf_counter() - t0
    s1 = max(1, min(20, int(0.25 * budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    step(g, ci.COURANT_HALF_DT, ci.COURANT_HALF_DT, s1, omp=False)
    d1 = time.perf_counter() - t0
    return {"value": round(rate, 4), "unit": "Gcell-updates/s", "cores": oracle.threads(True), "kind": "oracle",
            "affinity_cores": len(os.sched_getaffinity(0)),
            "sample": f"{nx}x{ny}x{nzs} slab of the {w['n'][0]}x{w['n'][1]}x{w['n'][2]} workload "
                      f"(same sphere layout), FP64 OpenMP oracle (order {w.get('order', 2)}), {steps} steps "
                      f"in {dt:.1f} s",
            "single_thread": {"value": round(128 ** 3 * s1 / d1 / 1e9, 4), "unit": "Gcell-updates/s",
                              "sample": f"128^3 vacuum, serial FP64 oracle, {s1} steps in {d1:.1f} s"}}


def run_reference(args, w, wname):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    if "n" not in w or w.get("kind"):
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm is timed on the single-cavity "
                                                              f"workloads only, not on '{wname}'"}), flush=True)
        return
    import oracle
    nx, ny, nz = w["n"]
    nzs = 16
    sph = ci.sphere_list(w["sphere_seed"], w["spheres"], w["n"], 8.0, 40.0)
    ce_s, ch_s = ci.sphere_coefficients(sph, nx, ny, nzs, ci.COURANT_HALF_DT)
    ce64 = [c.astype(np.float64) for c in ce_s]
    f = oracle.as_f64(ci.random_fields(w["field_seed"], nx, ny, nzs))
    per_step = 2  # oracle leapfrog steps per bench step: a bounded sample of the solve
    order4 = w.get("order", 2) == 4
    step = oracle.step4 if order4 else oracle.step
    energy = oracle.energy4 if order4 else oracle.energy
    for _ in range(args.warmup):
        step(f, ce64, ch_s, 1, omp=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(f, ce64, ch_s, per_step, omp=True)
        energy(f, ce64, ch_s, ci.COURANT_HALF_DT)
    dt = time.perf_counter() - t0
    val = nx * ny * nzs * per_step * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": "Gcell-updates/s", "value": round(val, 4), "unit": "Gcell-updates/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "cells": [nx, ny, nz], "sample_cells": [nx, ny, nzs],
                       "leapfrog_steps_per_bench_step": per_step},
            "cpu_baseline": {"value": round(val, 4), "unit": "Gcell-updates/s", "cores": oracle.threads(True),
                             "affinity_cores": len(os.sched_getaffinity(0)), "kind": "oracle", "sample": f"{nx}x{ny}x{nzs} slab, {per_step} FP64 steps + energy per bench step"},
            "e2e": {"value": round(val, 4), "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, w):
    """Batched persistent launches vs plain one-launch-per-step stepping of each cavity alone.
    Returns the leg's results (its own timed region and clock summary)."""
    import torch
    from paper_2504_09118_gb300 import Cavity, binding
    torch.cuda.set_device(0)
    cavs = ci.batch_cavities(w["seed"], w["count"], w["lo"], w["hi"])
    stream = torch.cuda.Stream()
    members = []
    for c in cavs:
        nx, ny, nz = c["nx"], c["ny"], c["nz"]
        ce = ch = None
        if c["spheres"]:
            ce, ch = ci.sphere_coefficients(c["spheres"], nx, ny, nz, ci.COURANT_HALF_DT)
        cav = Cavity(nx, ny, nz, ci.COURANT_HALF_DT, 1.0, ce, ch, w["storage"], stream)
        cav.set_fields(ci.random_fields(c["field_seed"], nx, ny, nz))
        members.append(cav)
    cells = sum(c.dims[0] * c.dims[1] * c.dims[2] for c in members)
    per = w["steps"]
    b = binding.fdtd_batch_create(w["storage"], stream)
    for m in members:
        binding.fdtd_batch_add(b, m.handle)
    # the batch's kernel and tile shape: timed on the members' own state by the library (restored after)
    t_tune = time.perf_counter()
    tuning, _ = binding.fdtd_batch_autotune(b, 32)
    t_tune = time.perf_counter() - t_tune
    for _ in range(args.warmup):
        binding.fdtd_batch_step(b, per)
    binding.fdtd_batch_sync(b)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0, args.clocks_csv) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            binding.fdtd_batch_step(b, per)
        ev1.record(stream)
        binding.fdtd_batch_sync(b)
    ms = ev0.elapsed_time(ev1)
    value = cells * per * args.steps / (ms / 1e3) / 1e9
    for m in members:
        binding.fdtd_batch_remove(b, m.handle)
    binding.fdtd_batch_destroy(b)
    # plain: every cavity alone, one launch per step, no graph
    for m in members:
        m.tune(kernel=2, tile_y=8, stages=4, use_graph=0)
        m.step(2)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain_steps = min(per, 100)
    p0.record(stream)
    for m in members:
        m.step(plain_steps)
    p1.record(stream)
    torch.cuda.synchronize()
    plain = cells * plain_steps / (p0.elapsed_time(p1) / 1e3) / 1e9
    for m in members:
        m.close()
    return {"metric": "Gcell-updates/s", "value": round(value, 3), "unit": "Gcell-updates/s",
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch256", "cavities": len(members), "cells": cells,
                       "sides": f"iid U{{{w['lo']}..{w['hi']}}} per axis, vacuum or spheres (p = 1/2), seed {w['seed']}",
                       "leapfrog_steps_per_bench_step": per, "graph_steps": 16,
                       "autotuned": tuning, "autotune_s": round(t_tune, 3)},
            "plain_one_launch_per_step": round(plain, 3), "plain_steps": plain_steps,
            "batched_vs_plain": round(value / plain, 3),
            "clocks": clk.summary(),
            # each launch (one step, or two with the two-step kernel) is followed by the clock kernel
            "gpu_launches": 2 * args.steps * per // (2 if tuning["kernel"] in (3, 4) else 1)}


def run_serve(args, w):
    """Continuous-batching server on a Poisson stream vs plain one-request-at-a-time stepping (the
    sequential baseline runs closed-loop over a stated prefix of the same stream).  Returns the leg's
    results."""
    import torch
    from paper_2504_09118_gb300.serve import Request, Server, serve_sequential
    torch.cuda.set_device(0)
    stream = ci.serve_stream(w["seed"], args.serve_requests, w["rate"])
    gen = torch.Generator(device="cuda")

    def fields_fn(r):   # seeded synthetic fields generated on the device (host generation would dominate)
        gen.manual_seed(r.id + 1)
        shape = (r.nz + 1, r.ny + 1, r.nx + 1)
        return [torch.rand(shape, generator=gen, device="cuda") * 2 - 1 for _ in range(6)]

    tuning = json.loads(args.serve_tuning) if args.serve_tuning else SERVE_TUNING

    def make_server(retune=False):
        return Server(ci.COURANT_HALF_DT, hbm_budget_bytes=int(w["budget_gb"] * (1 << 30)), max_slots=1024,
                      K=args.serve_chunk, tuning=tuning, result="energy", fields_fn=fields_fn, retune=retune)

    # untimed warm-up: a short stream of the same recipe (another seed) through a server of its own, so
    # that library load, pool growth, tensor maps and graph captures are not charged to the timed stream
    warm = ci.serve_stream(w["seed"] + 1000, args.warmup * 50, w["rate"]) if args.warmup > 0 else []
    if warm:
        srv = make_server()
        srv.run([Request(q["id"], q["arrival_s"], q["nx"], q["ny"], q["nz"], q["steps"], q["bf16"]) for q in warm])
        srv.close()
    reqs = [Request(q["id"], q["arrival_s"], q["nx"], q["ny"], q["nz"], q["steps"], q["bf16"]) for q in stream]
    srv = make_server()
    with ClockSampler(0, args.clocks_csv) as clk:
        st = srv.run(reqs)
    srv.close()
    # the same stream with online re-tuning (size-bucket model in the library; the warm-up stream, served
    # the same way first, leaves the model with the buckets it met)
    online = None
    if args.serve_retune:
        if warm:
            srv = make_server(retune=True)
            srv.run([Request(q["id"], q["arrival_s"], q["nx"], q["ny"], q["nz"], q["steps"], q["bf16"]) for q in warm])
            srv.close()
        srv = make_server(retune=True)
        st_r = srv.run([Request(q["id"], q["arrival_s"], q["nx"], q["ny"], q["nz"], q["steps"], q["bf16"])
                        for q in stream])
        online = {"gcells": round(st_r.gcells, 3), "p50_s": round(st_r.p50_s, 4), "p99_s": round(st_r.p99_s, 4),
                  "wall_s": round(st_r.wall_s, 3), "retunes": {k: (round(v, 3) if isinstance(v, float) else v)
                                                               for k, v in srv.retunes.items()}}
        srv.close()
    nseq = min(len(stream), args.serve_seq_requests)
    seq_reqs = [Request(q["id"], q["arrival_s"], q["nx"], q["ny"], q["nz"], q["steps"], q["bf16"])
                for q in stream[:nseq]]
    with ClockSampler(0, None) as clk_seq:
        sq = serve_sequential(seq_reqs, ci.COURANT_HALF_DT, result="energy", fields_fn=fields_fn)
    offered = st.cell_updates / max(r["arrival_s"] for r in stream) / 1e9
    return {"metric": "Gcell-updates/s", "value": round(st.gcells, 3), "unit": "Gcell-updates/s",
            "requests": st.n, "failed": st.failed, "ms_per_request": round(1e3 * st.wall_s / max(st.n, 1), 3),
            "dtype": "f32 or bf16-storage per request", "data": "synthetic",
            "config": {"workload": "serve", "requests": len(stream), "rate_hz": w["rate"],
                       "sides": "log-uniform 16-256 per axis", "steps": "U{100..2000}", "bf16": "Bernoulli(1/2)",
                       "budget_gb": w["budget_gb"], "graph_steps": args.serve_chunk, "tuning": tuning, "max_slots": 1024,
                       "warmup_requests": len(warm), "seed": w["seed"]},
            "serving": {"p50_s": round(st.p50_s, 4), "p99_s": round(st.p99_s, 4), "mean_s": round(st.mean_s, 4),
                        "wall_s": round(st.wall_s, 3), "max_active": st.max_active,
                        "offered_gcells": round(offered, 2)},
            "sequential": {"requests": sq.n, "gcells": round(sq.gcells, 3), "p50_s": round(sq.p50_s, 4),
                           "p99_s": round(sq.p99_s, 4), "wall_s": round(sq.wall_s, 3), "closed_loop": True,
                           "sample": f"the first {sq.n} requests of the same stream, one at a time, one plain "
                                     f"launch per step, each started as soon as the previous one finished",
                           "clocks": clk_seq.summary()},
            "served_vs_sequential": round(st.gcells / sq.gcells, 3), "online_retune": online,
            "clocks": clk.summary()}


def run_precision(args, w):
    """Storage precision (FP32 arithmetic): the same seeded 384^3 sphere cavity stepped 1000 times with
    FP32, FP16 and BF16 storage; per-field rel-L2 of the 16-bit runs against the FP32 run and every run's
    energy drift (the library's FP64 energy).  The FP32 run itself is held to the FP64 oracle by the
    full-size parity tests.  Returns the leg's results."""
    import torch
    from paper_2504_09118_gb300 import Cavity
    torch.cuda.set_device(0)
    nx, ny, nz = w["n"]
    steps = args.precision_steps or w["steps"]
    ce, ch = sphere_coefs(w)
    f = ci.random_fields(w["field_seed"], nx, ny, nz)
    runs, times = {}, {}
    stream = torch.cuda.Stream()
    with ClockSampler(0, None) as clk:
        for st, name in ((0, "f32"), (1, "f16"), (2, "bf16")):
            with Cavity(nx, ny, nz, ci.COURANT_HALF_DT, 1.0, ce, ch, st, stream) as cav:
                cav.tune(**BENCH_TUNING)
                cav.set_fields(f)
                w0 = cav.energy()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                cav.step(steps)
                e1.record(stream)
                w1 = cav.energy()
                times[name] = e0.elapsed_time(e1) / steps
                runs[name] = (cav.get_fields(), w0, w1)

    def rel(a, b):
        out = {}
        for c, name in enumerate(ci.COMPONENTS):
            m = ci.extent_mask(name, nx, ny, nz)
            d = np.asarray(a[c], np.float64)[m] - np.asarray(b[c], np.float64)[m]
            out[name] = float(np.linalg.norm(d) / np.linalg.norm(np.asarray(b[c], np.float64)[m]))
        return out

    res = {}
    for name, (g, w0, w1) in runs.items():
        res[name] = {"energy_drift": (w1 - w0) / w0, "ms_per_step": round(times[name], 4),
                     "gcells": round(nx * ny * nz / times[name] / 1e6, 2)}
        if name != "f32":
            res[name]["rel_l2_vs_f32_gpu"] = rel(g, runs["f32"][0])
    return {"metric": "rel-L2 vs the FP32 run, energy drift", "cells": [nx, ny, nz], "steps": steps,
            "config": {"workload": "precision384", "spheres": w["spheres"], "seeds": [w["sphere_seed"], w["field_seed"]],
                       "tuning": BENCH_TUNING, "scale": "one power-of-two scale per field (E, H), round to nearest even"},
            "storage": res, "clocks": clk.summary(),
            "oracle_parity": "tests/test_gpu_fullsize.py::test_384_precision_1000_steps_vs_oracle (FP64 oracle, "
                             "per field)"}


def run_slab(args, w):
    """The single-cavity workload split into z-slabs on this GPU (slab contexts on their own streams,
    device-to-device ghost exchanges between neighbours): Gcell-updates/s of the whole cavity, against the
    same cavity undivided in the same run.  Returns the leg's results."""
    import torch
    from paper_2504_09118_gb300 import Cavity
    from paper_2504_09118_gb300.slab import SlabDomain
    torch.cuda.set_device(0)
    nx, ny, nz = w["n"]
    cells, per = nx * ny * nz, w["steps"]
    ce, ch = sphere_coefs(w)
    f = ci.random_fields(w["field_seed"], nx, ny, nz)
    tuning = tuning_of(w)
    streams = [torch.cuda.Stream() for _ in range(w["nslabs"])]
    out = {}
    with SlabDomain(nx, ny, nz, ci.COURANT_HALF_DT, 1.0, ce, ch, w["storage"], w["nslabs"], w["ghost"], 2,
                    tuning, streams) as dom:
        dom.set_fields(f)
        for _ in range(args.warmup):
            dom.step(per)
        torch.cuda.synchronize()
        with ClockSampler(0, None) as clk:
            t0 = time.perf_counter()
            for _ in range(args.steps):
                dom.step(per)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        w_slab = dom.energy()
        out["slabs"] = {"value": round(cells * per * args.steps / dt / 1e9, 3), "clocks": clk.summary(),
                        "ms_per_step": round(1e3 * dt / args.steps, 3), "energy": w_slab}
    with Cavity(nx, ny, nz, ci.COURANT_HALF_DT, 1.0, ce, ch, w["storage"]) as cav:
        cav.tune(**tuning)
        cav.set_fields(f)
        for _ in range(args.warmup):
            cav.step(per)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            cav.step(per)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out["one_cavity"] = {"value": round(cells * per * args.steps / dt / 1e9, 3),
                             "ms_per_step": round(1e3 * dt / args.steps, 3)}
    return {"metric": "Gcell-updates/s", "value": out["slabs"]["value"], "unit": "Gcell-updates/s",
            "steps": args.steps, "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "slab512", "cells": [nx, ny, nz], "nslabs": w["nslabs"], "ghost": w["ghost"],
                       "leapfrog_steps_per_bench_step": per, "tuning": tuning,
                       "exchange": "device to device between neighbouring slab contexts, every 2 steps"},
            "slabs": out["slabs"], "one_cavity": out["one_cavity"],
            "slabs_vs_one_cavity": round(out["slabs"]["value"] / out["one_cavity"]["value"], 3)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="single512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--clocks-csv", default=None)
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-chunk", type=int, default=32,
                    help="serving: steps each batch advances per pass of the loop (one graph replay when a multiple of 16)")
    ap.add_argument("--serve-seq-requests", type=int, default=1000,
                    help="closed-loop prefix of the stream served by the sequential baseline")
    ap.add_argument("--serve-tuning", default=None,
                    help="JSON tuning of the serving batches (default: SERVE_TUNING)")
    ap.add_argument("--serve-retune", action="store_true",
                    help="serve the stream a second time with online re-tuning (fdtd_batch_retune)")
    ap.add_argument("--precision-steps", type=int, default=0)
    ap.add_argument("--legs", default="batched,served,precision",
                    help="comma-separated legs nested in the single-cavity line at N = 1 (batched: 256 uneven "
                         "cavities; served: the 10k-request Poisson stream; precision: 384^3 FP16/BF16); '' for none")
    ap.add_argument("--tuning", default=None,
                    help="JSON fields replacing those of the single-cavity workload's launch configuration (its "
                         "own, else BENCH_TUNING)")
    args = ap.parse_args()
    global TUNING_OVERRIDE
    if args.tuning:
        TUNING_OVERRIDE = json.loads(args.tuning)
    w = WORKLOADS[args.workload]
    standalone = {"batch": ("batched", run_batch), "serve": ("served", run_serve),
                  "precision": ("precision", run_precision), "slab": ("slab", run_slab)}
    if args.impl == "ours" and w.get("kind") in standalone:
        name, fn = standalone[w["kind"]]
        leg = fn(args, w)
        leg.update({"n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "leg": name})
        print(json.dumps(leg), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, w, args.workload)
        return

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2504_09118_gb300 import Cavity, binding

    nx, ny, nz = w["n"]
    cells = nx * ny * nz
    per = w["steps"]
    ce, ch = sphere_coefs(w)
    fields = ci.random_fields(w["field_seed"] + rank, nx, ny, nz)
    stream = torch.cuda.Stream()
    cav = Cavity(nx, ny, nz, ci.COURANT_HALF_DT, 1.0, ce, ch, w["storage"], stream, order=w.get("order", 2))
    tuning = tuning_of(w)
    cav.tune(**tuning)
    cav.set_fields(fields)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def bench_step():
        cav.step(per)
        return cav.energy()

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k_ms = []
    with ClockSampler(local, args.clocks_csv) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            ka, kb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ka.record(stream)
            cav.step(per)
            kb.record(stream)
            cav.energy()           # synchronises; part of the timed step (FP64 check, a7)
            k_ms.append(ka.elapsed_time(kb))
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, ws)
    value = job_rate(cells * per * args.steps, ws, ms / 1e3) / 1e9
    clocks = clk.summary()

    # roofline of the dominant kernel: algorithmic bytes per launch / mean launch time.  A launch of
    # the fused kernels reads and writes every field once (and reads the material id once), however
    # many leapfrog steps it advances; the solve is `per` steps = per / spl launches.
    esz = 4 if w["storage"] == 0 else 2
    spl = STEPS_PER_LAUNCH[tuning["kernel"]]
    alg_bytes = cells * (12 * esz + ID_BYTES)
    launches = per / spl
    launch_s = statistics.mean(k_ms) / 1e3 / launches
    achieved = alg_bytes / launch_s / 1e9
    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else 6800.0
    tr = MEASURED_TRAFFIC.get((args.workload, kernel_source_hash(w)))
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": tr,
                "frac_nominal": round(achieved / NOMINAL_HBM_GBS, 4), "peak_nominal": NOMINAL_HBM_GBS,
                "peak_source": "measured" if peaks else "fallback",
                "alg_bytes_per_launch": alg_bytes, "mean_launch_us": round(launch_s * 1e6, 2),
                "kernel": dominant_kernel(w), "steps_per_launch": spl,
                # the same time against one HBM sweep per step (12 x storage + 1 bytes per cell-update):
                # temporal blocking moves spl steps per sweep, so this exceeds the physical fraction
                "per_cell_update": {"bytes": 12 * esz + ID_BYTES,
                                    "achieved": round(alg_bytes * spl / launch_s / 1e9, 1),
                                    "frac": round(alg_bytes * spl / launch_s / 1e9 / peak, 4)}}

    # end to end through the C ABI with host buffers: H2D of the fields + solve + D2H of the energy
    # Each step's fields are copied from pinned host memory inside the timed region; the copy of step
    # i + 1's fields (fdtd_prefetch_fields, on the library's copy stream) runs while step i computes,
    # and the first step's copy is not overlapped.
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(a).pin_memory() for a in fields]
        host = [p.numpy() for p in pinned]
        cav.prefetch_fields(host)
        cav.set_fields_prefetched()
        bench_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        cav.prefetch_fields(host)
        for i in range(args.steps):
            cav.set_fields_prefetched()            # this step's inputs
            if i + 1 < args.steps:
                cav.prefetch_fields(host)          # the next step's, copied while this one computes
            bench_step()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if ws > 1:
            import torch.distributed as dist
            e2e_s = max_over_ranks(e2e_s, ws)
        e2e = {"value": round(job_rate(cells * per * args.steps, ws, e2e_s) / 1e9, 3), "unit": "Gcell-updates/s",
               "h2d_bytes_per_step": int(sum(a.nbytes for a in host)), "d2h_bytes_per_step": 8,
               "h2d": "pinned, overlapped with the previous step's solve (fdtd_prefetch_fields)"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)
    cav.close()
    # the other workloads of the method, each with its own timed region and clock record (one GPU only:
    # under torchrun every rank would hold its GPU while rank 0 alone ran them)
    legs = {}
    if ws == 1 and args.workload == "single512":
        wanted = [x.strip() for x in args.legs.split(",") if x.strip()]
        for name, wname, fn in (("batched", "batch256", run_batch), ("precision", "precision", run_precision),
                                ("served", "serve", run_serve)):
            if name in wanted:
                t0 = time.perf_counter()
                legs[name] = fn(args, WORKLOADS[wname])
                legs[name]["leg_wall_s"] = round(time.perf_counter() - t0, 1)
    if rank == 0:
        line = {"metric": "Gcell-updates/s", "value": round(value, 3), "unit": "Gcell-updates/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {0: "f32", 1: "f16-storage/f32-math", 2: "bf16-storage/f32-math"}[w["storage"]],
                "data": "synthetic",
                "config": {"workload": args.workload, "cells": [nx, ny, nz], "leapfrog_steps_per_bench_step": per,
                           "coefficients": f"{w['spheres']} dielectric spheres, 1-byte material id",
                           "parallelism": f"replicas x{ws}", "spatial_order": w.get("order", 2),
                           "l2": f"inputs larger than L2 ({6 * esz * cells / 1e9:.1f} GB of fields read and as many written per launch)",
                           "tuning": tuning, "hbm_fraction_of_roofline": round(achieved / peak, 4)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                # per bench step (one solve of `per` leapfrog steps, device time of the step launches)
                "solve_ms": {"best": round(min(k_ms), 3), "median": round(statistics.median(k_ms), 3),
                             "n": len(k_ms)},
                "gpu_launches": int(args.steps * (launches + 2))}
        line.update(legs)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
