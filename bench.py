"""Benchmark of the LOD diffusion-decay step on GB300 (one JSON line on rank 0).

Headline workload: 400 x 400 x 400 voxels x 4 substrates interleaved per voxel, dx = 20 um,
dt = 0.01 min, D = {1e5, 1e3, 5e2, 1e2} um^2/min, lambda = {0.1, 0.01, 0.4, 1e-3} /min,
1M agents with log-uniform secretion/uptake rates, initial field uniform in [0, 38] (seeded).
A bench step is one full LOD time step (Src, B, X^-1, B, Y^-1, B, Z^-1, B) of that grid.
The headline runs in FP64 (the paper's precision); FP32 is reported beside it, and the other
workloads (50^3 x 1 FP64, 1200^3 x 2 FP32 with Dirichlet faces, 256 batched environments,
the Sect. 5.3 end-to-end run, the adjoint) each get a leg of their own.

  value      voxel-substrate updates/s, field resident in HBM, graph-launched steps,
             CUDA events on the library's stream, max over ranks (replicas, weak scaling)
  e2e        the same metric through the C ABI from pinned host buffers: set_density(host),
             K steps, density(host), all inside the timed region
  roofline   dominant kernel: algorithmic bytes (one read + one write of the field per sweep)
             or FP64 operations per launch / its average CUDA-event duration over K steps; the
             FP64 arithmetic roof is the FMA rate measured in this run (biofvm_probe_fma_rate)
  error      every leg states its error: normwise max|got - ref| / max|ref| and the largest
             per-voxel relative error over voxels with |ref| above a floor, against the FP64
             oracle (FP64 legs) or the oracle-validated FP64 GPU path (FP32 legs)
  cpu_baseline  the FP64 oracle, single-threaded on this host, on a bounded slab sample, and
             its OpenMP copy on all host cores (the paper-style CPU rate)

`--impl reference` times the oracle instead (the reference arm), on the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
# Floating-point operations of the Thomas algorithm per element and sweep (Sect. 2.1, Eq. 2:
# forward axpy + division, backward negated axpy).
FLOPS_PER_ELEMENT_SWEEP = 5
# Sources whose kernels the traffic below was captured on (hash of their contents).
KERNEL_SOURCES = ["stream.cuh", "sweeps.cuh", "pipe.cuh", "pipe_args.h", "internal.h",
                  "sweeps_fp64.cu", "sweeps_fp32.cu", "pipe_fp32.cu", "pipe_h16.cu", "api.cpp"]
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of each sweep kernel of
# the 400^3 x 4 workload, from one ncu capture; reported only while the kernel sources still
# hash to `sources_sha256` (otherwise the kernels changed since and traffic is null).
MEASURED_TRAFFIC = {
    "sources_sha256": "dfdfcfc5517b3db62d07efd51e965a28556916ae6b5369129c40901f2a165b99",
    "bytes": {
        "fp64:x-sweep": 5710992896, "fp64:y-sweep": 5504968192, "fp64:z-sweep": 5532824320,
        "fp32:x-sweep": 2051157248, "fp32:y-sweep": 1983586816, "fp32:z-sweep": 1984059904,
        "bf16:x-sweep": 1027370496, "bf16:y-sweep": 965999616, "bf16:z-sweep": 966979072,
        "fp16:x-sweep": 1027427840, "fp16:y-sweep": 966120448, "fp16:z-sweep": 967207424,
    },
}
UNIT = "voxel-substrate updates/s"
# the headline workload's precisions: FP64 (the paper's), FP32, and 16-bit storage with FP32
# arithmetic
PRECISIONS = ("fp64", "fp32", "bf16", "fp16")
METRIC = "LOD step voxel-substrate updates/s (HBM GB/s vs peak in roofline)"


def kernel_sources_sha256():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2602_05017_gb300", "csrc", name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": HBM_FALLBACK_GBS, "sm_max_mhz": 2070.0}, "fallback"


def error_stats(got, ref, floor_rel):
    """Normwise max|got - ref| / max|ref|, and the largest |got - ref| / |ref| over elements
    with |ref| > floor_rel * max|ref| (the per-voxel measure; values near zero excluded)."""
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    d = np.abs(got - ref)
    m = float(np.abs(ref).max()) if ref.size else 0.0
    big = np.abs(ref) > floor_rel * m
    pv = float((d[big] / np.abs(ref[big])).max()) if big.any() else 0.0
    return {"normwise": float(d.max() / max(m, 1e-300)) if ref.size else 0.0,
            "per_voxel_max_rel": pv, "per_voxel_floor": f"|ref| > {floor_rel:g} max|ref|"}


def merge_errors(parts):
    """Worst of several error_stats over pieces of one result."""
    return {"normwise": max(p["normwise"] for p in parts),
            "per_voxel_max_rel": max(p["per_voxel_max_rel"] for p in parts),
            "per_voxel_floor": parts[0]["per_voxel_floor"]}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


SHAPE = None  # --shape overrides the grid (profiling a smaller case of the same recipe)
SUBS = None   # --subs keeps the first substrates of that recipe (profiling)


def aggregate(ms_local, world, units_per_rank, steps, device=None):
    """Max of the per-rank timed region over ranks and the whole-job rate it gives
    (every rank processes `units_per_rank` units per step: replicas, weak scaling)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * units_per_rank * steps / (ms_max * 1e-3)


def workload_config(with_field=True):
    from paper_2602_05017_gb300 import inputs
    if SHAPE is None:
        return inputs.workload(2, with_field=with_field)
    nvox = SHAPE[0] * SHAPE[1] * SHAPE[2]
    w = inputs.workload(2, shape=SHAPE, with_field=with_field, n_agents=nvox // 64)
    return w if SUBS is None else inputs.first_substrates(w, SUBS)


def flush_l2(dev):
    """Write a buffer larger than the 129 MB L2 (between timed repetitions of small fields)."""
    import torch
    buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB
    buf.fill_(1.0)
    del buf


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2602_05017_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload_config()
    nel = w.n_vs
    K, W = args.steps, args.warmup
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    results = {"fma_rate": {p: binding.probe_fma_rate(p, stream.cuda_stream)
                            for p in ("fp64", "fp32")}}
    ref100 = None  # FP64 GPU field after 100 steps (the FP32 leg's reference)
    for prec in ([] if args.batch_only else (args.only or PRECISIONS)):
        esz = {"fp64": 8, "fp32": 4, "bf16": 2, "fp16": 2}[prec]
        tdt = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16,
               "fp16": torch.float16}[prec]
        sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, precision=prec,
                             stream=stream.cuda_stream)
        host_in = torch.from_numpy(w.rho0).to(tdt).pin_memory()
        rho0 = host_in.to(dev)
        sim.set_density(rho0)
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake)
        sim.step(W)
        sim.sync()
        # --- timed region: K graph-launched steps, field resident in HBM ---
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            barrier()
            torch.cuda.synchronize(dev)
            e0.record(stream)
            sim.step(K)
            e1.record(stream)
            e1.synchronize()
            torch.cuda.synchronize(dev)
            barrier()
        ms_max, _ = aggregate(e0.elapsed_time(e1), world, nel, K, dev)
        # --- per-kernel durations over K steps (same stream, CUDA events between launches):
        # the x, y and z kernels as they run inside a renormalisation block, every 8th z the
        # renormalising one (timed apart) ---
        kev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
        for k in range(K):
            _stage_step(sim, kev[k], stream, renorm=(k % 8 == 7))
        stream.synchronize()
        blk = [k for k in range(K) if k % 8 != 7] or list(range(K))
        ren = [k for k in range(K) if k % 8 == 7]
        kms = [sum(kev[k][i].elapsed_time(kev[k][i + 1]) for k in blk) / len(blk)
               for i in range(3)]
        z_renorm = (sum(kev[k][2].elapsed_time(kev[k][3]) for k in ren) / len(ren)) if ren else None
        res = {"ms_total": ms_max, "ms_per_step": ms_max / K,
               "value": world * nel * K / (ms_max * 1e-3), "kernel_ms": kms,
               "z_renorm_ms": z_renorm, "clocks": clk.summary(),
               "launches": sim.launches_per_step() * K, "esz": esz, "prec": prec}
        # --- e2e: host buffers through the C ABI ---
        if rank == 0 and not args.no_e2e:
            host_out = torch.empty(w.shape, dtype=tdt).pin_memory()
            ts = []
            for rep in range(1 + args.e2e_reps):
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                sim.set_density(host_in)
                sim.step(K)
                sim.density(host_out)
                t1 = time.perf_counter()
                if rep > 0:
                    ts.append(t1 - t0)
            t = statistics.median(ts)
            res["e2e"] = {"value": nel * K / t, "unit": UNIT,
                          "h2d_bytes_per_step": nel * esz / K, "d2h_bytes_per_step": nel * esz / K,
                          "seconds_per_job": t,
                          "job": f"set_density(host) + {K} steps + density(host)"}
        # --- error of this leg (rank 0, full workload only) ---
        if rank == 0 and not args.no_error and SHAPE is None:
            n_err = w.n_steps  # 100 steps, the FP32 target's horizon
            sim.set_density(rho0)
            if prec == "fp64":
                sim.step(1)
                one = sim.density()
                res["error"] = {"vs_oracle_1_step_full_size":
                                fp64_vs_oracle_one_step(w, one),
                                "vs_oracle_100_steps_slab": fp64_slab_vs_oracle(stream)}
                sim.set_density(rho0)
                sim.step(n_err)
                ref100 = sim.density()
            else:
                sim.step(n_err)
                got = torch.empty(w.shape, dtype=tdt)
                sim.density(got)
                if ref100 is not None:
                    res["error"] = {f"vs_fp64_gpu_{n_err}_steps":
                                    error_stats(got.double().numpy(), ref100, 1e-6),
                                    "reference": "FP64 GPU path (oracle-validated) from the same "
                                                 "FP64 initial field (the storage rounding of the "
                                                 "initial field included)"}
                del got
        sim.close()
        del rho0, host_in
        torch.cuda.empty_cache()
        results[prec] = res
        barrier()
    del ref100
    full = not args.shape and not args.only and not args.batch_only
    if not args.no_batch and not args.shape and not args.only:
        results["fp32_batched"] = run_batched(args, stream, dev)
    if rank == 0 and full and not args.no_small:
        results["fp64_small"] = run_small(args, stream, dev)
    if rank == 0 and full and not args.no_large:
        results["fp32_large"] = run_large(args, stream, dev)
    if rank == 0 and full and not args.no_paper_e2e:
        results["paper_e2e"] = run_paper_e2e_both(args, stream, dev)
    if rank == 0 and full and not args.no_adjoint:
        results["adjoint"] = run_adjoint_both(dev)
    if world > 1:
        dist.destroy_process_group()
    return rank, world, results


def fp64_vs_oracle_one_step(w, got):
    """One full-size FP64 step against the oracle (OpenMP copy: the same bits, all cores)."""
    import oracle
    t0 = time.perf_counter()
    ref = oracle.Problem(**w.oracle_kwargs(), parallel=True).step(w.rho0, 1)
    out = error_stats(got, ref, 1e-9)
    out["oracle_seconds"] = time.perf_counter() - t0
    return out


def fp64_slab_vs_oracle(stream, steps=100, nz=8):
    """100 FP64 steps of a 400 x 400 x nz slab of the headline recipe against the oracle."""
    import oracle
    from paper_2602_05017_gb300 import binding, inputs
    w = inputs.workload(2, shape=(400, 400, nz), n_agents=1_000_000 * nz // 400)
    sim = binding.BioFVM.from_workload(w, precision="fp64", stream=stream.cuda_stream)
    sim.step(steps)
    got = sim.density()
    sim.close()
    ref = oracle.Problem(**w.oracle_kwargs(), parallel=True).step(w.rho0, steps)
    out = error_stats(got, ref, 1e-9)
    out["sample"] = f"400x400x{nz}x4 slab, {steps} steps, {w.n_agents} agents"
    return out


def run_batched(args, stream, dev):
    """256 uneven FP32 microenvironments, 50 steps per launch, tiles from the autotuner."""
    import torch

    from paper_2602_05017_gb300 import autotune, binding, inputs
    envs = inputs.batched_workloads(n_env=args.batch_envs, with_field=False,
                                    n_steps=args.batch_steps)
    cache_path = autotune.default_cache_path()
    if os.path.exists(cache_path):
        shapes, tuned = autotune.tile_shapes(envs, autotune.load(cache_path)), "autotuner cache"
    else:
        shapes, tuned = None, "library defaults (no autotuner cache)"
    K = args.batch_steps

    def make(mode):
        bb = binding.BioFVMBatch(envs, precision="fp32", tile_m=shapes, stream=stream.cuda_stream,
                                 mode=mode)
        g = torch.Generator(device=dev)
        g.manual_seed(2602050174)
        first = []
        for sim, w in zip(bb.envs, envs):
            with torch.cuda.stream(stream):
                t = sim.field_tensor()
                t.uniform_(0.0, 38.0, generator=g)
                first.append(t.clone())
            sim.set_sources(w.voxel, w.secretion, w.target, w.uptake)
        stream.synchronize()
        return bb, first

    def timed(bb):
        bb.step(args.warmup)
        bb.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev.index or 0) as clk:
            torch.cuda.synchronize(dev)
            e0.record(stream)
            bb.step(K)
            e1.record(stream)
            e1.synchronize()
        bb.sync()
        return e0.elapsed_time(e1), clk.summary()

    # the configuration's design: one persistent graph-captured launch with autotuned tiles;
    # the per-environment graph mode (the library's own choice for environments this large)
    # timed beside it
    bg, _ = make("graph")
    ms_g, clk_g = timed(bg)
    n_launch_g = sum(e.launches_per_step() for e in bg.envs)
    bg.close()
    torch.cuda.empty_cache()
    b, init = make("persistent")
    ms, clk = timed(b)
    n_vs = b.n_vs
    out = {"value": n_vs * K / (ms * 1e-3), "unit": UNIT, "dtype": "f32", "ms_per_step": ms / K,
           "steps": K, "n_env": len(envs), "voxel_substrates": n_vs,
           "mode": "persistent", "launches": 1, "grid": b.grid(), "tiles": tuned,
           "alg_GBps": 24.0 * n_vs * K / (ms * 1e-3) / 1e9, "clocks": clk,
           "per_environment_graphs": {
               "value": n_vs * K / (ms_g * 1e-3), "ms_per_step": ms_g / K,
               "launches": f"{n_launch_g} sweep kernels per step in CUDA graphs of 8 steps",
               "clocks": clk_g, "alg_GBps": 24.0 * n_vs * K / (ms_g * 1e-3) / 1e9,
               "note": "the library's automatic batch mode for environments of >= 2^20 "
                       "voxel-substrates on average"},
           "workload": "256 cubes, edge U{32..192}, 1-8 substrates, D logU[1e2,1e5], "
                       "lambda logU[1e-3,1], agents 1 per 64 voxels, zero-flux"}
    if not args.no_error:
        # every environment from its initial field: K batched steps in one launch against K
        # FP64 steps of the same environment on its own (oracle-validated) FP64 handle
        for sim, t in zip(b.envs, init):
            sim.set_density(t)
        b.step(K)
        b.sync()
        parts = []
        for sim, t, w in zip(b.envs, init, envs):
            got = sim.density()
            ref = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam,
                                 precision="fp64", stream=stream.cuda_stream)
            ref.set_density(t.double())
            ref.set_sources(w.voxel, w.secretion, w.target, w.uptake)
            ref.step(K)
            parts.append(error_stats(got, ref.density(), 1e-6))
            ref.close()
        out["error"] = {f"vs_fp64_gpu_{K}_steps": merge_errors(parts),
                        "reference": "each environment on its own FP64 GPU handle "
                                     "(oracle-validated), same inputs; worst environment"}
    del init
    b.close()
    torch.cuda.empty_cache()
    return out


def _time_job(sim, n_steps, stream, dev, reps, flush):
    """Median CUDA-event time of `reps` jobs of n_steps graph-launched steps (L2 flushed before
    each when the field fits in L2), with the clocks sampled."""
    import torch
    ts = []
    with ClockSampler(dev.index or 0) as clk:
        for _ in range(reps):
            if flush:
                flush_l2(dev)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(n_steps)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), clk.summary()


def run_small(args, stream, dev):
    """Workload 1: 50^3 x 1 FP64, 200 cells, 100 steps per job: the launch-bound case (the
    1 MB field lives in L2; 100 steps are 7 graph launches of at most 16 steps)."""
    import oracle
    from paper_2602_05017_gb300 import binding, inputs
    w = inputs.workload(1)
    sim = binding.BioFVM.from_workload(w, precision="fp64", stream=stream.cuda_stream)
    sim.step(w.n_steps)
    sim.sync()
    ms, clk = _time_job(sim, w.n_steps, stream, dev, reps=20, flush=True)
    out = {"value": w.n_vs * w.n_steps / (ms * 1e-3), "unit": UNIT, "dtype": "f64",
           "ms_per_job": ms, "ms_per_step": ms / w.n_steps, "steps_per_job": w.n_steps,
           "launches_per_step": sim.launches_per_step(), "clocks": clk,
           "l2": "field 1 MB < L2: a 256 MB buffer is written before each timed job",
           "workload": "lod_fp64_50c_s1: 50^3 x 1, D=1e5, lambda=0.1, 200 cells, 100 steps"}
    if not args.no_error:
        sim.set_density(w.rho0)
        sim.step(w.n_steps)
        got = sim.density()
        ref = oracle.Problem(**w.oracle_kwargs()).step(w.rho0, w.n_steps)
        out["error"] = {f"vs_oracle_{w.n_steps}_steps": error_stats(got, ref, 1e-9)}
    sim.close()
    return out


def run_large(args, stream, dev):
    """Workload 3: 1200^3 x 2 FP32 (13.8 GB), Dirichlet 38 on substrate 0, 10M agents, 20 steps;
    the initial field (64 Gaussian blobs) is evaluated on the device."""
    import torch

    from paper_2602_05017_gb300 import binding, inputs
    w = inputs.workload(3, with_field=False)
    field64 = inputs.gaussian_blobs_device(w.extra["blobs"], w.nx, w.ny, w.nz, w.ns, w.dx, dev)
    field32 = field64.float()
    sim = binding.BioFVM.from_workload(w, precision="fp32", stream=stream.cuda_stream)
    sim.set_density(field32)
    sim.step(args.warmup)
    sim.sync()
    ms, clk = _time_job(sim, w.n_steps, stream, dev, reps=3, flush=False)
    out = {"value": w.n_vs * w.n_steps / (ms * 1e-3), "unit": UNIT, "dtype": "f32",
           "ms_per_step": ms / w.n_steps, "steps_per_job": w.n_steps,
           "alg_GBps": 24.0 * w.n_vs * w.n_steps / (ms * 1e-3) / 1e9, "clocks": clk,
           "launches_per_step": sim.launches_per_step(),
           "workload": "lod_fp32_1200c_s2_dirichlet: 1200^3 x 2 (13.8 GB FP32; the stated "
                       "'6.9 GB' would be one substrate), Dirichlet 38 on substrate 0, 64 "
                       "Gaussian blobs, 10M agents, 20 steps"}
    if not args.no_error:
        sim.set_density(field32)
        sim.step(w.n_steps)
        got = torch.empty(w.shape, dtype=torch.float32, device=dev)
        sim.density(got)
        sim.close()
        del field32
        torch.cuda.empty_cache()
        ref = binding.BioFVM.from_workload(w, precision="fp64", stream=stream.cuda_stream)
        ref.set_density(field64)
        del field64
        torch.cuda.empty_cache()
        ref.step(w.n_steps)
        r = ref.field_tensor()
        torch.cuda.synchronize(dev)
        out["error"] = {f"vs_fp64_gpu_{w.n_steps}_steps": device_error_stats(got, r, 1e-6),
                        "reference": "FP64 GPU path (oracle-validated), same inputs",
                        "fp64_vs_oracle_2_steps_slab": large_slab_vs_oracle(stream)}
        ref.close()
        del got, r
    else:
        sim.close()
    torch.cuda.empty_cache()
    return out


def device_error_stats(got, ref, floor_rel):
    """error_stats on device tensors (fields too large to copy to the host twice)."""
    import torch
    m = ref.abs().max().double()
    d_max = torch.zeros((), dtype=torch.float64, device=ref.device)
    pv = torch.zeros((), dtype=torch.float64, device=ref.device)
    g = got.reshape(-1)
    r = ref.reshape(-1)
    chunk = 1 << 28
    for i in range(0, r.numel(), chunk):  # chunked: bounded temporaries
        rr = r[i:i + chunk].double()
        dd = (g[i:i + chunk].double() - rr).abs()
        d_max = torch.maximum(d_max, dd.max())
        big = rr.abs() > floor_rel * m
        if bool(big.any()):
            pv = torch.maximum(pv, (dd[big] / rr[big].abs()).max())
    return {"normwise": float(d_max / torch.clamp(m, min=1e-300)),
            "per_voxel_max_rel": float(pv), "per_voxel_floor": f"|ref| > {floor_rel:g} max|ref|"}


def large_slab_vs_oracle(stream, nz=8, steps=2):
    import oracle
    from paper_2602_05017_gb300 import binding, inputs
    w = inputs.workload(3, shape=(1200, 1200, nz), n_agents=10_000_000 * nz // 1200)
    sim = binding.BioFVM.from_workload(w, precision="fp64", stream=stream.cuda_stream)
    sim.step(steps)
    got = sim.density()
    sim.close()
    ref = oracle.Problem(**w.oracle_kwargs(), parallel=True).step(w.rho0, steps)
    out = error_stats(got, ref, 1e-9)
    out["sample"] = f"1200x1200x{nz}x2 slab of the recipe, {steps} steps, {w.n_agents} agents"
    return out


def run_paper_e2e_both(args, stream, dev):
    out = {p: run_paper_e2e(p, stream, dev) for p in ("fp64", "fp32")}
    for p in ("fp64", "fp32"):
        out[p]["moving_agents"] = run_paper_e2e_moving(p, stream, dev, not args.no_error)
    if not args.no_error:
        import oracle
        from paper_2602_05017_gb300 import binding, inputs
        f64, f32 = out["fp64"].pop("_final"), out["fp32"].pop("_final")
        out["fp32"]["error"] = {"vs_fp64_gpu_500_steps": error_stats(f32, f64, 1e-6)}
        w = inputs.workload(6)
        n = 20
        sim = binding.BioFVM.from_workload(w, precision="fp64", stream=stream.cuda_stream)
        sim.step(n)
        got = sim.density()
        sim.close()
        ref = oracle.Problem(**w.oracle_kwargs(), parallel=True).step(w.rho0, n)
        out["fp64"]["error"] = {f"vs_oracle_first_{n}_steps": error_stats(got, ref, 1e-9)}
    else:
        for p in out.values():
            p.pop("_final", None)
    return out


def run_paper_e2e(prec, stream, dev):
    """The end-to-end run of Sect. 5.3 through the public API, stage by stage (host wall clock,
    stream synchronised after each): create the microenvironment, load the Gaussian initial
    profile from host memory, create the 1000 agents, simulate 500 steps, read the final field
    back to host memory.  File output (the paper's MATLAB files) is not part of the library."""
    import torch

    from paper_2602_05017_gb300 import binding, inputs
    w = inputs.workload(6, field_dtype=np.float64 if prec == "fp64" else np.float32)
    tdt = torch.float64 if prec == "fp64" else torch.float32
    host_in = torch.from_numpy(w.rho0).pin_memory()
    host_out = torch.empty(w.shape, dtype=tdt).pin_memory()
    best = None
    for rep in range(3):  # the first repetition also loads and compiles nothing new: keep best
        torch.cuda.synchronize(dev)
        t = [time.perf_counter()]
        sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, precision=prec,
                             stream=stream.cuda_stream)
        sim.sync()
        t.append(time.perf_counter())
        sim.set_density(host_in)
        sim.sync()
        t.append(time.perf_counter())
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake)
        sim.sync()
        t.append(time.perf_counter())
        sim.step(w.n_steps)
        sim.sync()
        t.append(time.perf_counter())
        sim.density(host_out)
        t.append(time.perf_counter())
        sim.close()
        st = [t[i + 1] - t[i] for i in range(5)]
        if best is None or sum(st) < sum(best):
            best = st
    total = sum(best)
    return {"seconds": total, "unit": "s (time to solution)", "dtype": prec.replace("fp", "f"),
            "stages_s": dict(zip(("create", "initial_field", "agents", "simulate", "final_read"),
                                 best)),
            "simulate_vs_per_s": w.n_vs * w.n_steps / best[3],
            "workload": "Sect. 5.3 end-to-end run: 5 mm cube = 250^3 voxels x 1 substrate, "
                        "1000 agents (500 sources, 500 sinks), 500 steps, Gaussian profile",
            "_final": host_out.numpy().copy()}


def _walk(x, y, z, shape, gen):
    """One random-walk move per agent: one voxel along a random axis, clamped to the box
    (the agents' motion is an input of the step, drawn on the device)."""
    import torch
    nx, ny, nz = shape
    ax = torch.randint(0, 3, x.shape, generator=gen, device=x.device)
    d = torch.randint(0, 2, x.shape, generator=gen, device=x.device) * 2 - 1
    x = (x + d * (ax == 0)).clamp_(0, nx - 1)
    y = (y + d * (ax == 1)).clamp_(0, ny - 1)
    z = (z + d * (ax == 2)).clamp_(0, nz - 1)
    return x, y, z, (z * ny + y) * nx + x


def run_paper_e2e_moving(prec, stream, dev, with_error):
    """The Sect. 5.3 run with its 1000 agents moving every step (a random walk drawn on the
    device): before each of the 500 steps the source lists are rebuilt on the device from the
    agents' new voxels (biofvm_set_sources_device), then one step; field resident in HBM,
    CUDA events around the 500 steps."""
    import torch

    from paper_2602_05017_gb300 import binding, inputs
    w = inputs.workload(6, field_dtype=np.float64 if prec == "fp64" else np.float32)
    sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, precision=prec,
                         stream=stream.cuda_stream)
    sim.reserve_agents(w.n_agents)
    sec, tgt, upt = (torch.as_tensor(a, device=dev) for a in (w.secretion, w.target, w.uptake))
    v0 = torch.as_tensor(w.voxel, device=dev)
    x0, y0, z0 = v0 % w.nx, (v0 // w.nx) % w.ny, v0 // (w.nx * w.ny)

    def run(n_steps, seed, record=False):
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed)
        x, y, z = x0.clone(), y0.clone(), z0.clone()
        lists = []
        with torch.cuda.stream(stream):
            sim.set_density(torch.as_tensor(w.rho0, device=dev))
            for _ in range(n_steps):
                x, y, z, vox = _walk(x, y, z, (w.nx, w.ny, w.nz), gen)
                if record:
                    lists.append(vox.cpu().numpy())
                sim.set_sources_device(vox, sec, tgt, upt)
                sim.step(1)
        return lists

    run(5, 1)  # warm-up: graphs, buffers
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run(w.n_steps, 2602050176)
    e1.record(stream)
    e1.synchronize()
    sim.sync()
    ms = e0.elapsed_time(e1)
    out = {"simulate_vs_per_s": w.n_vs * w.n_steps / (ms * 1e-3), "simulate_ms": ms,
           "launches_per_step": "source-list rebuild (2 kernels up to 2048 agent entries, "
                                "about 30 above) + "
                                f"{sim.launches_per_step()} sweep kernels, plus the torch "
                                "kernels that draw the moves",
           "agents": "random walk, one voxel per step along a random axis, drawn on the device"}
    if with_error:
        import oracle
        n = 10
        lists = run(n, 7, record=True)
        got = sim.density()
        ref = w.rho0.astype(np.float64)
        for vox in lists:
            w.voxel = vox
            ref = oracle.Problem(**w.oracle_kwargs(), parallel=True).step(ref, 1)
        out["error"] = {f"vs_oracle_first_{n}_steps_same_moves":
                        error_stats(got, ref, 1e-9 if prec == "fp64" else 1e-6)}
    sim.close()
    return out


def run_adjoint_both(dev):
    out = {}
    grads = {}
    for p in ("fp64", "fp32"):
        out[p], grads[p] = run_adjoint(p, dev)
    g64, g32 = grads["fp64"], grads["fp32"]
    out["fp32"]["error"] = {
        "vs_fp64_gpu": {k: error_stats(g32[k], g64[k], 1e-6) for k in g64},
        "reference": "FP64 GPU gradients (adjoint checked against the CPU adjoint at 1e-10 and "
                     "FD at 1e-6 in the tests), same inputs"}
    return out


def run_adjoint(prec, dev):
    """Workload 5 (128^3 x 2, 200 steps, checkpoints every 20): the forward run alone, then the
    forward run plus the gradients of a probe loss with respect to the initial field, the
    per-voxel secretion and uptake rates, D and lambda (LODSteps: checkpoints, recomputation
    with biofvm_step_save, biofvm_adjoint_step_rates), timed on the host with the device
    synchronised."""
    import torch

    from paper_2602_05017_gb300 import binding, inputs
    from paper_2602_05017_gb300.adjoint import lod_steps
    w = inputs.workload(5)
    n, K = w.n_steps, w.extra["checkpoint_every"]
    fdt = torch.float64 if prec == "fp64" else torch.float32
    sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, precision=prec)
    agents = dict(voxel=w.voxel, target=w.target, weight=w.weight)
    pr = torch.as_tensor(w.extra["probe_index"], device=dev)
    tg = torch.as_tensor(w.extra["probe_target"], device=dev)
    grads = {}

    def run(steps, backward):
        rho0 = torch.tensor(w.rho0, dtype=torch.float64, device=dev, requires_grad=True)
        sec = torch.tensor(w.secretion, dtype=torch.float64, device=dev, requires_grad=True)
        D = torch.tensor(w.D, dtype=torch.float64, device=dev, requires_grad=True)
        lam = torch.tensor(w.lam, dtype=torch.float64, device=dev, requires_grad=True)
        upt = torch.tensor(w.uptake, dtype=torch.float64, device=dev, requires_grad=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = lod_steps(rho0.to(fdt), sec, D, lam, sim, agents, steps, K, uptake=upt)
        loss = ((out.reshape(-1).double()[pr] - tg) ** 2).sum()
        if backward:
            loss.backward()
        torch.cuda.synchronize(dev)
        t = time.perf_counter() - t0
        if backward and steps == n:
            for k, v in (("rho0", rho0), ("secretion", sec), ("uptake", upt), ("D", D),
                         ("lambda", lam)):
                grads[k] = v.grad.detach().cpu().numpy()
        return t

    run(K, True)  # warm-up: graphs, buffers
    t_fwd = min(run(n, False) for _ in range(2))
    t_all = min(run(n, True) for _ in range(2))
    sim.close()
    return ({"seconds_forward": t_fwd, "seconds_forward_and_gradients": t_all,
             "forward_vs_per_s": w.n_vs * n / t_fwd,
             "gradient_vs_per_s": w.n_vs * n / (t_all - t_fwd),
             "dtype": prec.replace("fp", "f"),
             "workload": "128^3 x 2, 200 steps, checkpoints every 20, 4096-probe loss; gradients "
                         "w.r.t. initial field, secretion and uptake rates, D, lambda"}, grads)


def _stage_step(sim, ev, stream, renorm):
    """One step as the three kernels biofvm_step launches, with an event between launches: the
    z-sweep of a step inside a renormalisation block (stage 12, FP64 leaves the field scaled)
    or of a renormalising step (stage 11)."""
    ev[0].record(stream)
    sim.run_stage(9)
    ev[1].record(stream)
    sim.run_stage(10)
    ev[2].record(stream)
    sim.run_stage(11 if renorm else 12)
    ev[3].record(stream)


def host_description():
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_count": os.cpu_count(), "lscpu_model": model, "machine": platform.machine()}


def _oracle_rate(p, w, seconds):
    p.step(w.rho0, 1)  # warm
    ts = []
    t_end = time.time() + seconds
    while time.time() < t_end or not ts:
        t0 = time.perf_counter()
        p.step(w.rho0, 1)
        ts.append(time.perf_counter() - t0)
    return w.n_vs / statistics.median(ts), ts


def cpu_baseline(args, sample_nz=8):
    """The FP64 oracle on a slab of the workload (400 x 400 x sample_nz x 4): single-threaded
    (the parity oracle), and its OpenMP copy on every host core (the paper-style CPU rate)."""
    import oracle
    from paper_2602_05017_gb300 import inputs
    w = inputs.workload(2, shape=(400, 400, sample_nz), n_agents=1_000_000 * sample_nz // 400)
    v1, ts1 = _oracle_rate(oracle.Problem(**w.oracle_kwargs()), w, args.cpu_seconds)
    host = host_description()
    out = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"one LOD step of a 400x400x{sample_nz}x4 slab of the workload (FP64, "
                     f"{len(ts1)} repetitions, median {w.n_vs / v1:.3f} s)", "host": host}
    vp, tsp = _oracle_rate(oracle.Problem(**w.oracle_kwargs(), parallel=True), w,
                           args.cpu_seconds / 3)
    out["openmp_all_cores"] = {"value": vp, "unit": UNIT, "cores": host["cpu_count"],
                               "kind": "oracle, OpenMP copy (line-parallel sweeps)",
                               "sample": f"same slab, {len(tsp)} repetitions"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2602_05017_gb300 import inputs
    oracle.build()
    nz = 8
    w = inputs.workload(2, shape=(400, 400, nz), n_agents=1_000_000 * nz // 400)
    p = oracle.Problem(**w.oracle_kwargs())
    rho = w.rho0
    for _ in range(args.warmup):
        rho = p.step(rho, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rho = p.step(rho, 1)
    t = time.perf_counter() - t0
    v = w.n_vs * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"lod_400c_s4 slab 400x400x{nz}x4 (bounded CPU sample)",
                       "steps_per_sample": 1},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: one LOD step of a 400x400x{nz}x4 slab, FP64"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--e2e-reps", type=int, default=7)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-error", action="store_true", help="skip the error checks of every leg")
    ap.add_argument("--no-small", action="store_true", help="skip the 50^3 x 1 FP64 leg")
    ap.add_argument("--no-large", action="store_true", help="skip the 1200^3 x 2 FP32 leg")
    ap.add_argument("--no-paper-e2e", action="store_true",
                    help="skip the Sect. 5.3 end-to-end run (time to solution)")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint run (workload 5: forward and gradients)")
    ap.add_argument("--batch-envs", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched leg (profiling only; not a bench line)")
    ap.add_argument("--shape", type=int, nargs=3, metavar=("NX", "NY", "NZ"),
                    help="smaller grid of the same recipe (profiling only; not a bench line)")
    ap.add_argument("--subs", type=int, default=None,
                    help="with --shape: the recipe's first N substrates (profiling only)")
    ap.add_argument("--only", nargs="+", choices=list(PRECISIONS),
                    help="run only these precisions (profiling only; not a bench line)")
    args = ap.parse_args()
    global SHAPE, SUBS
    SHAPE = tuple(args.shape) if args.shape else None
    SUBS = args.subs if args.shape else None
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    rank, world, res = run_gpu(args)
    if rank != 0:
        return 0
    if args.only or args.shape or args.batch_only:  # profiling run: numbers only
        print(json.dumps({"profiling_run": True, "shape": SHAPE, "results": res}), flush=True)
        return 0
    peaks, src = measured_peaks()
    w = workload_config(with_field=False)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic"}
    r64 = res["fp64"]
    line["value"] = r64["value"]
    line["ms_per_step"] = r64["ms_per_step"]
    line["config"] = {"workload": "lod_400c_s4: 400x400x400 voxels x 4 substrates, 1M agents, "
                                  "dx=20um, dt=0.01min, zero-flux",
                      "global_batch": world, "parallelism": f"replicas x{world}",
                      "l2": "field 2.05 GB (FP64) / 1.02 GB (FP32) > 129 MB L2: no flush needed"}
    line["gpu_launches"] = r64["launches"]
    line["clocks"] = r64["clocks"]
    line["e2e"] = r64.get("e2e")
    line["error"] = r64.get("error")
    fma = res["fma_rate"]
    line["roofline"] = roofline(r64, w, peaks, src, fma)
    for p, dt in (("fp32", "f32"), ("bf16", "bf16 storage, f32 arithmetic"),
                  ("fp16", "f16 storage, f32 arithmetic")):
        r = res[p]
        line[p] = {"value": r["value"], "ms_per_step": r["ms_per_step"], "dtype": dt,
                   "roofline": roofline(r, w, peaks, src, fma), "e2e": r.get("e2e"),
                   "clocks": r["clocks"], "error": r.get("error"),
                   "kernel_ms": dict(zip(("x", "y", "z"), r["kernel_ms"])),
                   "vs_fp64": r["value"] / r64["value"]}
    if "fp32_batched" in res:
        bt = dict(res["fp32_batched"])
        bt["vs_fp64"] = bt["value"] / r64["value"]
        if "per_environment_graphs" in bt:
            bt["per_environment_graphs"] = dict(bt["per_environment_graphs"])
            bt["per_environment_graphs"]["vs_fp64"] = (bt["per_environment_graphs"]["value"] /
                                                       r64["value"])
        line["fp32_batched"] = bt
    for k in ("fp64_small", "fp32_large", "paper_e2e", "adjoint"):
        if k in res:
            line[k] = res[k]
    line["kernel_ms"] = {"fp64": dict(zip(("x", "y", "z"), r64["kernel_ms"])),
                         "fp32": dict(zip(("x", "y", "z"), res["fp32"]["kernel_ms"]))}
    line["fma_rate_measured"] = {"fp64_fma_per_s": fma["fp64"], "fp32_fma_per_s": fma["fp32"],
                                 "how": "biofvm_probe_fma_rate: independent FMA chains, 32 warps "
                                        "per SM, best of 3 CUDA-event timings, this run"}
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)
    return 0


def roofline(r, w, peaks, src, fma):
    """Roofline of the dominant (longest) sweep kernel.  FP32: HBM-bound, algorithmic bytes =
    one read + one write of the field.  FP64: bound by the FP64 pipe, algorithmic flops =
    Eq. 2's 5 per element, against twice the FP64 FMA rate measured in this run.  traffic:
    ncu-measured DRAM bytes per launch, only while the kernel sources are the ones measured."""
    kms = r["kernel_ms"]
    i = int(np.argmax(kms))
    name = ("x", "y", "z")[i]
    traffic = None
    if SHAPE is None and MEASURED_TRAFFIC["sources_sha256"] == kernel_sources_sha256():
        traffic = MEASURED_TRAFFIC["bytes"].get(f"{r['prec']}:{name}-sweep")
    dram = None if traffic is None else traffic / (kms[i] * 1e-3) / 1e9
    alg_gbps = 2 * r["esz"] * w.n_vs / (kms[i] * 1e-3) / 1e9
    hbm_peak = float(peaks["hbm_gbs"])
    if r["esz"] == 8:
        peak = 2.0 * fma["fp64"] / 1e12
        achieved = FLOPS_PER_ELEMENT_SWEEP * w.n_vs / (kms[i] * 1e-3) / 1e12
        return {"bound": "alu", "kernel": f"{name}-sweep", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": "measured in this run: 2 x FP64 FMA/s of biofvm_probe_fma_rate",
                "hbm": {"achieved_alg_GBps": alg_gbps, "peak": hbm_peak,
                        "frac": alg_gbps / hbm_peak,
                        "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})"},
                "dram_GBps_measured_traffic": dram}
    return {"bound": "hbm", "kernel": f"{name}-sweep", "achieved": alg_gbps, "peak": hbm_peak,
            "unit": "GB/s", "frac": alg_gbps / hbm_peak, "traffic": traffic,
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})",
            "dram_GBps_measured_traffic": dram}


if __name__ == "__main__":
    sys.exit(main())
