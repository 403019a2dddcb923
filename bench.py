"""Benchmark of the LOD diffusion-decay step on GB300 (one JSON line on rank 0).

Workload: 400 x 400 x 400 voxels x 4 substrates interleaved per voxel, dx = 20 um,
dt = 0.01 min, D = {1e5, 1e3, 5e2, 1e2} um^2/min, lambda = {0.1, 0.01, 0.4, 1e-3} /min,
1M agents with log-uniform secretion/uptake rates, initial field uniform in [0, 38] (seeded).
A bench step is one full LOD time step (Src, B, X^-1, B, Y^-1, B, Z^-1, B) of that grid.
The headline runs in FP64 (the paper's precision); the FP32 path is reported beside it.

  value      voxel-substrate updates/s, field resident in HBM, graph-launched steps,
             CUDA events on the library's stream, max over ranks (replicas, weak scaling)
  e2e        the same metric through the C ABI from pinned host buffers: set_density(host),
             K steps, density(host), all inside the timed region
  roofline   dominant kernel: algorithmic bytes (one read + one write of the field per sweep)
             or FP64 operations per launch / its average CUDA-event duration over K steps
  cpu_baseline  the FP64 oracle, single-threaded on this host, on a bounded slab sample

`--impl reference` times the oracle instead (the reference arm), on the same metric.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
# FP64 ALU roof of a GB300: 2 FP64 FMA per clock per SM (0.5 per SM sub-partition, measured
# with an 8-chain FMA probe: 6.28e11 FMA/s) x 152 SMs x 2070 MHz, an FMA counting 2 flops.
FP64_FMA_PER_CLK_PER_SM = 2.0
GB300_SMS = 152
# Floating-point operations of the Thomas algorithm per element and sweep (Sect. 2.1, Eq. 2:
# forward axpy + division, backward negated axpy).
FLOPS_PER_ELEMENT_SWEEP = 5
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel each
# roofline names, from one ncu capture of this bench's 400^3 x 4 workload; valid only for the
# kernel version they were taken on (re-measure whenever that kernel changes).
MEASURED_TRAFFIC = {
    ("f64", "x-sweep"): 2858953728 + 2839952384,   # stream_sweep_kernel<double, 1>, with Src
    ("f64", "y-sweep"): 2693955072 + 2817628160,
    ("f64", "z-sweep"): 2713343488 + 2828182272,   # inside a renormalisation block
    ("f32", "x-sweep"): 1088906752 + 961776896,    # sweep_pipe_kernel<float, 32, 0, 4>, with Src
    ("f32", "y-sweep"): 1024289792 + 960146432,    # sweep_pipe_kernel<float, 32, 1, 0>
    ("f32", "z-sweep"): 1024184576 + 959291392,
}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": HBM_FALLBACK_GBS, "sm_max_mhz": 2070.0}, "fallback"


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


def workload_config():
    from paper_2602_05017_gb300 import inputs
    if SHAPE is None:
        return inputs.workload(2, with_field=False)
    nvox = SHAPE[0] * SHAPE[1] * SHAPE[2]
    return inputs.workload(2, shape=SHAPE, with_field=False, n_agents=nvox // 64)


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

    results = {}
    for prec in ([] if args.batch_only else (args.only or ("fp64", "fp32"))):
        esz = 8 if prec == "fp64" else 4
        tdt = torch.float64 if prec == "fp64" else torch.float32
        sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, precision=prec,
                             stream=stream.cuda_stream)
        g = torch.Generator(device=dev)
        g.manual_seed(2602050172 + rank)
        with torch.cuda.stream(stream):
            rho0 = torch.rand(w.shape, generator=g, device=dev, dtype=tdt) * 38.0
        stream.synchronize()
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
               "launches": sim.launches_per_step() * K, "esz": esz}
        # --- e2e: host buffers through the C ABI ---
        if rank == 0 and not args.no_e2e:
            host_in = torch.empty(w.shape, dtype=tdt).pin_memory()
            host_in.copy_(rho0.cpu())
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
            res["e2e"] = {"value": nel * K / t, "unit": "voxel-substrate updates/s",
                          "h2d_bytes_per_step": nel * esz / K, "d2h_bytes_per_step": nel * esz / K,
                          "seconds_per_job": t,
                          "job": f"set_density(host) + {K} steps + density(host)"}
        sim.close()
        del rho0
        torch.cuda.empty_cache()
        results[prec] = res
        barrier()
    if not args.no_batch and not args.shape and not args.only:
        results["fp32_batched"] = run_batched(args, stream, dev)
    if rank == 0 and not args.no_paper_e2e and not args.shape and not args.only \
            and not args.batch_only:
        results["paper_e2e"] = {p: run_paper_e2e(p, stream, dev) for p in ("fp64", "fp32")}
    if rank == 0 and not args.no_adjoint and not args.shape and not args.only \
            and not args.batch_only:
        results["adjoint"] = {p: run_adjoint(p, dev) for p in ("fp64", "fp32")}
    if world > 1:
        dist.destroy_process_group()
    return rank, world, results


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
    b = binding.BioFVMBatch(envs, precision="fp32", tile_m=shapes, stream=stream.cuda_stream)
    g = torch.Generator(device=dev)
    g.manual_seed(2602050174)
    for sim, w in zip(b.envs, envs):
        with torch.cuda.stream(stream):
            sim.field_tensor().uniform_(0.0, 38.0, generator=g)
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake)
    stream.synchronize()
    b.step(args.warmup)
    b.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    K = args.batch_steps
    with ClockSampler(dev.index or 0) as clk:
        torch.cuda.synchronize(dev)
        e0.record(stream)
        b.step(K)
        e1.record(stream)
        e1.synchronize()
    b.sync()
    ms = e0.elapsed_time(e1)
    n_vs = b.n_vs
    out = {"value": n_vs * K / (ms * 1e-3), "unit": UNIT, "dtype": "f32", "ms_per_step": ms / K,
           "steps": K, "n_env": len(envs), "voxel_substrates": n_vs,
           "launches": 1, "grid": b.grid(), "tiles": tuned,
           "alg_GBps": 24.0 * n_vs * K / (ms * 1e-3) / 1e9, "clocks": clk.summary(),
           "workload": "256 cubes, edge U{32..192}, 1-8 substrates, D logU[1e2,1e5], "
                       "lambda logU[1e-3,1], agents 1 per 64 voxels, zero-flux"}
    b.close()
    torch.cuda.empty_cache()
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
                        "1000 agents (500 sources, 500 sinks), 500 steps, Gaussian profile"}


def run_adjoint(prec, dev):
    """Workload 5 (128^3 x 2, 200 steps, checkpoints every 20): the forward run alone, then the
    forward run plus the gradients of a probe loss with respect to the initial field, the
    per-voxel secretion rates, D and lambda (LODSteps: checkpoints, recomputation with
    biofvm_step_save, biofvm_adjoint_step), timed on the host with the device synchronised."""
    import torch

    from paper_2602_05017_gb300 import binding, inputs
    from paper_2602_05017_gb300.adjoint import lod_steps
    w = inputs.workload(5)
    n, K = w.n_steps, w.extra["checkpoint_every"]
    fdt = torch.float64 if prec == "fp64" else torch.float32
    sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, precision=prec)
    agents = dict(voxel=w.voxel, target=w.target, uptake=w.uptake, weight=w.weight)
    pr = torch.as_tensor(w.extra["probe_index"], device=dev)
    tg = torch.as_tensor(w.extra["probe_target"], device=dev)

    def run(steps, backward):
        rho0 = torch.tensor(w.rho0, dtype=torch.float64, device=dev, requires_grad=True)
        sec = torch.tensor(w.secretion, dtype=torch.float64, device=dev, requires_grad=True)
        D = torch.tensor(w.D, dtype=torch.float64, device=dev, requires_grad=True)
        lam = torch.tensor(w.lam, dtype=torch.float64, device=dev, requires_grad=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = lod_steps(rho0.to(fdt), sec, D, lam, sim, agents, steps, K)
        loss = ((out.reshape(-1).double()[pr] - tg) ** 2).sum()
        if backward:
            loss.backward()
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0

    run(K, True)  # warm-up: graphs, buffers
    t_fwd = min(run(n, False) for _ in range(2))
    t_all = min(run(n, True) for _ in range(2))
    sim.close()
    return {"seconds_forward": t_fwd, "seconds_forward_and_gradients": t_all,
            "forward_vs_per_s": w.n_vs * n / t_fwd,
            "gradient_vs_per_s": w.n_vs * n / (t_all - t_fwd),
            "dtype": prec.replace("fp", "f"),
            "workload": "128^3 x 2, 200 steps, checkpoints every 20, 4096-probe loss; gradients "
                        "w.r.t. initial field, secretion rates, D, lambda"}


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


def cpu_baseline(args, sample_nz=8):
    """The FP64 oracle (single thread) on a slab of the workload: 400 x 400 x sample_nz x 4."""
    import oracle
    from paper_2602_05017_gb300 import inputs
    w = inputs.workload(2, shape=(400, 400, sample_nz), n_agents=1_000_000 * sample_nz // 400)
    p = oracle.Problem(**w.oracle_kwargs())
    p.step(w.rho0, 1)  # warm
    ts = []
    t_end = time.time() + args.cpu_seconds
    while time.time() < t_end or not ts:
        t0 = time.perf_counter()
        p.step(w.rho0, 1)
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    return {"value": w.n_vs / t, "unit": "voxel-substrate updates/s", "cores": 1, "kind": "oracle",
            "sample": f"one LOD step of a 400x400x{sample_nz}x4 slab of the workload (FP64, "
                      f"{len(ts)} repetitions, median {t:.3f} s)"}


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


METRIC = "LOD step voxel-substrate updates/s (HBM GB/s vs peak in roofline)"
UNIT = "voxel-substrate updates/s"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--e2e-reps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
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
    ap.add_argument("--only", nargs="+", choices=["fp64", "fp32"],
                    help="run only these precisions (profiling only; not a bench line)")
    args = ap.parse_args()
    global SHAPE
    SHAPE = tuple(args.shape) if args.shape else None
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
    w = workload_config()
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
    line["roofline"] = roofline(r64, w, peaks, src)
    line["fp32"] = {"value": res["fp32"]["value"], "ms_per_step": res["fp32"]["ms_per_step"],
                    "dtype": "f32", "roofline": roofline(res["fp32"], w, peaks, src),
                    "e2e": res["fp32"].get("e2e"), "clocks": res["fp32"]["clocks"],
                    "vs_fp64": res["fp32"]["value"] / r64["value"]}
    if "fp32_batched" in res:
        bt = dict(res["fp32_batched"])
        bt["vs_fp64"] = bt["value"] / r64["value"]
        line["fp32_batched"] = bt
    line["kernel_ms"] = {"fp64": dict(zip(("x", "y", "z"), r64["kernel_ms"])),
                         "fp32": dict(zip(("x", "y", "z"), res["fp32"]["kernel_ms"]))}
    if "paper_e2e" in res:
        line["paper_e2e"] = res["paper_e2e"]
    if "adjoint" in res:
        line["adjoint"] = res["adjoint"]
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)
    return 0


def roofline(r, w, peaks, src):
    """Roofline of the dominant (longest) sweep kernel.  FP32: HBM-bound, algorithmic bytes =
    one read + one write of the field.  FP64: bound by the FP64 pipe (its DRAM time, measured
    traffic included, stays below its FP64-ALU time), algorithmic flops = Eq. 2's 5 per
    element.  traffic: measured DRAM bytes per launch (full workload only)."""
    kms = r["kernel_ms"]
    i = int(np.argmax(kms))
    name = ("x", "y", "z")[i]
    traffic = None if SHAPE else MEASURED_TRAFFIC.get(("f64" if r["esz"] == 8 else "f32",
                                                       f"{name}-sweep"))
    dram = None if traffic is None else traffic / (kms[i] * 1e-3) / 1e9
    if r["esz"] == 8:
        clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
        peak = 2.0 * FP64_FMA_PER_CLK_PER_SM * GB300_SMS * clk / 1e12
        achieved = FLOPS_PER_ELEMENT_SWEEP * w.n_vs / (kms[i] * 1e-3) / 1e12
        return {"bound": "alu", "kernel": f"{name}-sweep", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": "FP64 FMA rate 2/clk/SM (measured probe) x 152 SMs x sm_max_mhz",
                "hbm_GBps": 2 * r["esz"] * w.n_vs / (kms[i] * 1e-3) / 1e9,
                "dram_GBps_measured_traffic": dram}
    alg_bytes = 2 * r["esz"] * w.n_vs  # one read + one write of the field per sweep
    achieved = alg_bytes / (kms[i] * 1e-3) / 1e9
    peak = float(peaks["hbm_gbs"])
    return {"bound": "hbm", "kernel": f"{name}-sweep", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})",
            "dram_GBps_measured_traffic": dram}


if __name__ == "__main__":
    sys.exit(main())
