"""Autotuner for the tile shapes of the batched persistent step.

The tunable shape of an environment is, per axis, either the chunk length m of the
partitioned Thomas solve (a line of n voxels cut into ceil(n/m) chunks, one warp each, at most
8, chunks of at most 48 in shared memory, carries across the CTA's warps) or the whole line
(m >= n: each warp streams 32 whole lines, no carries, the forward intermediate through L2).
It sets the warps per tile, the length of the serial recurrences and the memory traffic pattern.
For each class (edge-length bucket, substrate count) the tuner builds a batch of identical
environments large enough to fill the GPU, times the candidates with CUDA events (y/z first,
then x), and records the fastest in a JSON cache (WHOLE = -1 for whole lines).
``tile_shapes`` maps any list of environments to per-environment tile shapes from that cache.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import inputs

N_BUCKETS = (32, 64, 96, 128, 160, 192)
MAX_CHUNKS = 8     # warps of the batched CTA
MAX_CHUNK = 32     # longest chunk offered (the batched kernel allows 48; 32 keeps 3 CTAs per SM)
WHOLE = -1         # cache marker: whole lines


def candidates(n, S=None):
    """Tile shapes for an axis of n voxels: valid chunk lengths m < n (at most MAX_CHUNKS chunks
    of at most MAX_CHUNK; for the x axis, given S, also at most 32/S chunks so that a row's
    lines fit one warp), then n itself (whole lines)."""
    lo = max(4, math.ceil(n / MAX_CHUNKS))
    if S is not None:
        lo = max(lo, math.ceil(n / max(1, 32 // S)))
    out = sorted({min(c, MAX_CHUNK) for c in (lo, math.ceil(1.5 * lo), 2 * lo, 3 * lo)})
    return [c for c in out if lo <= c < n] + [n]


def _bucket(n):
    return min(N_BUCKETS, key=lambda b: (abs(b - n), b))


def _rate(torch, b, steps, reps):
    b.step(1)
    b.sync()
    best = float("inf")
    st = torch.cuda.current_stream()
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        b.step(steps)
        e1.record(st)
        b.sync()
        best = min(best, e0.elapsed_time(e1) / steps)
    return b.n_vs / (best * 1e-3)


def tune(precision="fp32", n_buckets=N_BUCKETS, subs=range(1, 9), target_vs=1.2e8, steps=3,
         reps=3, path=None, log=None):
    """Time the candidates of every class; returns and (if path) writes the cache."""
    import torch

    from . import binding
    cache = {"version": 1, "precision": precision, "device": torch.cuda.get_device_name(),
             "when": time.strftime("%Y-%m-%dT%H:%M:%S"), "classes": {}}
    for n in n_buckets:
        for S in subs:
            k = max(1, min(16, int(target_vs // (n ** 3 * S))))
            envs = [inputs.Workload(f"tune{n}_{S}", n, n, n, S, 20.0, 0.01, np.full(S, 1e4),
                                    np.full(S, 0.1), 1) for _ in range(k)]
            cands = candidates(n)
            cands_x = candidates(n, S)
            m_x = cands_x[0]
            # the tiles being tuned are the persistent kernel's
            b = binding.BioFVMBatch(envs, precision=precision,
                                    tile_m=[[m_x, cands[0], cands[0]]] * k, mode="persistent")
            try:
                for e in b.envs:
                    e.field_tensor().uniform_(0.0, 38.0)
                torch.cuda.synchronize()
                best_yz, best_rate = cands[0], -1.0
                for myz in cands:
                    b.set_tiles([[m_x, myz, myz]] * k)
                    rate = _rate(torch, b, steps, reps)
                    if rate > best_rate:
                        best_yz, best_rate = myz, rate
                best_x = m_x
                for mx in cands_x[1:]:
                    b.set_tiles([[mx, best_yz, best_yz]] * k)
                    rate = _rate(torch, b, steps, reps)
                    if rate > best_rate:
                        best_x, best_rate = mx, rate
            finally:
                b.close()
            m = [WHOLE if c >= n else c for c in (best_x, best_yz, best_yz)]
            cache["classes"][f"{n},{S}"] = {"m": m, "vs_per_s": best_rate, "envs": k}
            if log:
                log(f"tune n={n} S={S}: m={m} {best_rate:.3e} vs/s")
    if path:
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return cache


def load(path):
    with open(path) as f:
        return json.load(f)


def tile_shapes(envs, cache):
    """Per-environment [m_x, m_y, m_z] from a cache (nearest class), kept valid for each axis:
    WHOLE becomes the environment's own axis length, a chunk length is raised to the fewest
    chunks allowed and lowered to MAX_CHUNK (0: library default)."""
    out = []
    for w in envs:
        entry = cache["classes"].get(f"{_bucket(max(w.nx, w.ny, w.nz))},{min(max(w.ns, 1), 8)}")
        m = entry["m"] if entry else [0, 0, 0]
        row = []
        for a, (mm, n) in enumerate(zip(m, (w.nx, w.ny, w.nz))):
            if mm == WHOLE:
                row.append(int(n))
                continue
            lo = math.ceil(n / MAX_CHUNKS)
            if a == 0:
                lo = max(lo, math.ceil(n / max(1, 32 // w.ns)))
            row.append(int(min(MAX_CHUNK, max(mm, lo, 1))) if mm > 0 else 0)
        out.append(row)
    return out


def default_cache_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")
