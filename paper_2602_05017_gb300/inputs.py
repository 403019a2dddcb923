"""Seeded synthetic workloads shaped like the paper's benchmark cubes (Sect. 4.3, Table 1).

This module only draws inputs: grids, parameters, initial fields, agents, probes.  It holds
none of the method's arithmetic, imports neither the CUDA library nor the oracle, and is the
one module both sides of every parity test share.

The paper's workloads are cubic microenvironments of a given side and substrate count; no
public dataset is involved.  The five workloads below keep the paper's dx-scale resolution and
substrate counts but are sized for one GPU (the 4% liver cube, 500^3 x 2, lies between the
second and the third).  Random draws use NumPy's PCG64 (``numpy.random.default_rng``) with
seed 2602050170 + k for workload k.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 2602050170
TARGET_DENSITY = 38.0


@dataclass
class Workload:
    """One microenvironment: grid, parameters, boundary, initial field and agents (FP64 host)."""
    name: str
    nx: int
    ny: int
    nz: int
    ns: int
    dx: float
    dt: float
    D: np.ndarray
    lam: np.ndarray
    n_steps: int
    rho0: Optional[np.ndarray] = None            # [nz, ny, nx, ns]
    dirichlet_on: Optional[np.ndarray] = None     # [ns] uint8, None => all zero-flux
    dirichlet_value: Optional[np.ndarray] = None  # [ns]
    voxel: Optional[np.ndarray] = None            # [n_agents] int64, index (z*ny + y)*nx + x
    secretion: Optional[np.ndarray] = None        # [n_agents, ns]
    target: Optional[np.ndarray] = None           # [n_agents, ns]
    uptake: Optional[np.ndarray] = None           # [n_agents, ns]
    weight: Optional[np.ndarray] = None           # [n_agents] or None (=> 1)
    spacing: Optional[tuple] = None               # (dx, dy, dz) of an anisotropic grid, or None
    dirichlet_nodes: Optional[tuple] = None       # (voxel, substrate, value) arrays, or None
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx, self.ns)

    @property
    def n_vs(self):
        """Voxel-substrate count (the unit of the throughput metric)."""
        return self.nx * self.ny * self.nz * self.ns

    @property
    def n_agents(self):
        return 0 if self.voxel is None else int(self.voxel.size)

    def oracle_kwargs(self):
        return dict(nx=self.nx, ny=self.ny, nz=self.nz, ns=self.ns,
                    dx=self.dx if self.spacing is None else self.spacing, dt=self.dt,
                    D=self.D, lam=self.lam, dirichlet_on=self.dirichlet_on,
                    dirichlet_value=self.dirichlet_value, voxel=self.voxel,
                    secretion=self.secretion, target=self.target, uptake=self.uptake,
                    weight=self.weight, dirichlet_nodes=self.dirichlet_nodes)


def first_substrates(w: Workload, ns: int) -> Workload:
    """The same workload with its first `ns` substrates only (parameters, initial field, agent
    rate columns, Dirichlet flags): e.g. the 400^3 recipe at one substrate for profiling."""
    ns = int(ns)
    if not 1 <= ns <= w.ns:
        raise ValueError(f"ns must be in [1, {w.ns}]")
    cut = lambda a: None if a is None else np.ascontiguousarray(np.asarray(a)[..., :ns])
    return Workload(f"{w.name}_s{ns}", w.nx, w.ny, w.nz, ns, w.dx, w.dt, w.D[:ns].copy(),
                    w.lam[:ns].copy(), w.n_steps, rho0=cut(w.rho0),
                    dirichlet_on=None if w.dirichlet_on is None else w.dirichlet_on[:ns].copy(),
                    dirichlet_value=None if w.dirichlet_value is None else w.dirichlet_value[:ns].copy(),
                    voxel=w.voxel, secretion=cut(w.secretion), target=cut(w.target),
                    uptake=cut(w.uptake), weight=w.weight, spacing=w.spacing)


def _loguniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=size))


def random_agents(rng, nvox, ns, n_agents, kind="mixed", rate=(1e-3, 10.0)):
    """Agents at seeded random voxels (repeats allowed).

    kind="mixed": each agent is a source (secretion ~ logU[rate], uptake 0) or a sink
    (uptake ~ logU[rate], secretion 0) with probability 1/2, per substrate; target 38.
    """
    voxel = rng.integers(0, nvox, size=n_agents, dtype=np.int64)
    rates = _loguniform(rng, rate[0], rate[1], (n_agents, ns))
    is_src = rng.random((n_agents, ns)) < 0.5
    sec = np.where(is_src, rates, 0.0)
    upt = np.where(is_src, 0.0, rates)
    tgt = np.full((n_agents, ns), TARGET_DENSITY)
    return voxel, sec, tgt, upt


def blob_params(rng, nx, ny, nz, ns, dx, n_blobs=64, sigma=(100.0, 400.0), amp=(0.0, 38.0)):
    """Seeded Gaussian blobs: centres uniform in the box (um), sigma (um), amplitude per
    substrate.  Returns (cx, cy, cz, sigma, amp[n_blobs, ns])."""
    cx = rng.uniform(0, nx * dx, n_blobs)
    cy = rng.uniform(0, ny * dx, n_blobs)
    cz = rng.uniform(0, nz * dx, n_blobs)
    sg = rng.uniform(sigma[0], sigma[1], n_blobs)
    am = rng.uniform(amp[0], amp[1], (n_blobs, ns))
    return cx, cy, cz, sg, am


def _blob_support(g):
    k = np.nonzero(g > 1e-30)[0]  # only planes/rows where the blob is above 1e-30 of its peak
    return (k[0], k[-1] + 1) if k.size else None


def gaussian_blobs(rng, nx, ny, nz, ns, dx, n_blobs=64, sigma=(100.0, 400.0), amp=(0.0, 38.0),
                   dtype=np.float64, params=None):
    """Sum of seeded Gaussian blobs (centres uniform in the box, sigma in um, amplitude), voxel
    centres at (i + 1/2) dx: [nz, ny, nx, ns] on the host."""
    cx, cy, cz, sg, am = params or blob_params(rng, nx, ny, nz, ns, dx, n_blobs, sigma, amp)
    out = np.zeros((nz, ny, nx, ns), dtype=dtype)
    xs = (np.arange(nx) + 0.5) * dx
    ys = (np.arange(ny) + 0.5) * dx
    zs = (np.arange(nz) + 0.5) * dx
    for b in range(len(cx)):
        gx = np.exp(-0.5 * ((xs - cx[b]) / sg[b]) ** 2)
        gy = np.exp(-0.5 * ((ys - cy[b]) / sg[b]) ** 2)
        gz = np.exp(-0.5 * ((zs - cz[b]) / sg[b]) ** 2)
        sz, sy = _blob_support(gz), _blob_support(gy)
        if sz is None or sy is None:
            continue
        (z0, z1), (y0, y1) = sz, sy
        plane = (gy[y0:y1, None] * gx[None, :])  # [y, x]
        for z in range(z0, z1):
            w = gz[z] * plane
            out[z, y0:y1, :, :] += (w[:, :, None] * am[b][None, None, :]).astype(dtype)
    return out


def gaussian_blobs_device(params, nx, ny, nz, ns, dx, device, dtype=None):
    """The same blob sum evaluated with torch on `device` (for fields too large to draw on the
    host, e.g. 1200^3 x 2): the separable factors are formed on the host in FP64 exactly as
    ``gaussian_blobs`` forms them, and the products are accumulated on the device in FP64, so
    the two agree to rounding of the accumulation order."""
    import torch
    dtype = dtype or torch.float64
    cx, cy, cz, sg, am = params
    out = torch.zeros((nz, ny, nx, ns), dtype=torch.float64, device=device)
    xs = (np.arange(nx) + 0.5) * dx
    ys = (np.arange(ny) + 0.5) * dx
    zs = (np.arange(nz) + 0.5) * dx
    for b in range(len(cx)):
        gx = np.exp(-0.5 * ((xs - cx[b]) / sg[b]) ** 2)
        gy = np.exp(-0.5 * ((ys - cy[b]) / sg[b]) ** 2)
        gz = np.exp(-0.5 * ((zs - cz[b]) / sg[b]) ** 2)
        sz, sy = _blob_support(gz), _blob_support(gy)
        if sz is None or sy is None:
            continue
        (z0, z1), (y0, y1) = sz, sy
        tz = torch.as_tensor(gz[z0:z1], device=device)
        ty = torch.as_tensor(gy[y0:y1], device=device)
        tx = torch.as_tensor(gx, device=device)
        ta = torch.as_tensor(am[b], device=device)
        plane = ty[:, None] * tx[None, :]
        for z in range(z1 - z0):  # one plane at a time bounds the temporaries
            out[z0 + z, y0:y1] += (tz[z] * plane)[:, :, None] * ta[None, None, :]
    return out if dtype == torch.float64 else out.to(dtype)


# --------------------------------------------------------------------------------------------
# The workloads.  `shape` overrides the grid (parity tests at reduced size keep every
# other recipe); `with_field=False` skips the initial field for callers that draw their own.
# --------------------------------------------------------------------------------------------

def workload(k: int, shape=None, n_agents=None, with_field=True, field_dtype=np.float64,
             seed=None) -> Workload:
    rng = np.random.default_rng(SEED_BASE + k if seed is None else seed)
    if k == 1:
        nx, ny, nz = shape or (50, 50, 50)
        w = Workload("lod_fp64_50c_s1", nx, ny, nz, 1, 20.0, 0.01, np.array([1e5]),
                     np.array([0.1]), 100)
        if with_field:
            w.rho0 = rng.uniform(0.0, 38.0, w.shape).astype(field_dtype)
        na = 200 if n_agents is None else n_agents
        w.voxel = rng.integers(0, nx * ny * nz, size=na, dtype=np.int64)
        w.secretion = np.full((na, 1), 10.0)
        w.target = np.full((na, 1), TARGET_DENSITY)
        w.uptake = np.full((na, 1), 1.0)
        return w
    if k == 2:
        nx, ny, nz = shape or (400, 400, 400)
        w = Workload("lod_400c_s4", nx, ny, nz, 4, 20.0, 0.01,
                     np.array([1e5, 1e3, 5e2, 1e2]), np.array([0.1, 0.01, 0.4, 1e-3]), 100)
        if with_field:
            w.rho0 = rng.uniform(0.0, 38.0, w.shape).astype(field_dtype)
        na = 1_000_000 if n_agents is None else n_agents
        w.voxel, w.secretion, w.target, w.uptake = random_agents(rng, nx * ny * nz, 4, na)
        return w
    if k == 3:
        nx, ny, nz = shape or (1200, 1200, 1200)
        w = Workload("lod_fp32_1200c_s2_dirichlet", nx, ny, nz, 2, 20.0, 0.01,
                     np.array([1e5, 1e3]), np.array([0.1, 0.01]), 20)
        w.dirichlet_on = np.array([1, 0], dtype=np.uint8)
        w.dirichlet_value = np.array([TARGET_DENSITY, 0.0])
        # blob parameters are always drawn (so the agents do not depend on with_field);
        # gaussian_blobs_device evaluates them on a GPU when the host field is not wanted
        w.extra["blobs"] = blob_params(rng, nx, ny, nz, 2, w.dx)
        if with_field:
            w.rho0 = gaussian_blobs(rng, nx, ny, nz, 2, w.dx, dtype=field_dtype,
                                    params=w.extra["blobs"])
        na = 10_000_000 if n_agents is None else n_agents
        w.voxel, w.secretion, w.target, w.uptake = random_agents(rng, nx * ny * nz, 2, na)
        return w
    if k == 5:
        nx, ny, nz = shape or (128, 128, 128)
        w = Workload("adjoint_128c_s2", nx, ny, nz, 2, 20.0, 0.01, np.array([1e5, 1e3]),
                     np.array([0.1, 0.01]), 200)
        if with_field:
            w.rho0 = rng.uniform(0.0, 38.0, w.shape).astype(field_dtype)
        nvox = nx * ny * nz
        na = max(1, nvox // 100) if n_agents is None else n_agents
        w.voxel = rng.choice(nvox, size=na, replace=False).astype(np.int64)
        w.secretion = _loguniform(rng, 1e-3, 10.0, (na, 2))
        w.target = np.full((na, 2), TARGET_DENSITY)
        w.uptake = np.zeros((na, 2))
        n_probe = min(4096, nvox * 2)
        flat = rng.choice(nvox * 2, size=n_probe, replace=False)
        w.extra["probe_index"] = flat.astype(np.int64)       # flat index into [nz,ny,nx,ns]
        w.extra["probe_target"] = rng.uniform(0.0, 38.0, n_probe)
        w.extra["checkpoint_every"] = 20
        return w
    if k == 6:
        # End-to-end run of Sect. 5.3: a 5 mm cube (250^3 voxels of 20 um), one substrate,
        # 1000 basic agents -- 500 bulk sources, 500 uptake sinks -- at seeded voxels, 500 steps
        # (5 min), a Gaussian initial profile (centred, sigma 1 mm, peak 38).
        nx, ny, nz = shape or (250, 250, 250)
        w = Workload("e2e_5mm_s1", nx, ny, nz, 1, 20.0, 0.01, np.array([1e5]), np.array([0.1]),
                     500)
        if with_field:
            w.rho0 = gaussian_profile(nx, ny, nz, w.dx, 1000.0, TARGET_DENSITY, field_dtype)
        na = 1000 if n_agents is None else n_agents
        w.voxel = rng.integers(0, nx * ny * nz, size=na, dtype=np.int64)
        src = np.arange(na) < na // 2
        w.secretion = np.where(src, 10.0, 0.0)[:, None]
        w.target = np.full((na, 1), TARGET_DENSITY)
        w.uptake = np.where(src, 0.0, 1.0)[:, None]
        return w
    raise ValueError(f"unknown workload {k}")


def gaussian_profile(nx, ny, nz, dx, sigma, peak, dtype=np.float64):
    """A Gaussian centred in the box, voxel centres at (i + 1/2) dx: [nz, ny, nx, 1]."""
    def axis(n):
        c = (np.arange(n) + 0.5) * dx - 0.5 * n * dx
        return np.exp(-0.5 * (c / sigma) ** 2)
    gx, gy, gz = axis(nx), axis(ny), axis(nz)
    return (peak * gz[:, None, None] * gy[None, :, None] * gx[None, None, :])[..., None].astype(dtype)


def batched_workloads(n_env=256, edge=(32, 192), ns=(1, 8), seed=None, n_steps=50,
                      with_field=True, field_dtype=np.float32) -> List[Workload]:
    """Many independent microenvironments of uneven cubic size and substrate count."""
    rng = np.random.default_rng(SEED_BASE + 4 if seed is None else seed)
    envs = []
    for e in range(n_env):
        n = int(rng.integers(edge[0], edge[1] + 1))
        s = int(rng.integers(ns[0], ns[1] + 1))
        D = _loguniform(rng, 1e2, 1e5, s)
        lam = _loguniform(rng, 1e-3, 1.0, s)
        w = Workload(f"env{e}", n, n, n, s, 20.0, 0.01, D, lam, n_steps)
        if with_field:
            w.rho0 = rng.uniform(0.0, 38.0, w.shape).astype(field_dtype)
        na = max(1, (n * n * n) // 64)
        w.voxel, w.secretion, w.target, w.uptake = random_agents(rng, n * n * n, s, na)
        envs.append(w)
    return envs


def random_nodes(rng, nvox, ns, n, repeat=True):
    """Dirichlet nodes: n (voxel, substrate, value) triples at seeded random voxels (interior or
    on faces), values uniform in [0, 38]; with ``repeat`` a few (voxel, substrate) pairs occur
    twice with different values."""
    voxel = rng.integers(0, nvox, size=n, dtype=np.int64)
    sub = rng.integers(0, ns, size=n).astype(np.int32)
    val = rng.uniform(0.0, 38.0, n)
    if repeat and n >= 4:
        k = max(1, n // 8)
        voxel[-k:], sub[-k:] = voxel[:k], sub[:k]
    return voxel, sub, val


def face_value_nodes(nx, ny, nz, values):
    """Per-face Dirichlet values as nodes.  values[f, s] (NaN: no condition) for the faces
    f = x-, x+, y-, y+, z-, z+; listed in that order, so where faces meet (edges, corners) the
    later face's value is the one that stays."""
    values = np.asarray(values, dtype=np.float64)
    ns = values.shape[1]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    vox = ((z * ny + y) * nx + x).reshape(-1)
    on = [x.reshape(-1) == 0, x.reshape(-1) == nx - 1, y.reshape(-1) == 0, y.reshape(-1) == ny - 1,
          z.reshape(-1) == 0, z.reshape(-1) == nz - 1]
    vs, ss, vals = [], [], []
    for f in range(6):
        for s in range(ns):
            if np.isnan(values[f, s]):
                continue
            sel = vox[on[f]]
            vs.append(sel)
            ss.append(np.full(sel.size, s, dtype=np.int32))
            vals.append(np.full(sel.size, values[f, s]))
    if not vs:
        return (np.zeros(0, np.int64), np.zeros(0, np.int32), np.zeros(0))
    return np.concatenate(vs).astype(np.int64), np.concatenate(ss), np.concatenate(vals)


def random_problem(rng, nx, ny, nz, ns, n_agents=0, dirichlet=False, dx=20.0, dt=0.01,
                   D_range=(1e2, 1e5), lam_range=(1e-3, 1.0), n_nodes=0) -> Workload:
    """A small random problem for edge-case parity tests (any shape, optional Dirichlet faces
    and Dirichlet nodes)."""
    D = _loguniform(rng, D_range[0], D_range[1], ns)
    lam = _loguniform(rng, lam_range[0], lam_range[1], ns)
    w = Workload(f"rand_{nx}x{ny}x{nz}_s{ns}", nx, ny, nz, ns, dx, dt, D, lam, 1)
    w.rho0 = rng.uniform(0.0, 38.0, w.shape)
    if dirichlet:
        w.dirichlet_on = (rng.random(ns) < 0.5).astype(np.uint8)
        w.dirichlet_on[0] = 1
        w.dirichlet_value = rng.uniform(0.0, 38.0, ns)
    if n_agents:
        w.voxel, w.secretion, w.target, w.uptake = random_agents(rng, nx * ny * nz, ns, n_agents)
        w.weight = rng.uniform(0.5, 1.5, n_agents)
    if n_nodes:
        w.dirichlet_nodes = random_nodes(rng, nx * ny * nz, ns, n_nodes)
    return w
