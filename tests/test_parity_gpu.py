"""GPU parity of libbiofvm against the FP64 CPU oracle, through the C ABI.

Error measure (normwise): max |rho_gpu - rho_oracle| / max |rho_oracle|.
  FP64 path: <= 1e-12.  Thomas in double has a backward error of a few ulp per line and the
  solves are contractive (diagonally dominant M-matrices), so the forward error of a step stays
  within ~1e-15 relative; 1e-12 leaves room for many steps and chunked reassociation.
  FP32 path: <= 1e-5 after 100 steps (storage and arithmetic in float; constants from double).
At full workload sizes, where the oracle would take hours, parity is checked on one full step
(workload 2) and, over all steps, through closed forms that hold at any size (uniform-field
decay, cosine-mode decay, Dirichlet steady state).
"""
import numpy as np
import pytest

import oracle
from paper_2602_05017_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
# sweep implementations selected at create: BIOFVM_PIPELINE, BIOFVM_STREAM, BIOFVM_STREAM32
PATHS = {"plain": ("0", "0", "0"), "pipe": ("1", "0", "0"), "stream": ("1", "1", "1")}


@pytest.fixture(scope="module")
def binding():
    from paper_2602_05017_gb300 import binding as b
    return b


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def gpu_run(binding, w, prec, n_steps=1, rho=None):
    sim = binding.BioFVM.from_workload(w, precision=prec)
    if rho is not None:
        sim.set_density(rho)
    sim.step(n_steps)
    out = sim.density().astype(np.float64)
    sim.close()
    return out


def orc(w):
    return oracle.Problem(**w.oracle_kwargs())


SHAPES = [
    (37, 23, 19, 3), (1, 9, 7, 2), (8, 1, 5, 1), (6, 5, 1, 4), (1, 1, 1, 1), (2, 2, 2, 5),
    (65, 33, 17, 2), (200, 7, 9, 1), (9, 130, 11, 2), (5, 7, 300, 1), (64, 12, 10, 8),
    (31, 3, 4, 7), (513, 3, 2, 1), (50, 50, 50, 1),
    (1100, 3, 2, 3),  # FP64 x rows too long for register chunks: streaming solve only
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_matches_oracle(binding, shape, prec):
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(hash(shape) % 2**32)
    w = inputs.random_problem(rng, nx, ny, nz, ns, n_agents=max(1, nx * ny * nz // 20),
                              dirichlet=True)
    ref = orc(w).step(w.rho0, 2)
    got = gpu_run(binding, w, prec, 2)
    assert rel_err(got, ref) <= TOL[prec]


@pytest.mark.parametrize("shape", [(37, 23, 19, 3), (1, 9, 7, 2), (200, 7, 9, 1), (9, 70, 130, 2),
                                   (1100, 3, 2, 3)],
                         ids=lambda s: "x".join(map(str, s)))
def test_each_stage_matches_oracle(binding, shape):
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(11)
    w = inputs.random_problem(rng, nx, ny, nz, ns, n_agents=50, dirichlet=True)
    p = orc(w)
    expect = {
        4: lambda u: p.sources(u),
        5: lambda u: p.sweep(0, u),
        6: lambda u: p.sweep(1, u),
        7: lambda u: p.sweep(2, u),
        0: lambda u: p.dirichlet(p.sources(u)),
        1: lambda u: p.dirichlet(p.sweep(0, u)),
        2: lambda u: p.dirichlet(p.sweep(1, u)),
        3: lambda u: p.dirichlet(p.sweep(2, u)),
    }
    for stage, fn in expect.items():
        sim = binding.BioFVM.from_workload(w, precision="fp64")
        sim.run_stage(stage)
        got = sim.density()
        sim.close()
        assert rel_err(got, fn(w.rho0)) <= 1e-13, stage


@pytest.mark.parametrize("shape", [(50, 50, 50, 1), (17, 23, 9, 3), (40, 8, 70, 2), (1, 1, 5, 1),
                                   (12, 12, 1, 2), (7, 1, 30, 4)],
                         ids=lambda s: "x".join(map(str, s)))
def test_small_grid_cooperative_path_matches_oracle(binding, monkeypatch, shape):
    """Small FP64 grids run every step of a call in one cooperative launch (z-planes in shared
    memory, a bounded grid barrier between the plane and z-line phases): against the oracle
    over calls of 2 and 3 steps, and against the per-sweep kernels (BIOFVM_SMALL=0)."""
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(nx * 31 + nz)
    w = inputs.random_problem(rng, nx, ny, nz, ns, n_agents=max(1, nx * ny * nz // 25),
                              dirichlet=True)
    ref = orc(w).step(w.rho0, 5)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    assert sim.launches_per_step() == 1  # the cooperative path
    sim.step(2)
    sim.step(3)
    got = sim.density()
    sim.close()
    assert rel_err(got, ref) <= 1e-12
    monkeypatch.setenv("BIOFVM_SMALL", "0")
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    assert sim.launches_per_step() == 3
    sim.step(5)
    other = sim.density()
    sim.close()
    assert rel_err(got, other) <= 1e-13


@pytest.mark.parametrize("stream", ["0", "1"])
def test_graph_steps_equal_stage_sequence(binding, monkeypatch, stream):
    """Graph-launched steps against the same stages launched one by one.  Without the
    streaming sweep both run the same kernels: bit-identical.  With it, a whole step solves
    for scaled intermediates (x / sigma) while single stages solve for x itself: the two
    differ by rounding only."""
    monkeypatch.setenv("BIOFVM_STREAM", stream)
    rng = np.random.default_rng(3)
    w = inputs.random_problem(rng, 21, 17, 13, 2, n_agents=30, dirichlet=True)
    a = gpu_run(binding, w, "fp64", 3)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    for _ in range(3):
        for stage in (0, 1, 2, 3):
            sim.run_stage(stage)
    b = sim.density()
    sim.close()
    if stream == "0":
        assert np.array_equal(a, b)
    else:
        assert rel_err(a, b) <= 1e-14


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_kernels_one_by_one_equal_step(binding, monkeypatch, prec):
    """Stages 9, 10, 11 (the kernels of biofvm_step, launched one by one) make exactly one
    graph-launched step, bit for bit.  Over several steps the FP64 graph leaves the field scaled
    between steps of a renormalisation block (stage 12: the z-sweep without the multiply), so
    there the sequences agree up to rounding.  (A grid this small would otherwise take the
    cooperative one-launch step in FP64, and its 90-float rows the row-padded copy in FP32;
    both have tests of their own.)"""
    monkeypatch.setenv("BIOFVM_SMALL", "0")
    monkeypatch.setenv("BIOFVM_PITCHED", "0")
    rng = np.random.default_rng(8)
    w = inputs.random_problem(rng, 30, 26, 22, 3, n_agents=50, dirichlet=True)
    for n in (1, 3):
        a = gpu_run(binding, w, prec, n)
        sim = binding.BioFVM.from_workload(w, precision=prec)
        for _ in range(n):
            for stage in (9, 10, 11):
                sim.run_stage(stage)
        b = sim.density()
        sim.close()
        if n == 1 or prec == "fp32":
            assert np.array_equal(a, b), n
        else:
            assert rel_err(a, b) <= 1e-14, n


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paper_e2e_workload_reduced(binding, prec):
    """The Sect. 5.3 end-to-end recipe (Gaussian profile, 500 sources and 500 sinks) at 48^3,
    60 steps, against the oracle."""
    w = inputs.workload(6, shape=(48, 48, 48))
    ref = orc(w).step(w.rho0, 60)
    got = gpu_run(binding, w, prec, 60)
    assert rel_err(got, ref) <= TOL[prec]


@pytest.mark.slow
def test_paper_e2e_workload_full_size_first_steps(binding):
    """The full 5 mm cube (250^3), FP64, 5 steps against the oracle (7.8e7 element updates on
    the CPU), then 500 steps: finite, within the source-free bounds [0, 38]."""
    w = inputs.workload(6)
    ref = orc(w).step(w.rho0, 5)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    sim.step(5)
    assert rel_err(sim.density(), ref) <= 1e-12
    sim.step(495)
    out = sim.density()
    sim.close()
    assert np.isfinite(out).all() and out.min() >= 0.0 and out.max() <= 38.0 * (1 + 1e-12)


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_anisotropic_spacing_matches_oracle(binding, monkeypatch, path, prec):
    """dx != dy != dz (biofvm_set_spacing) on every sweep implementation, with Dirichlet faces
    and sources, over 20 steps (FP64: a renormalisation block and a tail)."""
    if prec == "fp64" and path == "pipe":
        pytest.skip("the pipelined sweep is FP32 only")
    monkeypatch.setenv("BIOFVM_PIPELINE", PATHS[path][0])
    monkeypatch.setenv("BIOFVM_STREAM", PATHS[path][1])
    monkeypatch.setenv("BIOFVM_STREAM32", PATHS[path][2])
    rng = np.random.default_rng(21)
    w = inputs.random_problem(rng, 45, 38, 33, 3, n_agents=90, dirichlet=True)
    w.spacing = (12.0, 20.0, 33.0)
    ref = orc(w).step(w.rho0, 20)
    got = gpu_run(binding, w, prec, 20)
    assert rel_err(got, ref) <= TOL[prec]


def test_set_spacing_rejects_bad_values_and_changes_nothing(binding):
    rng = np.random.default_rng(22)
    w = inputs.random_problem(rng, 10, 9, 8, 2)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    for bad in ((0.0, 1.0, 1.0), (1.0, -2.0, 1.0), (1.0, 1.0, float("nan"))):
        with pytest.raises(binding.BioFVMError):
            sim.set_spacing(*bad)
    sim.step(2)
    got = sim.density()
    sim.close()
    assert rel_err(got, orc(w).step(w.rho0, 2)) <= 1e-12


def test_renormalisation_blocks_and_tails_match_oracle(binding):
    """FP64 steps in renormalisation blocks: 1, 15, 16, 17 and 35 steps (tails, one block, a
    block and a tail, two blocks and a tail) against the oracle, with Dirichlet faces and
    sources, and two calls in a row (each call ends with the true field)."""
    rng = np.random.default_rng(9)
    w = inputs.random_problem(rng, 24, 21, 19, 3, n_agents=80, dirichlet=True)
    w.D = np.array([1e5, 1e3, 1e2])
    w.lam = np.array([0.1, 0.01, 1e-3])
    p = orc(w)
    for n in (1, 15, 16, 17, 35):
        sim = binding.BioFVM.from_workload(w, precision="fp64")
        sim.step(n)
        got = sim.density()
        sim.step(2)
        got2 = sim.density()
        sim.close()
        ref = p.step(w.rho0, n)
        assert rel_err(got, ref) <= 1e-12, n
        assert rel_err(got2, p.step(ref, 2)) <= 1e-12, n


def test_sources_can_be_replaced_and_cleared(binding):
    rng = np.random.default_rng(4)
    w = inputs.random_problem(rng, 12, 11, 10, 2, n_agents=40)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    sim.set_sources([])  # no agents
    sim.step(2)
    got = sim.density()
    sim.close()
    w2 = inputs.random_problem(np.random.default_rng(4), 12, 11, 10, 2)
    assert rel_err(got, orc(w2).step(w.rho0, 2)) <= 1e-12


def test_set_params_recomputes_constants(binding):
    rng = np.random.default_rng(5)
    w = inputs.random_problem(rng, 16, 15, 14, 3, n_agents=20)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    w.D = w.D * 3.0
    w.lam = w.lam * 0.5
    sim.set_params(w.D, w.lam)
    sim.step(2)
    got = sim.density()
    sim.close()
    assert rel_err(got, orc(w).step(w.rho0, 2)) <= 1e-12


def test_torch_device_tensors_roundtrip(binding):
    import torch
    rng = np.random.default_rng(6)
    w = inputs.random_problem(rng, 20, 10, 6, 2)
    sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam)
    t = torch.from_numpy(w.rho0).cuda()
    sim.set_density(t)
    sim.step(1)
    out = torch.empty_like(t)
    sim.density(out)
    view = sim.field_tensor()
    assert torch.equal(view, out)
    assert rel_err(out.cpu().numpy(), orc(w).step(w.rho0, 1)) <= 1e-12
    sim.close()


# ------------------------------------------------------------------------------------------------
# The workloads: small one in full, the others at reduced size and (properties) at full size.
# ------------------------------------------------------------------------------------------------

def test_workload1_full_100_steps_fp64(binding):
    w = inputs.workload(1)
    ref = orc(w).step(w.rho0, w.n_steps)
    got = gpu_run(binding, w, "fp64", w.n_steps)
    assert rel_err(got, ref) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_workload2_reduced_100_steps(binding, prec):
    w = inputs.workload(2, shape=(48, 40, 36), n_agents=3000)
    ref = orc(w).step(w.rho0, w.n_steps)
    got = gpu_run(binding, w, prec, w.n_steps)
    assert rel_err(got, ref) <= TOL[prec]


@pytest.mark.slow
def test_workload2_full_size_one_step_fp64(binding):
    """400^3 x 4 with 1M agents: one whole step against the oracle, every element."""
    w = inputs.workload(2)
    ref = orc(w).step(w.rho0, 1)
    got = gpu_run(binding, w, "fp64", 1)
    assert rel_err(got, ref) <= 1e-12


def _cosine_field(shape, k):
    nz, ny, nx, ns = shape
    fx = np.cos(k[0] * np.pi * (np.arange(nx) + 0.5) / nx)
    fy = np.cos(k[1] * np.pi * (np.arange(ny) + 0.5) / ny)
    fz = np.cos(k[2] * np.pi * (np.arange(nz) + 0.5) / nz)
    return fz[:, None, None, None] * fy[None, :, None, None] * fx[None, None, :, None]


def _mode_factor(w, s, k):
    r = w.D[s] * w.dt / w.dx ** 2
    f = 1.0
    for n, kd in zip((w.nx, w.ny, w.nz), k):
        f /= 1.0 + w.lam[s] * w.dt / 3.0 + 2.0 * r * (1.0 - np.cos(kd * np.pi / n))
    return f


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_workload2_full_size_100_steps_cosine_mode(binding, prec):
    """400^3 x 4, 100 steps, no agents: a separable cosine mode decays by the closed form."""
    import torch
    w = inputs.workload(2, with_field=False, n_agents=0)
    w.voxel = None
    k = (3, 1, 7)
    base = _cosine_field(w.shape, k)
    field = np.broadcast_to(38.0 * base, w.shape)
    sim = binding.BioFVM.from_workload(w, precision=prec)
    sim.set_density(torch.from_numpy(np.ascontiguousarray(field)).cuda())
    sim.step(w.n_steps)
    got = sim.field_tensor().double().cpu().numpy()
    sim.close()
    for s in range(w.ns):
        expect = 38.0 * base[..., 0] * _mode_factor(w, s, k) ** w.n_steps
        err = np.abs(got[..., s] - expect).max() / 38.0
        assert err <= TOL[prec], (s, err)


def test_workload3_reduced_20_steps_fp32(binding):
    w = inputs.workload(3, shape=(96, 80, 72), n_agents=20000)
    ref = orc(w).step(w.rho0, w.n_steps)
    got = gpu_run(binding, w, "fp32", w.n_steps)
    assert rel_err(got, ref) <= 1e-5


@pytest.mark.slow
def test_workload3_full_size_20_steps_fp32_properties(binding):
    """1200^3 x 2 FP32 (13.8 GB): substrate 0, uniform at its Dirichlet value 38 with its decay
    switched off, stays 38 (a steady state); substrate 1 (zero flux) carries a cosine mode that
    decays by the closed form."""
    import torch
    w = inputs.workload(3, with_field=False, n_agents=0)
    w.voxel = None
    w.lam = np.array([0.0, w.lam[1]])
    k = (2, 5, 1)
    nz, ny, nx, _ = w.shape
    fx = torch.cos(k[0] * torch.pi * (torch.arange(nx, device="cuda") + 0.5) / nx)
    fy = torch.cos(k[1] * torch.pi * (torch.arange(ny, device="cuda") + 0.5) / ny)
    fz = torch.cos(k[2] * torch.pi * (torch.arange(nz, device="cuda") + 0.5) / nz)
    sim = binding.BioFVM.from_workload(w, precision="fp32")
    f = sim.field_tensor()
    f[..., 0] = 38.0
    f[..., 1] = 38.0 * fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    torch.cuda.synchronize()
    sim.step(w.n_steps)
    sim.sync()
    f = sim.field_tensor()
    assert float((f[..., 0] - 38.0).abs().max()) <= 38.0 * 1e-5
    expect = (38.0 * _mode_factor(w, 1, k) ** w.n_steps) * (
        fz[:, None, None] * fy[None, :, None] * fx[None, None, :])
    err = float((f[..., 1].double() - expect.double()).abs().max()) / 38.0
    sim.close()
    assert err <= 1e-5


def _device_rel_err(got, ref):
    """Normwise error of two device fields, in FP64, in chunks (bounded temporaries)."""
    import torch
    g, r = got.reshape(-1), ref.reshape(-1)
    d = torch.zeros((), dtype=torch.float64, device=r.device)
    for i in range(0, r.numel(), 1 << 28):
        d = torch.maximum(d, (g[i:i + (1 << 28)].double() - r[i:i + (1 << 28)].double()).abs().max())
    return float(d / r.abs().max().double())


@pytest.mark.slow
def test_workload2_full_size_100_steps_fp32_with_agents_vs_fp64(binding):
    """400^3 x 4 with its 1M agents, 100 steps: FP32 against the FP64 GPU path on the same
    inputs (that path matches the oracle element by element on a full-size step and over 100
    steps at reduced size).  Target: normwise <= 1e-5."""
    import torch
    w = inputs.workload(2)
    out = {}
    for prec in ("fp64", "fp32"):
        sim = binding.BioFVM.from_workload(w, precision=prec)
        sim.step(w.n_steps)
        out[prec] = sim.field_tensor().clone()
        sim.close()
    err = _device_rel_err(out["fp32"], out["fp64"])
    del out
    torch.cuda.empty_cache()
    assert err <= 1e-5, err


@pytest.mark.slow
def test_workload3_full_size_20_steps_fp32_with_agents_vs_fp64(binding):
    """1200^3 x 2 (13.8 GB FP32), Dirichlet 38 on substrate 0, 64 Gaussian blobs and its 10M
    agents, 20 steps: FP32 against the FP64 GPU path (27.6 GB) on the same inputs, the blob
    field evaluated on the device.  Target: normwise <= 1e-5."""
    import torch
    w = inputs.workload(3, with_field=False)
    f64 = inputs.gaussian_blobs_device(w.extra["blobs"], w.nx, w.ny, w.nz, w.ns, w.dx, "cuda")
    sim = binding.BioFVM.from_workload(w, precision="fp32")
    sim.set_density(f64.float())
    sim.step(w.n_steps)
    got = sim.field_tensor().clone()
    sim.close()
    torch.cuda.empty_cache()
    ref = binding.BioFVM.from_workload(w, precision="fp64")
    ref.set_density(f64)
    del f64
    ref.step(w.n_steps)
    ref.sync()
    err = _device_rel_err(got, ref.field_tensor())
    ref.close()
    del got
    torch.cuda.empty_cache()
    assert err <= 1e-5, err


def test_workload3_slab_2_steps_fp64_vs_oracle(binding):
    """A 1200 x 1200 x 8 slab of the 1200^3 recipe (Dirichlet faces, blobs, agents at the same
    density), 2 steps: the FP64 GPU path against the oracle, every element."""
    w = inputs.workload(3, shape=(1200, 1200, 8), n_agents=10_000_000 * 8 // 1200)
    ref = orc(w).step(w.rho0, 2)
    got = gpu_run(binding, w, "fp64", 2)
    assert rel_err(got, ref) <= 1e-12


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("shape", [(40, 36, 28, 4), (64, 300, 9, 2), (8, 8, 520, 1), (16, 70, 70, 3),
                                   (33, 1, 47, 5), (1, 65, 2, 7), (100, 30, 20, 8),
                                   # long lines: pipelined tiles of 16 columns
                                   (12, 10, 1100, 1), (1000, 6, 5, 2), (9, 900, 7, 3),
                                   (1300, 3, 2, 1)],
                         ids=lambda s: "x".join(map(str, s)) if isinstance(s, tuple) else s)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sweep_paths_match_oracle(binding, monkeypatch, shape, path, prec):
    """Every sweep implementation -- plain kernels, the persistent TMA pipeline (FP32) and the
    streaming whole-line kernels, chosen at create through BIOFVM_PIPELINE / BIOFVM_STREAM /
    BIOFVM_STREAM32 -- against the oracle, with Dirichlet faces and sources."""
    if prec == "fp64" and path == "pipe":
        pytest.skip("the pipelined sweep is FP32 only")
    monkeypatch.setenv("BIOFVM_PIPELINE", PATHS[path][0])
    monkeypatch.setenv("BIOFVM_STREAM", PATHS[path][1])
    monkeypatch.setenv("BIOFVM_STREAM32", PATHS[path][2])
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(17)
    w = inputs.random_problem(rng, nx, ny, nz, ns, n_agents=100, dirichlet=True)
    ref = orc(w).step(w.rho0, 3)
    try:
        got = gpu_run(binding, w, prec, 3)
    except binding.BioFVMError as e:
        # only the plain kernels alone may refuse a grid: lines longer than their register
        # chunks hold (the library then needs the streaming or pipelined sweep)
        if path == "plain" and e.status == binding.ERR_ARG and "too long" in str(e):
            pytest.skip(f"plain kernels cannot hold these lines: {e}")
        raise
    assert rel_err(got, ref) <= TOL[prec]


@pytest.mark.parametrize("shape", [(37, 23, 19, 3), (250, 20, 16, 1), (9, 130, 11, 2),
                                   (31, 17, 9, 3), (101, 5, 300, 1), (3, 4, 5, 1)],
                         ids=lambda s: "x".join(map(str, s)))
def test_unaligned_rows_run_pitched_and_match_oracle(binding, monkeypatch, shape):
    """FP32 fields whose rows (nx * n_sub floats) are no 16-byte multiple: biofvm_step runs the
    pipelined sweeps on a row-padded copy of the field.  Against the oracle (sources, Dirichlet
    faces) over calls of 1 and 2 steps, and against the same problem without the padded copy
    (BIOFVM_PITCHED=0: the plain kernels along x and y)."""
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(nx + 7 * ns)
    w = inputs.random_problem(rng, nx, ny, nz, ns, n_agents=150, dirichlet=True)
    ref = orc(w).step(w.rho0, 3)
    outs = []
    for pitched in ("1", "0"):
        monkeypatch.setenv("BIOFVM_PITCHED", pitched)
        sim = binding.BioFVM.from_workload(w, precision="fp32")
        d = sim.describe()
        assert ("pitched" in d) == (pitched == "1"), d
        sim.step(1)
        sim.step(2)
        outs.append(sim.density().astype(np.float64))
        sim.close()
        assert rel_err(outs[-1], ref) <= 1e-5, (pitched, d)
    assert rel_err(outs[0], outs[1]) <= 1e-5


def test_describe_names_the_step_kernels(binding, monkeypatch):
    rng = np.random.default_rng(5)
    w = inputs.random_problem(rng, 40, 36, 28, 4, n_agents=50)
    sim = binding.BioFVM.from_workload(w, precision="fp32")
    assert sim.describe().startswith("x=pipe/cw32/m") and "pitched" not in sim.describe()
    sim.close()
    monkeypatch.setenv("BIOFVM_SMALL", "0")
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    assert sim.describe() == "x=stream y=stream z=stream scaled"
    sim.set_dirichlet_nodes([5], [1], [2.0])
    assert sim.describe().endswith(" nodes")
    sim.close()
    monkeypatch.setenv("BIOFVM_SMALL", "1")
    small = inputs.workload(1)
    sim = binding.BioFVM.from_workload(small, precision="fp64")
    assert sim.describe() == "cooperative"
    sim.close()


@pytest.mark.parametrize("r", ["16", "8"])
@pytest.mark.parametrize("xt,ks", [("2", "32"), ("4", "48"), ("4", "0"), ("2", "16"), ("0", "64")],
                         ids=lambda v: v)
@pytest.mark.parametrize("shape", [(37, 23, 19, 1), (70, 9, 11, 2), (250, 6, 5, 1),
                                   (33, 17, 9, 4), (19, 13, 7, 2)],
                         ids=lambda s: "x".join(map(str, s)))
def test_fp64_streaming_x_sweep_row_forms_match_oracle(binding, monkeypatch, shape, xt, ks, r):
    """The FP64 streaming x-sweep with the warp's rows moved as contiguous segments through the
    transpose buffer (S <= BIOFVM_STREAM_XT, S in 1, 2, 4; S = 4 with 16-position blocks only)
    and with lane-owned rows (BIOFVM_STREAM_XT=0), slabs of BIOFVM_STREAM_KS_XT positions (0:
    none; 16, 48: a backward block straddles the slab's end on these lengths), register blocks
    of 16 or 8 positions (BIOFVM_STREAM_R): against the oracle over calls of 1 and 2 steps, with
    sources and Dirichlet faces, rows that do not fill a warp, and line lengths that are no
    multiple of the blocks.  Small grids would take the cooperative step, so the per-sweep
    kernels are forced."""
    monkeypatch.setenv("BIOFVM_SMALL", "0")
    monkeypatch.setenv("BIOFVM_STREAM_XT", xt)
    monkeypatch.setenv("BIOFVM_STREAM_KS_XT", ks)
    monkeypatch.setenv("BIOFVM_STREAM_R", r)
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(nx * 3 + ns)
    w = inputs.random_problem(rng, nx, ny, nz, ns, n_agents=120, dirichlet=True)
    ref = orc(w).step(w.rho0, 3)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    assert sim.describe() == "x=stream y=stream z=stream scaled", sim.describe()
    sim.step(1)
    sim.step(2)
    got = sim.density()
    sim.close()
    assert rel_err(got, ref) <= 1e-12


@pytest.mark.parametrize("shape", [(40, 20, 16, 2), (37, 22, 14, 3), (64, 10, 12, 4)],
                         ids=lambda s: "x".join(map(str, s)))
def test_fp32_x_tiles_dense_and_sparse_sources_match_oracle(binding, shape):
    """Pipelined x tiles whose rows hold more source entries than the preparer warp prefetches
    (the consumers then apply the tile's sources and Dirichlet rows) beside sparse tiles (the
    preparer applies them) in one launch: agents packed into the lowest z-planes, a few more
    scattered, Dirichlet faces; rows aligned or on the row-padded copy.  Against the oracle."""
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(nx + nz)
    w = inputs.random_problem(rng, nx, ny, nz, ns, n_agents=0, dirichlet=True)
    dense = rng.integers(0, nx * ny * 3, 6 * nx * ny)      # z < 3: several per voxel
    sparse = rng.integers(nx * ny * 3, nx * ny * nz, 40)   # elsewhere: a few
    w.voxel = np.concatenate([dense, sparse]).astype(np.int64)
    n = w.voxel.size
    w.secretion = rng.uniform(0.1, 10.0, (n, ns))
    w.target = rng.uniform(1.0, 38.0, (n, ns))
    w.uptake = rng.uniform(0.0, 1.0, (n, ns))
    w.weight = rng.uniform(0.5, 1.0, n)
    ref = orc(w).step(w.rho0, 3)
    sim = binding.BioFVM.from_workload(w, precision="fp32")
    assert sim.describe().startswith("x=pipe"), sim.describe()
    sim.step(3)
    got = sim.density()
    sim.close()
    assert rel_err(got, ref) <= 1e-5
