"""Batched persistent step (biofvm_batch_*) against the FP64 oracle, environment by environment,
plus the autotuner's cache plumbing."""
import numpy as np
import pytest

import oracle
from paper_2602_05017_gb300 import autotune, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def binding():
    from paper_2602_05017_gb300 import binding as b
    return b


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _envs(seed, shapes, agents=True):
    rng = np.random.default_rng(seed)
    out = []
    for (nx, ny, nz, ns) in shapes:
        w = inputs.random_problem(rng, nx, ny, nz, ns,
                                  n_agents=max(1, nx * ny * nz // 30) if agents else 0)
        out.append(w)
    return out


SHAPES = [(33, 17, 9, 3), (8, 40, 21, 1), (50, 50, 50, 4), (7, 5, 3, 8), (64, 9, 30, 2),
          (1, 12, 12, 2), (20, 20, 1, 5), (96, 11, 13, 6)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_oracle_per_environment(binding, prec):
    envs = _envs(1, SHAPES)
    b = binding.BioFVMBatch(envs, precision=prec)
    for sim, w in zip(b.envs, envs):
        sim.set_density(w.rho0)
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
    b.step(4)
    b.sync()
    for sim, w in zip(b.envs, envs):
        ref = oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 4)
        assert rel(sim.density(), ref) <= TOL[prec], w.name
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_whole_lines_match_oracle(binding, prec):
    """Whole-line tiles (m >= n on every axis: one warp streams 32 whole lines) against the
    oracle, environment by environment, with sources."""
    envs = _envs(11, SHAPES)
    b = binding.BioFVMBatch(envs, precision=prec, tile_m=[[w.nx, w.ny, w.nz] for w in envs])
    for sim, w in zip(b.envs, envs):
        sim.set_density(w.rho0)
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
    b.step(4)
    b.sync()
    for sim, w in zip(b.envs, envs):
        ref = oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 4)
        assert rel(sim.density(), ref) <= TOL[prec], w.name
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_mixed_whole_and_chunked_axes_and_retiling(binding, prec):
    """Whole lines on some axes and chunks on others in one launch, then re-tiled the other
    way round (biofvm_batch_set_tiles) with the field carried over."""
    envs = _envs(12, [(64, 40, 36, 3), (150, 20, 90, 2), (33, 96, 17, 5)])
    first = [[w.nx, 16, w.nz] for w in envs]
    second = [[0, w.ny, 24] for w in envs]
    b = binding.BioFVMBatch(envs, precision=prec, tile_m=first)
    for sim, w in zip(b.envs, envs):
        sim.set_density(w.rho0)
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
    b.step(2)
    b.set_tiles(second)
    b.step(3)
    b.sync()
    for sim, w in zip(b.envs, envs):
        ref = oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 5)
        assert rel(sim.density(), ref) <= TOL[prec], w.name
    b.close()


def test_batch_with_explicit_tile_shapes_and_repeated_calls(binding):
    envs = _envs(2, [(48, 40, 36, 2), (25, 31, 19, 4), (64, 64, 8, 1)])
    shapes = [[m, m, m] for m in (8, 12, 16)]
    b = binding.BioFVMBatch(envs, precision="fp64", tile_m=shapes)
    for sim, w in zip(b.envs, envs):
        sim.set_density(w.rho0)
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
    b.step(2)
    b.step(3)  # a second graph for another step count, the field carried over
    b.sync()
    for sim, w in zip(b.envs, envs):
        ref = oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 5)
        assert rel(sim.density(), ref) <= 1e-12
    b.close()


def test_batch_sources_changed_between_launches(binding):
    envs = _envs(3, [(30, 20, 10, 2), (12, 12, 12, 3)])
    b = binding.BioFVMBatch(envs, precision="fp64")
    for sim, w in zip(b.envs, envs):
        sim.set_density(w.rho0)
    b.step(1)
    mid = [sim.density() for sim in b.envs]
    for sim, w in zip(b.envs, envs):
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
    b.step(2)
    b.sync()
    for sim, w, m in zip(b.envs, envs, mid):
        ref = oracle.Problem(**w.oracle_kwargs()).step(m, 2)
        assert rel(sim.density(), ref) <= 1e-12
    b.close()


def test_batch_rejects_invalid_tile_shapes(binding):
    envs = _envs(4, [(100, 10, 10, 1)])
    with pytest.raises(binding.BioFVMError):
        binding.BioFVMBatch(envs, tile_m=[[8, 8, 8]])  # 100/8 -> 13 chunks > 8
    with pytest.raises(binding.BioFVMError):
        binding.BioFVMBatch(envs, tile_m=[[60, 8, 8]])  # chunks of more than 48 (not whole)


def test_batched_workload_recipe_reduced(binding):
    """The batched recipe (uneven cubes, 1-8 substrates, log-uniform D and lambda, agents 1 per
    64 voxels) with 12 environments of edge 16-48, 10 steps, FP32 vs the FP64 oracle."""
    envs = inputs.batched_workloads(n_env=12, edge=(16, 48), n_steps=10, field_dtype=np.float64)
    b = binding.BioFVMBatch(envs, precision="fp32")
    for sim, w in zip(b.envs, envs):
        sim.set_density(w.rho0)
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
    b.step(10)
    b.sync()
    for sim, w in zip(b.envs, envs):
        ref = oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 10)
        assert rel(sim.density(), ref) <= 1e-5, w.name
    b.close()


def test_autotuner_cache_roundtrip(binding, tmp_path):
    cache = autotune.tune("fp32", n_buckets=(32,), subs=(2,), target_vs=2e6, steps=1, reps=1,
                          path=str(tmp_path / "c.json"))
    loaded = autotune.load(str(tmp_path / "c.json"))
    assert loaded["classes"].keys() == cache["classes"].keys()
    envs = _envs(5, [(30, 33, 31, 2), (32, 32, 32, 2)], agents=False)
    shapes = autotune.tile_shapes(envs, loaded)
    b = binding.BioFVMBatch(envs, precision="fp32", tile_m=shapes)
    for sim, w in zip(b.envs, envs):
        sim.set_density(w.rho0)
    b.step(2)
    b.sync()
    for sim, w in zip(b.envs, envs):
        ref = oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 2)
        assert rel(sim.density(), ref) <= 1e-5
    b.close()


def test_bounded_wait_expires_reports_timeout_and_context_stays_usable(binding):
    """Failure detection without a GPU fault: a dependency wait that can never be satisfied gives
    up (about two seconds), the host reads TIMEOUT, and the next normal launch is correct."""
    envs = _envs(6, [(24, 20, 16, 2), (16, 16, 16, 1)], agents=False)
    b = binding.BioFVMBatch(envs, precision="fp64")
    for sim, w in zip(b.envs, envs):
        sim.set_density(w.rho0)
    b.test_stall(True)
    b.step(1)
    with pytest.raises(binding.BioFVMError) as err:
        b.sync()
    assert err.value.status == binding.ERR_TIMEOUT
    b.test_stall(False)
    for sim, w in zip(b.envs, envs):
        sim.set_density(w.rho0)
    b.step(2)
    b.sync()
    for sim, w in zip(b.envs, envs):
        ref = oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 2)
        assert rel(sim.density(), ref) <= 1e-12
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_graph_mode_matches_oracle(binding, prec):
    """Per-environment graph mode (each environment on the single-grid sweeps, one graph of
    every environment's launches per step): against the oracle environment by environment,
    over calls of 4 and 2 steps with the sources replaced in between (a new graph), including
    environments whose FP32 rows are no 16-byte multiple (row-padded copies)."""
    envs = _envs(21, SHAPES)
    b = binding.BioFVMBatch(envs, precision=prec, mode="graph")
    assert b.mode() == "graph" and b.grid() == 0
    for sim, w in zip(b.envs, envs):
        sim.set_density(w.rho0)
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
    b.step(4)
    b.sync()
    mid = []
    for sim, w in zip(b.envs, envs):
        ref = oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 4)
        got = sim.density()
        assert rel(got, ref) <= TOL[prec], w.name
        mid.append(np.asarray(got, dtype=np.float64))
    rng = np.random.default_rng(5)
    for sim, w in zip(b.envs, envs):  # new agents: the graph is captured again
        w.secretion = w.secretion * rng.uniform(0.5, 1.5, w.secretion.shape)
        sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
    b.step(2)
    b.sync()
    for sim, w, m in zip(b.envs, envs, mid):
        ref = oracle.Problem(**w.oracle_kwargs()).step(m, 2)
        assert rel(sim.density(), ref) <= TOL[prec], w.name
    with pytest.raises(binding.BioFVMError) as e:
        b.set_tiles([[8, 8, 8]] * len(envs))
    assert e.value.status == binding.ERR_STATE
    with pytest.raises(binding.BioFVMError) as e:
        b.test_stall(True)
    assert e.value.status == binding.ERR_STATE
    b.envs[1].set_dirichlet_nodes([3], [0], [1.0])
    with pytest.raises(binding.BioFVMError) as e:
        b.step(1)
    assert e.value.status == binding.ERR_ARG
    b.close()


def test_batch_mode_follows_environment_size(binding):
    """Without an explicit mode: the persistent kernel for small environments, per-environment
    graphs once the mean environment holds 2^20 voxel-substrates."""
    small = binding.BioFVMBatch(_envs(22, [(20, 20, 20, 2), (30, 10, 10, 1)], agents=False))
    assert small.mode() == "persistent" and small.grid() > 0
    small.close()
    big = binding.BioFVMBatch(_envs(23, [(128, 128, 64, 1), (64, 64, 64, 8)], agents=False))
    assert big.mode() == "graph"
    big.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_item_claims_and_grid_sizes_give_identical_fields(binding, prec, monkeypatch):
    """The persistent kernel's schedule does not touch the arithmetic: items claimed from the
    counter (default), statically strided (BIOFVM_BATCH_DYNAMIC=0) and on one CTA per SM
    (BIOFVM_BATCH_CTAS=1) give bit-identical fields, whole-line and chunked axes mixed, long
    lines included; the first also against the oracle."""
    envs = _envs(31, [(150, 40, 36, 3), (33, 96, 17, 5), (64, 9, 130, 1), (7, 5, 3, 8)])
    tiles = [[w.nx, 16, w.nz] for w in envs]
    fields, grids = [], []
    for knobs in ({}, {"BIOFVM_BATCH_DYNAMIC": "0"}, {"BIOFVM_BATCH_CTAS": "1"}):
        for k in ("BIOFVM_BATCH_DYNAMIC", "BIOFVM_BATCH_CTAS"):
            monkeypatch.delenv(k, raising=False)
        for k, v in knobs.items():
            monkeypatch.setenv(k, v)
        b = binding.BioFVMBatch(envs, precision=prec, tile_m=tiles, mode="persistent")
        grids.append(b.grid())
        for sim, w in zip(b.envs, envs):
            sim.set_density(w.rho0)
            sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
        b.step(3)
        b.sync()
        fields.append([np.asarray(sim.density()).copy() for sim in b.envs])
        b.close()
    assert grids[0] == grids[1] and grids[0] % grids[2] == 0 and grids[2] < grids[0]
    for other in fields[1:]:
        for a, c in zip(fields[0], other):
            assert np.array_equal(a, c)
    for got, w in zip(fields[0], envs):
        ref = oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 3)
        assert rel(got, ref) <= TOL[prec], w.name
