"""Moving agents: source lists rebuilt on the device from device agent arrays
(biofvm_reserve_agents / biofvm_set_sources_device), through the C ABI.

The device rebuild sums the agents of a voxel in the same order as the host builder
(biofvm_set_sources), so a step with either list gives the same bits; agents that move every
step are checked against the FP64 oracle given the same per-step agent lists.
"""
import numpy as np
import pytest

import oracle
from paper_2602_05017_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def binding():
    from paper_2602_05017_gb300 import binding as b
    return b


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def dev(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


def agents_with_collisions(rng, nvox, ns, n, weight=True):
    """Mixed sources and sinks; a fifth of them share voxels with others, some have zero
    rates, weights in [0.5, 1.5]."""
    voxel, sec, tgt, upt = inputs.random_agents(rng, nvox, ns, n)
    k = n // 5
    voxel[-k:] = voxel[:k]
    sec[: n // 10] = 0.0
    upt[: n // 10] = 0.0
    w = rng.uniform(0.5, 1.5, n) if weight else None
    return voxel, sec, tgt, upt, w


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,n", [((23, 17, 13, 3), 400), ((64, 48, 40, 4), 60000)],
                         ids=["small", "multi-block"])
def test_device_lists_give_the_host_lists_bits(binding, prec, shape, n):
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(5 + n)
    w = inputs.random_problem(rng, nx, ny, nz, ns, dirichlet=True, n_nodes=30)
    voxel, sec, tgt, upt, wt = agents_with_collisions(rng, nx * ny * nz, ns, n)
    nodes = w.dirichlet_nodes
    voxel[:3] = nodes[0][:3]  # agents on Dirichlet-node voxels: their entries are dropped
    host = binding.BioFVM.from_workload(w, precision=prec)
    host.set_sources(voxel, sec, tgt, upt, wt)
    devh = binding.BioFVM.from_workload(w, precision=prec)
    devh.reserve_agents(n + 5)
    devh.set_sources_device(dev(voxel), dev(sec), dev(tgt), dev(upt), dev(wt))
    host.step(4)
    devh.step(4)
    a, b = host.density(), devh.density()
    host.close()
    devh.close()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_one_voxel_holding_many_agents(binding, prec):
    """10000 agents in one voxel (a run the device sums serially) plus scattered ones."""
    rng = np.random.default_rng(9)
    w = inputs.random_problem(rng, 20, 18, 16, 2)
    voxel, sec, tgt, upt, wt = agents_with_collisions(rng, 20 * 18 * 16, 2, 12000)
    voxel[:10000] = 777
    host = binding.BioFVM.from_workload(w, precision=prec)
    host.set_sources(voxel, sec, tgt, upt, wt)
    devh = binding.BioFVM.from_workload(w, precision=prec)
    devh.reserve_agents(12000)
    devh.set_sources_device(dev(voxel), dev(sec), dev(tgt), dev(upt), dev(wt))
    host.step(2)
    devh.step(2)
    assert np.array_equal(host.density(), devh.density())
    host.close()
    devh.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(30, 26, 22, 2), (31, 26, 22, 2)],
                         ids=["rows-aligned", "rows-unaligned"])
def test_agents_moving_every_step_match_the_oracle(binding, prec, shape):
    """A random walk of 300 agents (one voxel along a random axis per step, clamped to the
    box), 12 steps, Dirichlet faces: each step's agent list goes to the oracle and, as device
    arrays, to the library before that step.  31 x 2 floats per row is no 16-byte multiple:
    the FP32 steps then run on the row-padded copy."""
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(21)
    w = inputs.random_problem(rng, nx, ny, nz, ns, dirichlet=True)
    voxel, sec, tgt, upt, wt = agents_with_collisions(rng, nx * ny * nz, ns, 300)
    sim = binding.BioFVM.from_workload(w, precision=prec)
    if prec == "fp32":
        assert ("pitched" in sim.describe()) == (nx * ns * 4 % 16 != 0), sim.describe()
    sim.reserve_agents(300)
    ref = w.rho0.copy()
    x, y, z = voxel % nx, (voxel // nx) % ny, voxel // (nx * ny)
    for _ in range(12):
        ax = rng.integers(0, 3, voxel.size)
        d = rng.choice([-1, 1], voxel.size)
        x = np.clip(x + d * (ax == 0), 0, nx - 1)
        y = np.clip(y + d * (ax == 1), 0, ny - 1)
        z = np.clip(z + d * (ax == 2), 0, nz - 1)
        voxel = (z * ny + y) * nx + x
        w.voxel, w.secretion, w.target, w.uptake, w.weight = voxel, sec, tgt, upt, wt
        ref = oracle.Problem(**w.oracle_kwargs()).step(ref, 1)
        sim.set_sources_device(dev(voxel), dev(sec), dev(tgt), dev(upt), dev(wt))
        sim.step(1)
    got = sim.density()
    sim.close()
    assert rel_err(got, ref) <= TOL[prec]


def test_no_agents_and_invalid_agents(binding):
    rng = np.random.default_rng(3)
    w = inputs.random_problem(rng, 12, 10, 8, 2)
    nvox = 12 * 10 * 8
    p = oracle.Problem(**w.oracle_kwargs())
    sim = binding.BioFVM.from_workload(w)
    sim.reserve_agents(50)
    import torch
    sim.set_sources_device(torch.zeros(0, dtype=torch.int64, device="cuda"))
    sim.step(1)
    assert rel_err(sim.density(), p.step(w.rho0, 1)) <= 1e-12
    voxel, sec, tgt, upt, _ = agents_with_collisions(rng, nvox, 2, 40, weight=False)
    bad = voxel.copy()
    bad[7] = nvox  # out of range: dropped, reported at the next synchronising call
    sim.set_density(w.rho0)
    sim.set_sources_device(dev(bad), dev(sec), dev(tgt), dev(upt))
    sim.step(1)
    with pytest.raises(binding.BioFVMError) as e:
        sim.sync()
    assert e.value.status == binding.ERR_ARG
    keep = np.arange(40) != 7
    w.voxel, w.secretion, w.target, w.uptake = voxel[keep], sec[keep], tgt[keep], upt[keep]
    assert rel_err(sim.density(), oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 1)) <= 1e-12
    with pytest.raises(binding.BioFVMError) as e:  # more agents than reserved
        sim.set_sources_device(dev(np.zeros(51, dtype=np.int64)))
    assert e.value.status == binding.ERR_ARG
    g = torch.zeros(sim.n_elem, dtype=torch.float64, device="cuda")
    saved = torch.zeros(4 * sim.n_elem, dtype=torch.float64, device="cuda")
    d2 = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.BioFVMError) as e:  # the adjoint needs host agent arrays
        sim.adjoint_step(g, g, d2, d2.clone(), None, saved)
    assert e.value.status == binding.ERR_STATE
    sim.set_sources(voxel[keep], sec[keep], tgt[keep], upt[keep])  # back to host lists
    sim.set_density(w.rho0)
    sim.step(1)
    assert rel_err(sim.density(), oracle.Problem(**w.oracle_kwargs()).step(w.rho0, 1)) <= 1e-12
    sim.close()
