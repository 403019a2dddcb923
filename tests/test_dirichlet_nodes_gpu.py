"""Dirichlet nodes (biofvm_set_dirichlet_nodes) against the FP64 CPU oracle, through the C ABI:
voxels held at a value anywhere in the grid and per-face Dirichlet values, on every sweep
implementation, together with the flagged faces of the boundary and the agents' sources."""
import numpy as np
import pytest

import oracle
from paper_2602_05017_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
PATHS = {"plain": ("0", "0", "0"), "pipe": ("1", "0", "0"), "stream": ("1", "1", "1")}


@pytest.fixture(scope="module")
def binding():
    from paper_2602_05017_gb300 import binding as b
    return b


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def orc(w):
    return oracle.Problem(**w.oracle_kwargs())


def run(binding, w, prec, n_steps):
    sim = binding.BioFVM.from_workload(w, precision=prec)
    sim.step(n_steps)
    out = sim.density().astype(np.float64)
    sim.close()
    return out


def set_path(monkeypatch, path):
    monkeypatch.setenv("BIOFVM_PIPELINE", PATHS[path][0])
    monkeypatch.setenv("BIOFVM_STREAM", PATHS[path][1])
    monkeypatch.setenv("BIOFVM_STREAM32", PATHS[path][2])


def interior(nx, ny, nz, voxel):
    x, y, z = voxel % nx, (voxel // nx) % ny, voxel // (nx * ny)
    return (x > 0) & (x < nx - 1) & (y > 0) & (y < ny - 1) & (z > 0) & (z < nz - 1)


@pytest.mark.parametrize("on_faces", [False, True], ids=["inside", "on-faces"])
@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nodes_match_oracle(binding, monkeypatch, path, prec, on_faces):
    """60 nodes (some repeated, some on agents' voxels) with flagged faces and sources, 20 steps
    (FP64: a renormalisation block and a tail).  on-faces: nodes also sit on flagged faces, so
    those faces are applied as nodes and the nodes win there."""
    if prec == "fp64" and path == "pipe":
        pytest.skip("the pipelined sweep is FP32 only")
    set_path(monkeypatch, path)
    rng = np.random.default_rng(41)
    nx, ny, nz = 45, 38, 33
    w = inputs.random_problem(rng, nx, ny, nz, 3, n_agents=90, dirichlet=True, n_nodes=60)
    voxel, sub, val = w.dirichlet_nodes
    if not on_faces:
        keep = interior(nx, ny, nz, voxel)
        voxel, sub, val = voxel[keep], sub[keep], val[keep]
    else:
        voxel[10:14] = [0, nx - 1, nx * ny * (nz - 1), nx * (ny - 1)]  # corners and edges
        sub[10:14] = 0                                                 # substrate 0 is flagged
    voxel[:4], sub[:4] = w.voxel[:4], np.arange(4) % 3                 # nodes on agents
    w.dirichlet_nodes = (voxel, sub, val)
    ref = orc(w).step(w.rho0, 20)
    got = run(binding, w, prec, 20)
    assert rel_err(got, ref) <= TOL[prec]
    flat = got.reshape(-1)
    last = {}
    for v, s, x in zip(voxel, sub, val):
        last[int(v) * 3 + int(s)] = x
    for e, x in last.items():  # every node holds its (last) value
        assert abs(flat[e] - x) <= TOL[prec] * 38.0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_per_face_values_match_oracle(binding, prec):
    """Six different values on the six faces for substrate 0, one face for substrate 1, none for
    substrate 2 (given as nodes, the later face winning at edges and corners), 20 steps."""
    rng = np.random.default_rng(42)
    nx, ny, nz = 40, 31, 27
    w = inputs.random_problem(rng, nx, ny, nz, 3, n_agents=60)
    faces = np.full((6, 3), np.nan)
    faces[:, 0] = [2.0, 30.0, 11.0, 19.0, 5.0, 37.0]
    faces[1, 1] = 25.0
    w.dirichlet_nodes = inputs.face_value_nodes(nx, ny, nz, faces)
    ref = orc(w).step(w.rho0, 20)
    got = run(binding, w, prec, 20)
    assert rel_err(got, ref) <= TOL[prec]


@pytest.mark.parametrize("path", ["plain", "stream"])
def test_each_stage_with_nodes_matches_oracle(binding, monkeypatch, path):
    """Stages 0-3 (Src then B, X^-1 then B, Y^-1 then B, Z^-1 then B) with nodes and flagged
    faces, one by one against the oracle's stages."""
    set_path(monkeypatch, path)
    rng = np.random.default_rng(43)
    w = inputs.random_problem(rng, 29, 23, 21, 2, n_agents=50, dirichlet=True, n_nodes=40)
    p = orc(w)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    ref = w.rho0
    steps = [lambda u: p.dirichlet(p.sources(u))] + [
        (lambda a: (lambda u: p.dirichlet(p.sweep(a, u))))(a) for a in range(3)]
    for stage, f in enumerate(steps):
        sim.run_stage(stage)
        ref = f(ref)
        assert rel_err(sim.density(), ref) <= 1e-12, stage
    sim.close()


def test_nodes_replaced_cleared_and_rejected(binding):
    """Nodes set, replaced, cleared (n = 0) between calls; bad nodes (voxel or substrate out of
    range, a value that is not finite) are refused and change nothing."""
    rng = np.random.default_rng(44)
    w = inputs.random_problem(rng, 21, 18, 16, 2, n_agents=30, dirichlet=True, n_nodes=25)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    p1 = orc(w)
    sim.step(3)
    ref = p1.step(w.rho0, 3)
    assert rel_err(sim.density(), ref) <= 1e-12
    nodes2 = inputs.random_nodes(rng, 21 * 18 * 16, 2, 12)
    sim.set_dirichlet_nodes(*nodes2)
    w.dirichlet_nodes = nodes2
    sim.step(2)
    ref = orc(w).step(ref, 2)
    assert rel_err(sim.density(), ref) <= 1e-12
    for bad in (([21 * 18 * 16], [0], [1.0]), ([3], [2], [1.0]), ([3], [0], [np.nan])):
        with pytest.raises(binding.BioFVMError):
            sim.set_dirichlet_nodes(*bad)
    sim.step(1)
    ref = orc(w).step(ref, 1)
    assert rel_err(sim.density(), ref) <= 1e-12
    sim.set_dirichlet_nodes([], [], [])
    w.dirichlet_nodes = None
    sim.step(2)
    ref = orc(w).step(ref, 2)
    assert rel_err(sim.density(), ref) <= 1e-12
    # without nodes: the three sweeps, or one cooperative launch (a grid this small)
    assert " nodes" not in sim.describe()
    assert sim.launches_per_step() == (1 if sim.describe() == "cooperative" else 3)
    sim.close()


def test_nodes_refused_in_a_batch(binding):
    rng = np.random.default_rng(45)
    envs = [inputs.random_problem(rng, 20, 20, 20, 2), inputs.random_problem(rng, 12, 9, 7, 1)]
    b = binding.BioFVMBatch(envs, precision="fp32")
    b.envs[1].set_dirichlet_nodes([5], [0], [1.0])
    with pytest.raises(binding.BioFVMError):
        b.step(1)
    b.close()
