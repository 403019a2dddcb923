"""GPU adjoint (biofvm_step_save / biofvm_adjoint_step / LODSteps) against the FP64 CPU
adjoint of the oracle and against central finite differences.

Targets: FP64 gradients within 1e-10 (relative, normwise) of the CPU adjoint and within 1e-6 of
central FD (plus the FD's own rounding bound eps*|L|/h).
"""
import copy

import numpy as np
import pytest

import oracle
from paper_2602_05017_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def cpu_loss_and_grads(w, n_steps, probes, targets):
    p = oracle.Problem(**w.oracle_kwargs())
    states = [w.rho0.copy()]
    for _ in range(n_steps):
        states.append(p.step(states[-1], 1))
    fin = states[-1].reshape(-1)
    loss = float(((fin[probes] - targets) ** 2).sum())
    g = np.zeros(fin.size)
    g[probes] = 2.0 * (fin[probes] - targets)
    g = g.reshape(w.shape)
    dD, dl = np.zeros(w.ns), np.zeros(w.ns)
    ds = np.zeros((w.n_agents, w.ns))
    du = np.zeros((w.n_agents, w.ns))
    for k in range(n_steps - 1, -1, -1):
        g, a, b, c, u = p.adjoint_step(states[k], g)
        dD += a
        dl += b
        ds += c
        du += u
    return loss, g, dD, dl, ds, du


def gpu_loss_and_grads(torch, w, n_steps, probes, targets, prec="fp64", ckpt=3):
    from paper_2602_05017_gb300 import binding
    from paper_2602_05017_gb300.adjoint import lod_steps
    dt = torch.float64 if prec == "fp64" else torch.float32
    sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, w.dirichlet_on,
                         w.dirichlet_value, precision=prec)
    if w.dirichlet_nodes is not None:
        sim.set_dirichlet_nodes(*w.dirichlet_nodes)
    rho0 = torch.tensor(w.rho0, dtype=torch.float64, device="cuda", requires_grad=True)
    sec = torch.tensor(w.secretion, dtype=torch.float64, device="cuda", requires_grad=True)
    D = torch.tensor(w.D, dtype=torch.float64, device="cuda", requires_grad=True)
    lam = torch.tensor(w.lam, dtype=torch.float64, device="cuda", requires_grad=True)
    upt = torch.tensor(w.uptake, dtype=torch.float64, device="cuda", requires_grad=True)
    agents = dict(voxel=w.voxel, target=w.target, weight=w.weight)
    out = lod_steps(rho0.to(dt), sec, D, lam, sim, agents, n_steps, ckpt, uptake=upt)
    flat = out.reshape(-1).double()
    pr = torch.as_tensor(probes, device="cuda")
    tg = torch.as_tensor(targets, device="cuda")
    loss = ((flat[pr] - tg) ** 2).sum()
    loss.backward()
    res = (float(loss.detach()), rho0.grad.cpu().numpy(), D.grad.cpu().numpy(), lam.grad.cpu().numpy(),
           sec.grad.cpu().numpy(), upt.grad.cpu().numpy())
    sim.close()
    return res


def _problem(seed, shape=(13, 11, 9), ns=2, dirichlet=True, n_agents=40):
    rng = np.random.default_rng(seed)
    w = inputs.random_problem(rng, *shape, ns, n_agents=n_agents, dirichlet=dirichlet)
    probes = rng.choice(w.rho0.size, min(200, w.rho0.size), replace=False)
    targets = rng.uniform(0, 38, probes.size)
    return w, probes, targets


@pytest.mark.parametrize("stream", ["0", "1"])
def test_one_adjoint_step_matches_cpu_adjoint(torch, monkeypatch, stream):
    from paper_2602_05017_gb300 import binding
    monkeypatch.setenv("BIOFVM_STREAM", stream)
    w, _, _ = _problem(1)
    p = oracle.Problem(**w.oracle_kwargs())
    gout = np.random.default_rng(2).normal(size=w.shape)
    gin_c, dD_c, dl_c, ds_c, du_c = p.adjoint_step(w.rho0, gout)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    saved = torch.empty(4 * sim.n_elem, dtype=torch.float64, device="cuda")
    sim.step_save(saved)
    g = torch.tensor(gout, device="cuda")
    dD = torch.zeros(w.ns, dtype=torch.float64, device="cuda")
    dl = torch.zeros_like(dD)
    ds = torch.zeros(w.n_agents * w.ns, dtype=torch.float64, device="cuda")
    du = torch.zeros_like(ds)
    sim.adjoint_step(g, g, dD, dl, ds, saved, dupt=du)
    sim.sync()
    # the saved step is also the forward step
    assert rel(sim.density(), p.step(w.rho0, 1)) <= 1e-12
    sim.close()
    assert rel(g.cpu().numpy(), gin_c) <= 1e-10
    assert rel(dD.cpu().numpy(), dD_c) <= 1e-10
    assert rel(dl.cpu().numpy(), dl_c) <= 1e-10
    assert rel(ds.cpu().numpy(), ds_c.reshape(-1)) <= 1e-10
    assert rel(du.cpu().numpy(), du_c.reshape(-1)) <= 1e-10


@pytest.mark.parametrize("stream", ["0", "1"])
def test_adjoint_with_dirichlet_nodes_matches_cpu_adjoint(torch, monkeypatch, stream):
    """Dirichlet nodes inside, on flagged faces and on agents' voxels: one adjoint step (the
    gradient zeroed at the nodes at every application, no secretion gradient where a node
    sits) and a 7-step loss against the CPU adjoint."""
    from paper_2602_05017_gb300 import binding
    monkeypatch.setenv("BIOFVM_STREAM", stream)
    w, probes, targets = _problem(31, shape=(14, 12, 10))
    rng = np.random.default_rng(32)
    voxel, sub, val = inputs.random_nodes(rng, 14 * 12 * 10, w.ns, 40)
    voxel[:5], sub[:5] = w.voxel[:5], 0
    w.dirichlet_nodes = (voxel, sub, val)
    p = oracle.Problem(**w.oracle_kwargs())
    gout = rng.normal(size=w.shape)
    gin_c, dD_c, dl_c, ds_c, du_c = p.adjoint_step(w.rho0, gout)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    saved = torch.empty(4 * sim.n_elem, dtype=torch.float64, device="cuda")
    sim.step_save(saved)
    g = torch.tensor(gout, device="cuda")
    dD = torch.zeros(w.ns, dtype=torch.float64, device="cuda")
    dl = torch.zeros_like(dD)
    ds = torch.zeros(w.n_agents * w.ns, dtype=torch.float64, device="cuda")
    du = torch.zeros_like(ds)
    sim.adjoint_step(g, g, dD, dl, ds, saved, dupt=du)
    sim.sync()
    assert rel(sim.density(), p.step(w.rho0, 1)) <= 1e-12
    sim.close()
    assert rel(g.cpu().numpy(), gin_c) <= 1e-10
    assert rel(dD.cpu().numpy(), dD_c) <= 1e-10
    assert rel(dl.cpu().numpy(), dl_c) <= 1e-10
    assert rel(ds.cpu().numpy(), ds_c.reshape(-1)) <= 1e-10
    assert rel(du.cpu().numpy(), du_c.reshape(-1)) <= 1e-10
    assert np.all(ds.cpu().numpy().reshape(w.n_agents, w.ns)[:5, 0] == 0.0)
    Lc, gc, dDc, dlc, dsc, duc = cpu_loss_and_grads(w, 7, probes, targets)
    Lg, gg, dDg, dlg, dsg, dug = gpu_loss_and_grads(torch, w, 7, probes, targets, ckpt=3)
    assert abs(Lg - Lc) <= 1e-12 * abs(Lc)
    for a, b in ((gg, gc), (dDg, dDc), (dlg, dlc), (dsg, dsc), (dug, duc)):
        assert rel(a, b) <= 1e-10


def test_anisotropic_adjoint_matches_cpu_adjoint(torch):
    """dx != dy != dz: one adjoint step (D gradient scaled per axis) against the CPU adjoint."""
    from paper_2602_05017_gb300 import binding
    w, _, _ = _problem(11, shape=(14, 12, 10))
    w.spacing = (11.0, 19.0, 27.0)
    p = oracle.Problem(**w.oracle_kwargs())
    gout = np.random.default_rng(12).normal(size=w.shape)
    gin_c, dD_c, dl_c, ds_c, du_c = p.adjoint_step(w.rho0, gout)
    sim = binding.BioFVM.from_workload(w, precision="fp64")
    saved = torch.empty(4 * sim.n_elem, dtype=torch.float64, device="cuda")
    sim.step_save(saved)
    g = torch.tensor(gout, device="cuda")
    dD = torch.zeros(w.ns, dtype=torch.float64, device="cuda")
    dl = torch.zeros_like(dD)
    ds = torch.zeros(w.n_agents * w.ns, dtype=torch.float64, device="cuda")
    du = torch.zeros_like(ds)
    sim.adjoint_step(g, g, dD, dl, ds, saved, dupt=du)
    sim.sync()
    sim.close()
    assert rel(g.cpu().numpy(), gin_c) <= 1e-10
    assert rel(dD.cpu().numpy(), dD_c) <= 1e-10
    assert rel(dl.cpu().numpy(), dl_c) <= 1e-10
    assert rel(ds.cpu().numpy(), ds_c.reshape(-1)) <= 1e-10
    assert rel(du.cpu().numpy(), du_c.reshape(-1)) <= 1e-10


@pytest.mark.parametrize("dirichlet", [False, True])
def test_multi_step_gradients_match_cpu_adjoint(torch, dirichlet):
    w, probes, targets = _problem(3, shape=(17, 14, 12), dirichlet=dirichlet)
    n = 7
    Lc, gc, dDc, dlc, dsc, duc = cpu_loss_and_grads(w, n, probes, targets)
    Lg, gg, dDg, dlg, dsg, dug = gpu_loss_and_grads(torch, w, n, probes, targets, ckpt=3)
    assert abs(Lg - Lc) <= 1e-12 * abs(Lc)
    assert rel(gg, gc) <= 1e-10
    assert rel(dDg, dDc) <= 1e-10
    assert rel(dlg, dlc) <= 1e-10
    assert rel(dsg, dsc) <= 1e-10
    assert rel(dug, duc) <= 1e-10


def test_gradients_are_bit_reproducible(torch):
    w, probes, targets = _problem(4)
    a = gpu_loss_and_grads(torch, w, 4, probes, targets)
    b = gpu_loss_and_grads(torch, w, 4, probes, targets)
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)


def test_gradients_match_central_fd_on_the_gpu(torch):
    """FD of the GPU FP64 forward (h = 1e-6 relative) for D, lambda, secretion and uptake rates
    and rho0."""
    from paper_2602_05017_gb300 import binding
    w, probes, targets = _problem(5, shape=(12, 10, 9), n_agents=12)
    n = 5
    L0, g0, dD, dl, ds, du = gpu_loss_and_grads(torch, w, n, probes, targets)

    def loss_of(ww):
        sim = binding.BioFVM.from_workload(ww, precision="fp64")
        sim.step(n)
        fin = sim.density().reshape(-1)
        sim.close()
        return float(((fin[probes] - targets) ** 2).sum())

    def fd(name, idx, scale=1e-6):
        base = np.array(getattr(w, name), dtype=np.float64)
        h = scale * max(1.0, abs(base.reshape(-1)[idx]))
        up, dn = copy.deepcopy(w), copy.deepcopy(w)
        bu, bd = base.copy(), base.copy()
        bu.reshape(-1)[idx] += h
        bd.reshape(-1)[idx] -= h
        setattr(up, name, bu)
        setattr(dn, name, bd)
        return (loss_of(up) - loss_of(dn)) / (2 * h), h

    def check(grad, name, idx):
        v, h = fd(name, idx)
        noise = 8 * np.finfo(float).eps * abs(L0) / h
        assert grad == pytest.approx(v, rel=1e-6, abs=noise), (name, idx)

    for s in range(w.ns):
        check(dD[s], "D", s)
        check(dl[s], "lam", s)
    for i in (0, 5, 13, 22):
        check(ds.reshape(-1)[i], "secretion", i)
    # uptake rates: the sinks (rates must stay >= 0, so not at the sources' zero uptake)
    for i in np.nonzero(np.asarray(w.uptake).reshape(-1) > 0)[0][:4]:
        check(du.reshape(-1)[i], "uptake", i)
    for e in np.random.default_rng(6).choice(w.rho0.size, 6, replace=False):
        check(g0.reshape(-1)[e], "rho0", e)


@pytest.mark.parametrize("stream32", ["0", "1"])
def test_fp32_adjoint_tracks_fp64(torch, monkeypatch, stream32):
    monkeypatch.setenv("BIOFVM_STREAM32", stream32)
    w, probes, targets = _problem(7, shape=(20, 16, 14))
    _, gc, dDc, dlc, dsc, duc = cpu_loss_and_grads(w, 6, probes, targets)
    _, gg, dDg, dlg, dsg, dug = gpu_loss_and_grads(torch, w, 6, probes, targets, prec="fp32")
    assert rel(gg, gc) <= 1e-4
    assert rel(dDg, dDc) <= 1e-4
    assert rel(dlg, dlc) <= 1e-4
    assert rel(dsg, dsc) <= 1e-4
    assert rel(dug, duc) <= 1e-4


def test_workload5_reduced_matches_cpu_adjoint(torch):
    """The adjoint workload's recipe (1% secreting voxels, probes) at 40^3 x 2, 40 steps,
    checkpoints every 20."""
    w = inputs.workload(5, shape=(40, 40, 40))
    probes, targets = w.extra["probe_index"], w.extra["probe_target"]
    n = 40
    Lc, gc, dDc, dlc, dsc, duc = cpu_loss_and_grads(w, n, probes, targets)
    Lg, gg, dDg, dlg, dsg, dug = gpu_loss_and_grads(torch, w, n, probes, targets, ckpt=20)
    assert rel(gg, gc) <= 1e-10
    assert rel(dDg, dDc) <= 1e-10
    assert rel(dlg, dlc) <= 1e-10
    assert rel(dsg, dsc) <= 1e-10
    assert rel(dug, duc) <= 1e-10


# Bound on the FP64 path's normwise forward error after the 200 steps of workload 5: the bench
# measures about 1.2e-13 after 100 steps on the 50^3 workload (r = 2.5, the largest r of
# workload 5) and 5e-14 on a 100-step 400 x 400 x 8 slab; linear growth to 200 steps, rounded up.
EPS_FORWARD_200 = 3e-13


@pytest.mark.slow
def test_workload5_full_size_gradients_match_fd(torch):
    """128^3 x 2, 200 steps, checkpoints every 20: gradients from the GPU adjoint against central
    FD of the GPU FP64 forward, for D, lambda, secretion rates and initial-field entries (the
    workload has no uptake; uptake gradients are checked against the CPU adjoint and FD on
    smaller problems).

    FD: Richardson-extrapolated central differences (4 f(h) - f(2h)) / 3, h = 1e-4 relative,
    whose truncation error is O(h^4).  Each loss L = sum_p (rho_p - t_p)^2 carries a rounding
    error of at most dL = 2 eps max|rho| sum_p |rho_p - t_p| (eps: EPS_FORWARD_200), which the
    combination of four losses turns into at most 1.5 dL / h; the tolerance is 1e-6 relative
    plus that fixed bound."""
    from paper_2602_05017_gb300 import binding
    w = inputs.workload(5)
    probes, targets = w.extra["probe_index"], w.extra["probe_target"]
    n = w.n_steps
    L0, g0, dD, dl, ds, du = gpu_loss_and_grads(torch, w, n, probes, targets, ckpt=20)

    def final(ww):
        sim = binding.BioFVM.from_workload(ww, precision="fp64")
        sim.step(n)
        fin = sim.density().reshape(-1)
        sim.close()
        return fin

    def loss_of(ww):
        return float(((final(ww)[probes] - targets) ** 2).sum())

    fin0 = final(w)
    dL = 2 * EPS_FORWARD_200 * np.abs(fin0).max() * np.abs(fin0[probes] - targets).sum()

    def fd(name, idx, h):
        base = np.array(getattr(w, name), dtype=np.float64)
        up, dn = copy.deepcopy(w), copy.deepcopy(w)
        bu, bd = base.copy(), base.copy()
        bu.reshape(-1)[idx] += h
        bd.reshape(-1)[idx] -= h
        setattr(up, name, bu)
        setattr(dn, name, bd)
        return (loss_of(up) - loss_of(dn)) / (2 * h)

    def check(grad, name, idx, scale=1e-4):
        base = np.array(getattr(w, name)).reshape(-1)[idx]
        h = scale * max(1.0, abs(base))
        rich = (4 * fd(name, idx, h) - fd(name, idx, 2 * h)) / 3
        assert grad == pytest.approx(rich, rel=1e-6, abs=1.5 * dL / h), (name, idx, grad, rich)

    for s in range(w.ns):
        check(dD[s], "D", s)
        check(dl[s], "lam", s)
    rng = np.random.default_rng(8)
    for i in rng.choice(ds.size, 4, replace=False):
        check(ds.reshape(-1)[i], "secretion", i)
    near = probes[:3]  # initial-field entries that sit on probes: large, well-conditioned
    for e in near:
        check(g0.reshape(-1)[e], "rho0", e)
