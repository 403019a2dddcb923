"""Fields stored in 16 bits (bfloat16, IEEE half) with FP32 arithmetic, through the C ABI,
against the FP64 oracle on the same (16-bit-rounded) initial field.

Error bound: a step stores each element at most four times (after the source update and
after each of the three solves), each store rounds to the nearest 16-bit value (relative error
at most u: 2^-8 for bf16, 2^-11 for fp16), and each solve is a contraction in the max norm
(the inverse of an M-matrix whose rows sum to at least 1), so a rounding error is never
amplified by later sweeps: after s steps the normwise error is at most 4 s u, plus the FP32
arithmetic's 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_2602_05017_gb300 import inputs

pytestmark = pytest.mark.gpu

UNIT_ROUNDOFF = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -11}


@pytest.fixture(scope="module")
def binding():
    from paper_2602_05017_gb300 import binding as b
    return b


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def as_f64(field):
    """density() returns a torch bfloat16 tensor (bf16) or a numpy float16 array (fp16)."""
    return field.double().numpy() if hasattr(field, "double") else field.astype(np.float64)


def rounded(a, prec):
    import torch
    t = torch.as_tensor(a).to(torch.bfloat16 if prec == "bf16" else torch.float16)
    return t, t.double().numpy()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("shape", [(40, 36, 28, 4), (64, 30, 20, 2), (24, 20, 18, 1),
                                   (16, 12, 1100, 1)],
                         ids=lambda s: "x".join(map(str, s)))
def test_step_matches_oracle_within_the_storage_bound(binding, prec, shape):
    nx, ny, nz, ns = shape
    rng = np.random.default_rng(nx * 7 + ns)
    w = inputs.random_problem(rng, nx, ny, nz, ns, n_agents=max(1, nx * ny * nz // 30),
                              dirichlet=True)
    t0, r0 = rounded(w.rho0, prec)
    steps = 3
    ref = oracle.Problem(**w.oracle_kwargs()).step(r0, steps)
    sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, w.dirichlet_on,
                         w.dirichlet_value, precision=prec)
    sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
    sim.set_density(t0.cuda())
    sim.step(steps)
    got = as_f64(sim.density())
    sim.close()
    err = rel_err(got, ref)
    assert err <= 4 * steps * UNIT_ROUNDOFF[prec] + 1e-5, err


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_workload2_reduced_100_steps(binding, prec):
    """The 400^3 x 4 recipe at 48 x 40 x 36 with 3000 agents, 100 steps."""
    w = inputs.workload(2, shape=(48, 40, 36), n_agents=3000)
    t0, r0 = rounded(w.rho0, prec)
    ref = oracle.Problem(**w.oracle_kwargs()).step(r0, w.n_steps)
    sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, precision=prec)
    sim.set_sources(w.voxel, w.secretion, w.target, w.uptake)
    sim.set_density(t0.cuda())
    sim.step(w.n_steps)
    got = as_f64(sim.density())
    sim.close()
    assert rel_err(got, ref) <= 4 * w.n_steps * UNIT_ROUNDOFF[prec] + 1e-5


def test_16bit_handles_refuse_what_they_do_not_run(binding):
    import torch
    rng = np.random.default_rng(2)
    w = inputs.random_problem(rng, 16, 10, 8, 2)
    with pytest.raises(binding.BioFVMError) as e:  # nx * n_sub = 10: not a multiple of 8
        binding.BioFVM(5, 10, 8, 2, w.dx, w.dt, w.D, w.lam, precision="bf16")
    assert e.value.status == binding.ERR_ARG
    sim = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, precision="fp16")
    for call in (lambda: sim.set_dirichlet_nodes([3], [0], [1.0]),
                 lambda: sim.run_stage(0),
                 lambda: sim.step_save(torch.zeros(4 * sim.n_elem, dtype=torch.float16,
                                                   device="cuda"))):
        with pytest.raises(binding.BioFVMError) as e:
            call()
        assert e.value.status == binding.ERR_STATE
    sim.close()
