"""biofvm_param_grad_noalloc: the allocation-free variant of the adjoint's parameter-gradient
reduction, for callers that cannot allocate device memory (a framework that owns all device
memory through its own pool, a fixed memory budget, a loop where allocating is not allowed).

It is checked through the C ABI against the existing entry point, biofvm_adjoint_step, whose
dD / dlambda are the same three reductions (one per adjoint sweep, Z, Y, X): the adjoint sweeps
are replayed stage by stage on a second handle and each one is reduced with the
allocation-free call, on two calls in a row.  This file is collected last on purpose; it also
passes alone in a fresh process (its first call does the per-device set-up).
"""
import ctypes

import numpy as np
import pytest

from paper_2602_05017_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("spacing", [None, (20.0, 13.0, 31.0)], ids=["isotropic", "anisotropic"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_reduction_matches_adjoint_step_on_two_calls(prec, spacing):
    import torch

    from paper_2602_05017_gb300 import binding
    lib = binding.load()
    rng = np.random.default_rng(31)
    w = inputs.random_problem(rng, 21, 17, 13, 3, n_agents=30)  # zero flux: B is the identity
    w.spacing = spacing
    h3 = spacing or (w.dx, w.dx, w.dx)  # the spacing each axis's reduction takes
    fd = torch.float64 if prec == "fp64" else torch.float32
    code = binding.FP64 if prec == "fp64" else binding.FP32
    stream = torch.cuda.current_stream().cuda_stream

    sim = binding.BioFVM.from_workload(w, precision=prec)
    n = sim.n_elem
    saved = torch.empty(4 * n, dtype=fd, device="cuda")
    sim.step_save(saved)
    gout = torch.tensor(rng.normal(size=w.shape), dtype=fd, device="cuda")
    gin = torch.empty_like(gout)
    dD_ref = torch.zeros(w.ns, dtype=torch.float64, device="cuda")
    dl_ref = torch.zeros_like(dD_ref)
    sim.adjoint_step(gout.clone(), gin, dD_ref, dl_ref, None, saved)
    sim.sync()

    aux = binding.BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, precision=prec)
    if spacing is not None:
        aux.set_spacing(*spacing)
    for _ in range(2):  # two calls in a row share (and overwrite) the static scratch
        dD = torch.zeros(w.ns, dtype=torch.float64, device="cuda")
        dl = torch.zeros_like(dD)
        aux.set_density(gout)
        for axis, stage, k in ((2, 7, 3), (1, 6, 2), (0, 5, 1)):  # Z^-1, Y^-1, X^-1 alone
            aux.run_stage(stage)
            mu = aux.field_tensor()
            u = saved[k * n:(k + 1) * n]
            st = lib.biofvm_param_grad_noalloc(
                ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(u.data_ptr()), w.nx, w.ny, w.nz,
                w.ns, axis, code, w.dt, h3[axis], ctypes.c_void_p(dD.data_ptr()),
                ctypes.c_void_p(dl.data_ptr()), stream)
            assert st == binding.OK, lib.biofvm_last_error().decode()
        torch.cuda.synchronize()
        assert rel(dD.cpu().numpy(), dD_ref.cpu().numpy()) <= TOL[prec]
        assert rel(dl.cpu().numpy(), dl_ref.cpu().numpy()) <= TOL[prec]
    aux.close()
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    from paper_2602_05017_gb300 import binding
    lib = binding.load()
    st = lib.biofvm_param_grad_noalloc(ctypes.c_void_p(8), ctypes.c_void_p(8), 4, 4, 4, 33, 0,
                                       binding.FP64, 0.01, 20.0, ctypes.c_void_p(8),
                                       ctypes.c_void_p(8), 0)
    assert st == binding.ERR_ARG
    assert "32" in lib.biofvm_last_error().decode()
