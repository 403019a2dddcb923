"""The C-ABI library loads, exports what include/biofvm.h declares, and validates arguments
on the host before touching a device (CPU only; no compute call needs a GPU here)."""
import ctypes

import numpy as np
import pytest

from paper_2602_05017_gb300 import binding
from paper_2602_05017_gb300 import build as libbuild


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = binding.declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def _create(lib, nx=4, ny=4, nz=4, ns=1, dx=20.0, dt=0.01, D=(1e5,), lam=(0.1,), prec=0,
            bc=None):
    g = binding.Grid(nx, ny, nz, ns)
    D = np.asarray(D, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    h = ctypes.c_void_p()
    st = lib.biofvm_create(ctypes.byref(g), dx, dt,
                           D.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           bc, prec, 0, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw", [
    dict(nx=0), dict(ny=-1), dict(nz=0), dict(ns=0, D=(), lam=()),
    dict(ns=33, D=(1.0,) * 33, lam=(0.0,) * 33), dict(dx=0.0), dict(dx=float("nan")),
    dict(dt=-1.0), dict(D=(-1.0,)), dict(lam=(-0.5,)), dict(D=(float("inf"),)), dict(prec=7),
])
def test_create_rejects_bad_arguments(lib, kw):
    st, h = _create(lib, **kw)
    assert st == binding.ERR_ARG
    assert not h.value
    assert lib.biofvm_last_error().decode() != ""


def test_create_without_a_device_fails_cleanly(lib):
    """Valid arguments reach the device checks; with no GPU the call reports ERR_CUDA."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = _create(lib)
    assert st == binding.ERR_CUDA
    assert not h.value
    assert "device" in lib.biofvm_last_error().decode().lower()


def test_null_handles_are_rejected(lib):
    assert lib.biofvm_step(None, 1) == binding.ERR_ARG
    assert lib.biofvm_sync(None) == binding.ERR_ARG
    assert lib.biofvm_run_stage(None, 0) == binding.ERR_ARG
    assert lib.biofvm_launches_per_step(None) == 0
    assert lib.biofvm_set_dirichlet_nodes(None, 0, None, None, None) == binding.ERR_ARG
    assert lib.biofvm_set_spacing(None, 1.0, 1.0, 1.0) == binding.ERR_ARG
    assert lib.biofvm_set_sources(None, 0, None, None, None, None, None) == binding.ERR_ARG
    lib.biofvm_destroy(None)  # no-op


def test_python_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        binding.load()
