"""Python binding of libbiofvm (ctypes): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module turns torch
tensors / numpy arrays into pointers and status codes into exceptions.  PyTorch supplies
device memory and the CUDA stream.  Importing it loads ``libbiofvm.so`` and raises if the
library has not been built (``python -m paper_2602_05017_gb300.build``): there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbiofvm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "biofvm.h")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = range(6)
FP64, FP32, BF16, FP16 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "fp16": FP16}
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_TIMEOUT",
                5: "ERR_STATE"}


class BioFVMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("n_sub", ctypes.c_int)]


class Boundary(ctypes.Structure):
    _fields_ = [("dirichlet_on", ctypes.POINTER(ctypes.c_uint8)),
                ("dirichlet_value", ctypes.POINTER(ctypes.c_double))]


def declared_functions(header=HEADER):
    """Names of the functions include/biofvm.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(biofvm_[a-z_0-9]+)\s*\(", text)))


_lib = None


def load():
    """Load libbiofvm.so (raises if it is missing) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_2602_05017_gb300.build`"
                          " (the CUDA library is the only compute path)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    st = ctypes.c_int
    sig = {
        "biofvm_create": (st, [ctypes.POINTER(Grid), ctypes.c_double, ctypes.c_double, dp, dp,
                               ctypes.POINTER(Boundary), ctypes.c_int, ctypes.c_size_t,
                               ctypes.POINTER(vp)]),
        "biofvm_set_density": (st, [vp, vp, ctypes.c_int]),
        "biofvm_set_sources": (st, [vp, ctypes.c_int64, i64p, dp, dp, dp, dp]),
        "biofvm_reserve_agents": (st, [vp, ctypes.c_int64]),
        "biofvm_set_sources_device": (st, [vp, ctypes.c_int64, vp, vp, vp, vp, vp]),
        "biofvm_step": (st, [vp, ctypes.c_int]),
        "biofvm_density": (st, [vp, vp, ctypes.c_int]),
        "biofvm_set_params": (st, [vp, dp, dp]),
        "biofvm_run_stage": (st, [vp, ctypes.c_int]),
        "biofvm_set_spacing": (st, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        "biofvm_set_dirichlet_nodes": (st, [vp, ctypes.c_int64, i64p,
                                            ctypes.POINTER(ctypes.c_int32), dp]),
        "biofvm_sync": (st, [vp]),
        "biofvm_density_ptr": (st, [vp, ctypes.POINTER(vp)]),
        "biofvm_launches_per_step": (ctypes.c_int, [vp]),
        "biofvm_describe": (st, [vp, ctypes.c_char_p, ctypes.c_size_t]),
        "biofvm_step_save": (st, [vp, vp]),
        "biofvm_adjoint_step": (st, [vp, vp, vp, vp, vp, vp, vp]),
        "biofvm_adjoint_step_rates": (st, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "biofvm_batch_create": (st, [ctypes.c_int, ctypes.POINTER(Grid), dp, dp, dp, dp,
                                     ctypes.c_int, ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(vp)]),
        "biofvm_batch_env": (st, [vp, ctypes.c_int, ctypes.POINTER(vp)]),
        "biofvm_batch_step": (st, [vp, ctypes.c_int]),
        "biofvm_batch_sync": (st, [vp]),
        "biofvm_batch_grid": (ctypes.c_int, [vp]),
        "biofvm_batch_mode": (ctypes.c_int, [vp]),
        "biofvm_batch_test_stall": (st, [vp, ctypes.c_int]),
        "biofvm_batch_set_tiles": (st, [vp, ctypes.POINTER(ctypes.c_int)]),
        "biofvm_batch_destroy": (None, [vp]),
        "biofvm_param_grad_noalloc": (st, [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double, vp, vp,
                                           ctypes.c_size_t]),
        "biofvm_probe_fma_rate": (st, [ctypes.c_int, ctypes.c_size_t, dp]),
        "biofvm_destroy": (None, [vp]),
        "biofvm_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def probe_fma_rate(precision="fp64", stream=None):
    """FMA/s of the current device in FP64 or FP32 (biofvm_probe_fma_rate)."""
    lib = load()
    out = ctypes.c_double()
    _check(lib.biofvm_probe_fma_rate(FP64 if precision == "fp64" else FP32,
                                     _current_stream() if stream is None else int(stream),
                                     ctypes.byref(out)), lib)
    return out.value


def _check(status, lib=None):
    if status != OK:
        lib = lib or load()
        raise BioFVMError(status, lib.biofvm_last_error().decode())


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0


class BioFVM:
    """One microenvironment on the GPU behind the C ABI (see include/biofvm.h).

    Field layout ``[nz, ny, nx, n_sub]``; ``precision`` is "fp64", "fp32", or "bf16" / "fp16"
    (16-bit storage, FP32 arithmetic: fields are exchanged as torch bfloat16 / float16 tensors;
    numpy float16 also works for "fp16").
    """

    def __init__(self, nx, ny, nz, n_sub, dx, dt, D, lam, dirichlet_on=None,
                 dirichlet_value=None, precision="fp64", stream=None, _handle=None):
        self.lib = load()
        self.shape = (int(nz), int(ny), int(nx), int(n_sub))
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        self.precision = precision
        self.dtype = {"fp64": np.float64, "fp32": np.float32, "fp16": np.float16,
                      "bf16": None}[precision]
        self.n_elem = int(np.prod(self.shape))
        self._owned = _handle is None
        if _handle is not None:  # an environment of a batch (the batch owns it)
            self.stream = stream
            self.h = _handle
            return
        grid = Grid(int(nx), int(ny), int(nz), int(n_sub))
        D = _f64(D, n_sub)
        lam = _f64(lam, n_sub)
        bc = None
        if dirichlet_on is not None:
            self._on = np.ascontiguousarray(np.asarray(dirichlet_on, dtype=np.uint8).reshape(-1))
            self._val = _f64(dirichlet_value, n_sub)
            bc = Boundary(self._on.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _dptr(self._val))
        self.stream = _current_stream() if stream is None else int(stream)
        h = ctypes.c_void_p()
        st = self.lib.biofvm_create(ctypes.byref(grid), float(dx), float(dt), _dptr(D), _dptr(lam),
                                    ctypes.byref(bc) if bc is not None else None,
                                    PRECISIONS[precision], self.stream, ctypes.byref(h))
        _check(st, self.lib)
        self.h = h

    # -- field ------------------------------------------------------------------------------
    def set_density(self, rho):
        """rho: torch tensor (CUDA or CPU) or numpy array with n_elem elements."""
        try:
            import torch
            if isinstance(rho, torch.Tensor) or self.dtype is None:
                t = rho if isinstance(rho, torch.Tensor) else torch.as_tensor(np.asarray(rho))
                t = t.detach().to(dtype=self._field_dtype()).contiguous()
                if t.numel() != self.n_elem:
                    raise ValueError("field has the wrong size")
                _check(self.lib.biofvm_set_density(self.h, ctypes.c_void_p(t.data_ptr()),
                                                   1 if t.is_cuda else 0), self.lib)
                if t.is_cuda:
                    self._keep = t  # the copy is stream-ordered; keep the source alive
                return
        except ImportError:  # pragma: no cover
            pass
        a = np.ascontiguousarray(np.asarray(rho, dtype=self.dtype))
        if a.size != self.n_elem:
            raise ValueError("field has the wrong size")
        _check(self.lib.biofvm_set_density(self.h, a.ctypes.data_as(ctypes.c_void_p), 0), self.lib)

    def density(self, out=None):
        """Copy the field out: into ``out`` (torch tensor or numpy array) or a new numpy array."""
        if out is None:
            if self.dtype is None:  # bf16: a torch CPU tensor (numpy has no bfloat16)
                import torch
                out = torch.empty(self.shape, dtype=torch.bfloat16)
            else:
                out = np.empty(self.shape, dtype=self.dtype)
        try:
            import torch
            if isinstance(out, torch.Tensor):
                assert out.is_contiguous() and out.numel() == self.n_elem
                _check(self.lib.biofvm_density(self.h, ctypes.c_void_p(out.data_ptr()),
                                               1 if out.is_cuda else 0), self.lib)
                return out
        except ImportError:  # pragma: no cover
            pass
        assert out.flags.c_contiguous and out.size == self.n_elem and out.dtype == self.dtype
        _check(self.lib.biofvm_density(self.h, out.ctypes.data_as(ctypes.c_void_p), 0), self.lib)
        return out

    def density_ptr(self):
        p = ctypes.c_void_p()
        _check(self.lib.biofvm_density_ptr(self.h, ctypes.byref(p)), self.lib)
        return p.value

    def field_tensor(self):
        """Zero-copy torch view of the library-owned device field (valid until close)."""
        import torch

        class _CAI:
            pass
        obj = _CAI()
        typestr = {"fp64": "<f8", "fp32": "<f4", "fp16": "<f2", "bf16": "<i2"}[self.precision]
        obj.__cuda_array_interface__ = {
            "shape": self.shape, "typestr": typestr,
            "data": (self.density_ptr(), False), "version": 3, "strides": None,
            "stream": None}
        t = torch.as_tensor(obj, device="cuda")
        return t.view(torch.bfloat16) if self.precision == "bf16" else t

    # -- agents and parameters --------------------------------------------------------------
    def set_sources(self, voxel, secretion=None, target=None, uptake=None, weight=None):
        vox = np.ascontiguousarray(np.asarray(voxel, dtype=np.int64)).reshape(-1)
        n = vox.size
        ns = self.shape[3]
        arrs = [None if a is None else _f64(a, n * ns) for a in (secretion, target, uptake)]
        w = None if weight is None else _f64(weight, n)
        _check(self.lib.biofvm_set_sources(
            self.h, n, vox.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if n else None,
            *[_dptr(a) for a in arrs], _dptr(w)), self.lib)

    def reserve_agents(self, n_max):
        """Device buffers for up to n_max agents given by set_sources_device."""
        _check(self.lib.biofvm_reserve_agents(self.h, int(n_max)), self.lib)

    def set_sources_device(self, voxel, secretion=None, target=None, uptake=None, weight=None):
        """Agents from CUDA tensors (voxel int64 [n]; rates float64 [n, n_sub]; weight [n]),
        rebuilt into source lists on the device, stream-ordered (the tensors are kept alive
        until the next call)."""
        import torch
        ns = self.shape[3]
        vox = voxel.contiguous()
        n = vox.numel()
        if vox.dtype != torch.int64 or not vox.is_cuda:
            raise ValueError("voxel must be a CUDA int64 tensor")
        keep = [vox]

        def rate(a, count):
            if a is None:
                return None
            t = a.contiguous()
            if t.dtype != torch.float64 or not t.is_cuda or t.numel() != count:
                raise ValueError(f"expected a CUDA float64 tensor of {count} values")
            keep.append(t)
            return ctypes.c_void_p(t.data_ptr())
        args = [rate(secretion, n * ns), rate(target, n * ns), rate(uptake, n * ns),
                rate(weight, n)]
        _check(self.lib.biofvm_set_sources_device(self.h, n, ctypes.c_void_p(vox.data_ptr()),
                                                  *args), self.lib)
        self._keep_agents = keep

    def set_dirichlet_nodes(self, voxel, substrate, value):
        """Dirichlet nodes (voxel, substrate, value), overwritten at every Dirichlet application
        after the flagged faces; a repeated (voxel, substrate) keeps its last value.  Empty
        arrays remove them."""
        vox = np.ascontiguousarray(np.asarray(voxel, dtype=np.int64)).reshape(-1)
        sub = np.ascontiguousarray(np.asarray(substrate, dtype=np.int32)).reshape(-1)
        val = _f64(value, vox.size)
        if sub.size != vox.size:
            raise ValueError("voxel and substrate arrays differ in length")
        n = vox.size
        _check(self.lib.biofvm_set_dirichlet_nodes(
            self.h, n, vox.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if n else None,
            sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if n else None,
            _dptr(val) if n else None), self.lib)

    def set_params(self, D, lam):
        ns = self.shape[3]
        _check(self.lib.biofvm_set_params(self.h, _dptr(_f64(D, ns)), _dptr(_f64(lam, ns))),
               self.lib)

    # -- stepping ---------------------------------------------------------------------------
    def step(self, n_steps=1):
        _check(self.lib.biofvm_step(self.h, int(n_steps)), self.lib)

    def _dev(self, t, n, dtype):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise ValueError("expected a contiguous CUDA tensor")
        if t.dtype != dtype or t.numel() != n:
            raise ValueError(f"expected {n} elements of {dtype}, got {t.numel()} of {t.dtype}")
        return ctypes.c_void_p(t.data_ptr())

    def _field_dtype(self):
        import torch
        return {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16,
                "fp16": torch.float16}[self.precision]

    def step_save(self, saved):
        """One step that also writes the adjoint's forward states into `saved` (4 fields)."""
        _check(self.lib.biofvm_step_save(self.h, self._dev(saved, 4 * self.n_elem,
                                                              self._field_dtype())), self.lib)

    def adjoint_step(self, grad_out, grad_in, dD, dlam, dsec, saved, dupt=None):
        """Reverse mode of one step; accumulates into dD, dlam (and dsec, dupt if given: the
        agents' secretion and uptake rates), FP64 CUDA tensors."""
        import torch
        fd = self._field_dtype()
        ns = self.shape[3]
        _check(self.lib.biofvm_adjoint_step_rates(
            self.h, self._dev(grad_out, self.n_elem, fd), self._dev(grad_in, self.n_elem, fd),
            self._dev(dD, ns, torch.float64), self._dev(dlam, ns, torch.float64),
            None if dsec is None else self._dev(dsec, dsec.numel(), torch.float64),
            None if dupt is None else self._dev(dupt, dupt.numel(), torch.float64),
            self._dev(saved, 4 * self.n_elem, fd)), self.lib)

    def set_spacing(self, dx, dy, dz):
        """Anisotropic grid: voxel spacing along x, y, z (recomputes the constants)."""
        _check(self.lib.biofvm_set_spacing(self.h, float(dx), float(dy), float(dz)), self.lib)

    def run_stage(self, stage):
        _check(self.lib.biofvm_run_stage(self.h, int(stage)), self.lib)

    def sync(self):
        _check(self.lib.biofvm_sync(self.h), self.lib)

    def launches_per_step(self):
        return int(self.lib.biofvm_launches_per_step(self.h))

    def describe(self):
        """The kernels biofvm_step runs for this handle (biofvm_describe)."""
        buf = ctypes.create_string_buffer(256)
        _check(self.lib.biofvm_describe(self.h, buf, len(buf)), self.lib)
        return buf.value.decode()

    def close(self):
        if getattr(self, "h", None):
            if self._owned:
                self.lib.biofvm_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    @classmethod
    def from_workload(cls, w, precision="fp64", stream=None):
        """Create, upload the initial field and the agents of an ``inputs.Workload``."""
        sim = cls(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam, w.dirichlet_on,
                  w.dirichlet_value, precision=precision, stream=stream)
        if w.spacing is not None:
            sim.set_spacing(*w.spacing)
        if w.rho0 is not None:
            sim.set_density(w.rho0)
        if w.dirichlet_nodes is not None:
            sim.set_dirichlet_nodes(*w.dirichlet_nodes)
        if w.n_agents:
            sim.set_sources(w.voxel, w.secretion, w.target, w.uptake, w.weight)
        return sim


class BioFVMBatch:
    """Many microenvironments advanced together: one persistent launch per step() call, or one
    graph of per-environment sweep launches per step (large environments).

    envs: list of ``inputs.Workload`` (grids, dx, dt, D, lambda; zero-flux).  tile_m: optional
    [n_env][3] chunk lengths (x, y, z) of the persistent kernel -- from ``autotune`` -- else
    library defaults.  mode: None (the library's choice), "persistent" or "graph" (passed to
    biofvm_batch_create through BIOFVM_BATCH_MODE).
    """

    def __init__(self, envs, precision="fp32", tile_m=None, stream=None, mode=None):
        self.lib = load()
        if mode is not None and mode not in ("persistent", "graph"):
            raise ValueError("mode must be None, 'persistent' or 'graph'")
        n = len(envs)
        grids = (Grid * n)(*[Grid(w.nx, w.ny, w.nz, w.ns) for w in envs])
        dx = _f64([w.dx for w in envs])
        dt = _f64([w.dt for w in envs])
        D = _f64(np.concatenate([np.asarray(w.D, dtype=np.float64) for w in envs]))
        lam = _f64(np.concatenate([np.asarray(w.lam, dtype=np.float64) for w in envs]))
        tm = None
        if tile_m is not None:
            self._tm = np.ascontiguousarray(np.asarray(tile_m, dtype=np.int32).reshape(n, 3))
            tm = self._tm.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        self.stream = _current_stream() if stream is None else int(stream)
        h = ctypes.c_void_p()
        saved = os.environ.get("BIOFVM_BATCH_MODE")
        if mode is not None:
            os.environ["BIOFVM_BATCH_MODE"] = mode
        try:
            _check(self.lib.biofvm_batch_create(n, grids, _dptr(dx), _dptr(dt), _dptr(D),
                                                _dptr(lam), FP64 if precision == "fp64" else FP32,
                                                self.stream, tm, ctypes.byref(h)), self.lib)
        finally:
            if mode is not None:
                if saved is None:
                    os.environ.pop("BIOFVM_BATCH_MODE", None)
                else:
                    os.environ["BIOFVM_BATCH_MODE"] = saved
        self.h = h
        self.precision = precision
        self.envs = []
        for e, w in enumerate(envs):
            eh = ctypes.c_void_p()
            _check(self.lib.biofvm_batch_env(self.h, e, ctypes.byref(eh)), self.lib)
            self.envs.append(BioFVM(w.nx, w.ny, w.nz, w.ns, w.dx, w.dt, w.D, w.lam,
                                    precision=precision, stream=self.stream, _handle=eh))

    @property
    def n_vs(self):
        return sum(e.n_elem for e in self.envs)

    def step(self, n_steps=1):
        _check(self.lib.biofvm_batch_step(self.h, int(n_steps)), self.lib)

    def sync(self):
        _check(self.lib.biofvm_batch_sync(self.h), self.lib)

    def grid(self):
        return int(self.lib.biofvm_batch_grid(self.h))

    def mode(self):
        """'persistent' or 'graph' (biofvm_batch_mode)."""
        return "graph" if self.lib.biofvm_batch_mode(self.h) == 1 else "persistent"

    def set_tiles(self, tile_m):
        """Re-partition every environment with [n_env][3] chunk lengths (fields kept)."""
        tm = np.ascontiguousarray(np.asarray(tile_m, dtype=np.int32).reshape(len(self.envs), 3))
        _check(self.lib.biofvm_batch_set_tiles(self.h, tm.ctypes.data_as(
            ctypes.POINTER(ctypes.c_int))), self.lib)

    def test_stall(self, on=True):
        """Failure-detection hook: the next launches hit a bounded wait that expires."""
        _check(self.lib.biofvm_batch_test_stall(self.h, 1 if on else 0), self.lib)

    def close(self):
        if getattr(self, "h", None):
            for e in self.envs:
                e.h = None
            self.lib.biofvm_batch_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
