"""FP64 CPU oracle of the BioFVM-B diffusion-decay step (ctypes over biofvm_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the library in ``paper_2602_05017_gb300`` never
does, and it shares no code with it.

Every function follows one passage of the paper (arXiv 2602.05017):
  * ``axis_coefficients`` -- Appendix A (a, b, c, constant_c, denom), with the readings
    a_i = c_i = -D dt/dx^2 and b = 1 + lambda dt/3 on a one-voxel axis;
  * ``thomas``            -- the TDMA of Sect. 2.1 (forward: divide, backward: negated axpy);
  * ``sweep``             -- Algorithm 1 for one dimension over every line and substrate;
  * ``dirichlet``         -- one of the four Dirichlet applications of the 7-stage solver (Sect. 2):
    the flagged faces, then the Dirichlet nodes (listed voxels, in list order);
  * ``sources``           -- the cell source/uptake update of the end-to-end run (Sect. 5.3),
    in the implicit form of the cited BioFVM, agents sharing a voxel aggregated;
  * ``step``              -- Src, B, X^-1, B, Y^-1, B, Z^-1, B, repeated n_steps times;
  * ``adjoint_step``      -- reverse mode of ``step`` (symmetric 1D operators: A^-T = A^-1).

Pins (tests/test_oracle_pins.py) tie it to dense LU solves, closed forms (uniform decay,
cosine modes, D = 0), exact invariants (mass, maximum principle, Dirichlet steady state,
sweep-order independence) and finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "biofvm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64p = ctypes.POINTER(ctypes.c_longlong)


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree bit for bit).

    parallel=True builds the OpenMP copy (liboracle_omp.so): the same source with its line
    loops split over the host's cores, the paper-style CPU rate; it gives the same bits."""
    lib = _LIB_OMP if parallel else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-shared", "-fPIC"]
            + (["-fopenmp"] if parallel else []) + [_SRC, "-o", tmp])
        os.replace(tmp, lib)
    return lib


_libs = {}


def _get(parallel=False):
    if parallel not in _libs:
        lib = ctypes.CDLL(build(parallel=parallel))
        i, d, L = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        lib.oracle_axis_coefficients.argtypes = [i, d, d, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_thomas.argtypes = [i, _dp, _dp, _dp, _dp]
        lib.oracle_sweep.argtypes = [i, i, i, i, i, d, d, _dp, _dp, _dp]
        lib.oracle_dirichlet.argtypes = [i, i, i, i, _u8p, _dp, _dp]
        lib.oracle_dirichlet_nodes.argtypes = [i, i, i, i, L, _i64p, _dp, _dp]
        lib.oracle_sources.argtypes = [i, i, i, i, d, L, _i64p, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_step.argtypes = [i, i, i, i, _dp, d, _dp, _dp, _u8p, _dp, L, _i64p, _dp,
                                    L, _i64p, _dp, _dp, _dp, _dp, i, _dp]
        lib.oracle_adjoint_step.argtypes = [i, i, i, i, _dp, d, _dp, _dp, _u8p, _dp, L, _i64p,
                                            _dp, L, _i64p, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                            _dp, _dp, _dp, _dp]
        for f in (lib.oracle_axis_coefficients, lib.oracle_thomas, lib.oracle_sweep,
                  lib.oracle_dirichlet, lib.oracle_dirichlet_nodes, lib.oracle_sources,
                  lib.oracle_step, lib.oracle_adjoint_step):
            f.restype = ctypes.c_int
        _libs[parallel] = lib
    return _libs[parallel]


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


class Problem:
    """Grid, parameters, boundary and agents of one microenvironment (all FP64, host).

    Field layout is ``rho[z, y, x, s]`` (substrates interleaved per voxel, x fastest of the axes).
    dx: the voxel spacing, or three spacings (x, y, z) for an anisotropic grid.
    dirichlet_nodes: None or (voxel, substrate, value) arrays of Dirichlet nodes, overwritten at
    each Dirichlet application after the flagged faces (a repeated (voxel, substrate) takes its
    last value).
    parallel: run on the OpenMP copy (all host cores; bit-identical results).
    """

    def __init__(self, nx, ny, nz, ns, dx, dt, D, lam, dirichlet_on=None, dirichlet_value=None,
                 voxel=None, secretion=None, target=None, uptake=None, weight=None,
                 dirichlet_nodes=None, parallel=False):
        self.parallel = bool(parallel)
        self.nx, self.ny, self.nz, self.ns = int(nx), int(ny), int(nz), int(ns)
        self.h3 = np.ascontiguousarray(np.broadcast_to(np.asarray(dx, dtype=np.float64),
                                                       (3,)).copy())
        self.dx, self.dt = float(self.h3[0]), float(dt)
        self.D = _f64(D, self.ns)
        self.lam = _f64(lam, self.ns)
        if dirichlet_on is not None:
            self.on = np.ascontiguousarray(np.asarray(dirichlet_on, dtype=np.uint8).reshape(-1))
            self.val = _f64(dirichlet_value, self.ns)
        else:
            self.on, self.val = None, None
        if dirichlet_nodes is not None and len(dirichlet_nodes[0]) > 0:
            nv, ns_, val = (np.asarray(a).reshape(-1) for a in dirichlet_nodes)
            if not (nv.size == ns_.size == val.size):
                raise ValueError("node voxel, substrate and value arrays differ in length")
            self.node_elem = np.ascontiguousarray(nv.astype(np.int64) * self.ns
                                                  + ns_.astype(np.int64))
            self.node_val = _f64(val)
        else:
            self.node_elem, self.node_val = None, None
        if voxel is not None and len(voxel) > 0:
            self.voxel = np.ascontiguousarray(np.asarray(voxel, dtype=np.int64).reshape(-1))
            na = self.voxel.size
            self.sec = None if secretion is None else _f64(secretion, na * self.ns)
            self.tgt = None if target is None else _f64(target, na * self.ns)
            self.upt = None if uptake is None else _f64(uptake, na * self.ns)
            self.w = None if weight is None else _f64(weight, na)
        else:
            self.voxel = None
            self.sec = self.tgt = self.upt = self.w = None

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx, self.ns)

    @property
    def n_agents(self):
        return 0 if self.voxel is None else int(self.voxel.size)

    def _field(self, rho):
        a = np.array(rho, dtype=np.float64, order="C", copy=True)
        if a.size != self.nx * self.ny * self.nz * self.ns:
            raise ValueError("field has the wrong size")
        return a.reshape(self.shape)

    def _nodes(self):
        n = 0 if self.node_elem is None else int(self.node_elem.size)
        return (n, _ptr(self.node_elem, _i64p), _ptr(self.node_val))

    def _agents(self):
        return (self.n_agents, _ptr(self.voxel, _i64p), _ptr(self.sec), _ptr(self.tgt),
                _ptr(self.upt), _ptr(self.w))

    def sweep(self, axis, rho):
        out = self._field(rho)
        _check(_get(self.parallel).oracle_sweep(axis, self.nx, self.ny, self.nz, self.ns,
                                   float(self.h3[axis]), self.dt,
                                   _ptr(self.D), _ptr(self.lam), _ptr(out)), "sweep")
        return out

    def dirichlet(self, rho):
        out = self._field(rho)
        _check(_get(self.parallel).oracle_dirichlet(self.nx, self.ny, self.nz, self.ns, _ptr(self.on, _u8p),
                                       _ptr(self.val), _ptr(out)), "dirichlet")
        _check(_get(self.parallel).oracle_dirichlet_nodes(self.nx, self.ny, self.nz, self.ns, *self._nodes(),
                                             _ptr(out)), "dirichlet nodes")
        return out

    def sources(self, rho):
        out = self._field(rho)
        _check(_get(self.parallel).oracle_sources(self.nx, self.ny, self.nz, self.ns, self.dt, *self._agents(),
                                     _ptr(out)), "sources")
        return out

    def step(self, rho, n_steps=1):
        out = self._field(rho)
        _check(_get(self.parallel).oracle_step(self.nx, self.ny, self.nz, self.ns, _ptr(self.h3), self.dt,
                                  _ptr(self.D), _ptr(self.lam), _ptr(self.on, _u8p),
                                  _ptr(self.val), *self._nodes(), *self._agents(), int(n_steps),
                                  _ptr(out)), "step")
        return out

    def adjoint_step(self, rho_in, gbar_out):
        """Adjoint of one step: returns (gbar_in, dD, dlambda, dsecretion, duptake)."""
        rho_in = self._field(rho_in)
        gout = self._field(gbar_out)
        gin = np.zeros_like(gout)
        dD = np.zeros(self.ns)
        dl = np.zeros(self.ns)
        na = self.n_agents
        dsec = np.zeros(na * self.ns)
        dupt = np.zeros(na * self.ns)
        _check(_get(self.parallel).oracle_adjoint_step(
            self.nx, self.ny, self.nz, self.ns, _ptr(self.h3), self.dt, _ptr(self.D), _ptr(self.lam),
            _ptr(self.on, _u8p), _ptr(self.val), *self._nodes(), *self._agents(), _ptr(rho_in),
            _ptr(gout),
            _ptr(gin), _ptr(dD), _ptr(dl), _ptr(dsec) if na else None,
            _ptr(dupt) if na else None), "adjoint_step")
        return gin, dD, dl, dsec.reshape(na, self.ns), dupt.reshape(na, self.ns)


def axis_coefficients(n, r, lam3):
    """Appendix A for one axis: returns (a, b, c, denom, cprime), each of length n."""
    arrs = [np.zeros(n) for _ in range(5)]
    _check(_get().oracle_axis_coefficients(int(n), float(r), float(lam3),
                                           *[_ptr(x) for x in arrs]), "axis_coefficients")
    return tuple(arrs)


def thomas(a, b, c, d):
    """Solve one tridiagonal system with the TDMA of Sect. 2.1 (returns a new array)."""
    a, b, c = _f64(a), _f64(b), _f64(c)
    x = _f64(d).copy()
    n = x.size
    if not (a.size == b.size == c.size == n):
        raise ValueError("a, b, c, d must have the same length")
    _check(_get().oracle_thomas(n, _ptr(a), _ptr(b), _ptr(c), _ptr(x)), "thomas")
    return x
