"""Correctness oracle for the S-model DVM step (arXiv:1912.04582).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by
``bench.py``'s CPU-baseline leg, never by the library.  It is independent of the CUDA
path (no shared code, headers, tables or helpers); the only thing both sides consume
is the seeded input from ``workloads``.

* ``FullGridOracle`` wraps ``dvm_oracle.c``: the plain FP64 full-grid method
  (Algorithms 1 and 2 of Section 3) on an unstructured hex mesh, and its implicit step
  (Section 3, linear-system equation: one LU-SGS pass over the cells in index order).
* ``oracle.tucker`` holds the Tucker-format reference operations of Sections 4-5 in
  numpy (expansion, HOSVD, sum, Hadamard product, weighted convolution, rank-1
  Maxwellian, Lemma 1, the low-rank Shakhov function, the rank-1 diagonal estimate and
  division, the Tucker format's implicit step) used to pin the Tucker path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dvm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libdvm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the C oracle with gcc (OpenMP, no fast-math, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.orc_create.restype = P
    L.orc_create.argtypes = [ctypes.c_int64, dp, ctypes.c_int64, i64p, ctypes.c_int64, i64p,
                             i32p, i32p, dp, dp, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, ctypes.c_char_p]
    L.orc_destroy.argtypes = [P]
    L.orc_error.restype = ctypes.c_char_p
    L.orc_error.argtypes = [P]
    L.orc_set_bc.argtypes = [P, ctypes.c_int32, ctypes.c_int32, dp]
    L.orc_init_maxwellian.argtypes = [P, dp, dp, dp]
    L.orc_init_f.argtypes = [P, dp]
    L.orc_get_f.argtypes = [P, dp]
    L.orc_macro.argtypes = [P, dp]
    L.orc_geometry.argtypes = [P, dp, i64p, dp]
    L.orc_num_faces.restype = ctypes.c_int64
    L.orc_num_faces.argtypes = [P]
    L.orc_dt.restype = ctypes.c_double
    L.orc_dt.argtypes = [P, ctypes.c_double]
    L.orc_step.argtypes = [P, ctypes.c_int32, ctypes.c_double, dp]
    L.orc_step_lusgs.argtypes = [P, ctypes.c_int32, ctypes.c_double, dp]
    L.orc_rhs.argtypes = [P, dp]
    L.orc_lusgs_diag.argtypes = [P, ctypes.c_double, dp]
    L.orc_cell_shakhov.argtypes = [P, dp, dp, dp]
    L.orc_shakhov_from_macro.argtypes = [P, dp, dp]
    L.orc_maxwellian.argtypes = [P, ctypes.c_double, dp, ctypes.c_double, dp]
    L.orc_nu.restype = ctypes.c_double
    L.orc_nu.argtypes = [P, ctypes.c_double, ctypes.c_double]
    L.orc_nodes.argtypes = [P, ctypes.c_int32, dp]
    L.orc_weight.restype = ctypes.c_double
    L.orc_weight.argtypes = [P]
    L.orc_wall_density.argtypes = [P, dp]
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class FullGridOracle:
    """FP64 full-grid S-model DVM on one workload (see ``dvm_oracle.c``)."""

    def __init__(self, wl, init=True):
        L = _load()
        self.wl = wl
        self._keep = [_c(wl.xyz, np.float64), _c(wl.hex8, np.int64), _c(wl.bface, np.int64),
                      _c(wl.bgroup, np.int32), _c(wl.N, np.int32), _c(wl.lo, np.float64),
                      _c(wl.hi, np.float64)]
        xyz, hex8, bface, bgroup, N, lo, hi = self._keep
        err = ctypes.create_string_buffer(256)
        self.h = L.orc_create(
            xyz.shape[0], _dp(xyz), hex8.shape[0],
            hex8.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), bface.shape[0],
            bface.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            bgroup.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            N.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(lo), _dp(hi),
            wl.Pr, wl.omega, wl.Kn, err)
        if not self.h:
            raise ValueError("oracle mesh error: " + err.value.decode())
        self.L = L
        self.n_cell = hex8.shape[0]
        self.nn = int(np.prod(wl.N))
        for g, t, par in wl.bcs:
            p = _c(par, np.float64)
            rc = L.orc_set_bc(self.h, g, t, _dp(p))
            if rc != 0:
                raise ValueError(f"oracle bc error {rc}: " + L.orc_error(self.h).decode())
        if init:
            self.init_maxwellian(wl.n0, wl.u0, wl.T0)

    def __del__(self):
        if getattr(self, "h", None):
            self.L.orc_destroy(self.h)
            self.h = None

    def init_maxwellian(self, n, u, T):
        n, u, T = _c(n, np.float64), _c(u, np.float64), _c(T, np.float64)
        if self.L.orc_init_maxwellian(self.h, _dp(n), _dp(u), _dp(T)) != 0:
            raise ValueError(self.L.orc_error(self.h).decode())

    def init_f(self, f):
        f = _c(f, np.float64).reshape(-1)
        assert f.size == self.n_cell * self.nn
        if self.L.orc_init_f(self.h, _dp(f)) != 0:
            raise ValueError(self.L.orc_error(self.h).decode())

    def f(self):
        out = np.empty((self.n_cell,) + tuple(int(v) for v in self.wl.N))
        self.L.orc_get_f(self.h, _dp(out))
        return out

    def macro(self):
        """[n_cell, 8] = n, u1, u2, u3, T, q1, q2, q3 (Algorithm 2)."""
        out = np.empty((self.n_cell, 8))
        self.L.orc_macro(self.h, _dp(out))
        return out

    def dt(self, cfl=None):
        return self.L.orc_dt(self.h, self.wl.cfl if cfl is None else cfl)

    def step(self, nsteps, dt):
        r = ctypes.c_double(0.0)
        self.L.orc_step(self.h, int(nsteps), float(dt), ctypes.byref(r))
        return r.value

    def step_lusgs(self, nsteps, dt):
        """Implicit steps (linear-system equation of Section 3), one LU-SGS pass
        each over the cells in index order; returns the last residual."""
        r = ctypes.c_double(0.0)
        self.L.orc_step_lusgs(self.h, int(nsteps), float(dt), ctypes.byref(r))
        return r.value

    def rhs(self):
        """R^n of every cell: the explicit right-hand side of Algorithm 1."""
        out = np.empty((self.n_cell,) + tuple(int(v) for v in self.wl.N))
        self.L.orc_rhs(self.h, _dp(out))
        return out

    def lusgs_diag(self, dt):
        """The diagonal tensors D_i of the implicit system (diagonal_term equation)."""
        out = np.empty((self.n_cell,) + tuple(int(v) for v in self.wl.N))
        self.L.orc_lusgs_diag(self.h, float(dt), _dp(out))
        return out

    def geometry(self):
        nf = self.L.orc_num_faces(self.h)
        vol = np.empty(self.n_cell)
        fcell = np.empty((nf, 3), dtype=np.int64)
        fgeo = np.empty((nf, 4))
        self.L.orc_geometry(self.h, _dp(vol), fcell.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            _dp(fgeo))
        return vol, fcell, fgeo

    def nodes(self):
        out = []
        for a in range(3):
            x = np.empty(int(self.wl.N[a]))
            self.L.orc_nodes(self.h, a, _dp(x))
            out.append(x)
        return out

    def weight(self):
        return self.L.orc_weight(self.h)

    def maxwellian(self, n, u, T):
        out = np.empty(tuple(int(v) for v in self.wl.N))
        uu = _c(u, np.float64)
        self.L.orc_maxwellian(self.h, float(n), _dp(uu), float(T), _dp(out))
        return out

    def shakhov_of(self, fcell):
        """(f^S, macroparameters) of a single-cell tensor (Algorithm 2)."""
        f = _c(fcell, np.float64)
        fs = np.empty_like(f)
        a = np.empty(8)
        self.L.orc_cell_shakhov(self.h, _dp(f), _dp(fs), _dp(a))
        return fs, a

    def shakhov_from_macro(self, a):
        aa = _c(a, np.float64)
        fs = np.empty(tuple(int(v) for v in self.wl.N))
        self.L.orc_shakhov_from_macro(self.h, _dp(aa), _dp(fs))
        return fs

    def nu(self, n, T):
        return self.L.orc_nu(self.h, float(n), float(T))

    def wall_density(self):
        nf = self.L.orc_num_faces(self.h)
        out = np.empty(nf)
        self.L.orc_wall_density(self.h, _dp(out))
        return out


def run_full(wl, steps=None, dt=None):
    """Run the oracle for ``steps`` steps; returns (f, macro, dt, residual)."""
    o = FullGridOracle(wl)
    dt = o.dt() if dt is None else dt
    res = o.step(wl.steps if steps is None else steps, dt)
    return o.f(), o.macro(), dt, res
