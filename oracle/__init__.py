"""Plain FP64 CPU oracle for the exponential-integrator step (arXiv 2402.02273).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package.  The product library
(`paper_2402_02273_gb300`) never imports it, and the two share no code.

The arithmetic lives in `oracle.c` (plain C loops, FP64, OpenMP over
z-planes); this module compiles it with gcc on first use and exposes it to
numpy through ctypes.  `multinomial.py` holds the paper's multinomial form of
the sub-stepped Taylor product for tiny problems.

Operator kinds: "conservative" (div(D grad u) with harmonic-mean faces, the
default reading) and "literal" (the Sec. 2.1 formula / eq. Amatrix as printed).
Schemes: "rosenbrock" (rho(1-2u^n) folded into A, f = rho (u^n)^2, eq. newF)
and "expeuler" (A = L, f = rho u (1-u)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

OPS = {"conservative": 0, "literal": 1}
SCHEMES = {"rosenbrock": 0, "expeuler": 1}


def build(force: bool = False) -> str:
    """Compile oracle.c into _liboracle.so (gcc, -O2, no FP contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("D", ctypes.POINTER(ctypes.c_double)),
                ("op", ctypes.c_int), ("scheme", ctypes.c_int), ("rho", ctypes.c_double)]


class _Schedule(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("stop_tol", ctypes.c_double),
                ("max_terms", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("umin", ctypes.c_double), ("umax", ctypes.c_double),
                ("s", ctypes.c_int), ("m", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(_Problem)
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_get_threads.restype = ctypes.c_int
            lib.oracle_apply_A.argtypes = [pp, dp, dp, dp]
            lib.oracle_apply_L.argtypes = [pp, dp, dp]
            lib.oracle_row_A.argtypes = [pp, dp, ctypes.c_long, dp]
            lib.oracle_assemble_A.argtypes = [pp, dp, dp]
            lib.oracle_norm_inf_A.argtypes = [pp, dp]
            lib.oracle_norm_inf_A.restype = ctypes.c_double
            lib.oracle_residual.argtypes = [pp, dp, dp]
            lib.oracle_phi1_action.argtypes = [pp, dp, dp, ctypes.c_double, ctypes.POINTER(_Schedule),
                                               dp, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int)]
            lib.oracle_phi1_action.restype = ctypes.c_int
            lib.oracle_step.argtypes = [pp, dp, ctypes.c_double, ctypes.POINTER(_Schedule),
                                        ctypes.POINTER(_Stats)]
            lib.oracle_step.restype = ctypes.c_int
            lib.oracle_run.argtypes = [pp, dp, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(_Schedule), ctypes.POINTER(_Stats)]
            lib.oracle_run.restype = ctypes.c_int
            lib.oracle_step_adjoint.argtypes = [pp, dp, ctypes.c_double, ctypes.POINTER(_Schedule), dp, dp,
                                                dp, dp]
            lib.oracle_step_adjoint.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Problem:
    """Grid, coefficients and model constants of one oracle problem.

    D is an (nz, ny, nx) float64 array (x fastest); h the voxel width (mm);
    rho the proliferation rate (1/day).
    """

    def __init__(self, D: np.ndarray, h: float = 1.0, rho: float = 0.025,
                 op: str = "conservative", scheme: str = "rosenbrock"):
        D = np.ascontiguousarray(D, dtype=np.float64)
        if D.ndim != 3:
            raise ValueError("D must be (nz, ny, nx)")
        self.D = D
        self.shape = D.shape
        self.h = float(h)
        self.rho = float(rho)
        self.op = op
        self.scheme = scheme
        nz, ny, nx = D.shape
        self._p = _Problem(nx, ny, nz, self.h, _dptr(self.D), OPS[op], SCHEMES[scheme], self.rho)
        self._lib = _load()

    def _vec(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        if v.shape != self.shape:
            v = v.reshape(self.shape)
        return v

    def apply_A(self, un, v):
        un, v = self._vec(un), self._vec(v)
        out = np.empty(self.shape)
        self._lib.oracle_apply_A(ctypes.byref(self._p), _dptr(un), _dptr(v), _dptr(out))
        return out

    def apply_L(self, v):
        v = self._vec(v)
        out = np.empty(self.shape)
        self._lib.oracle_apply_L(ctypes.byref(self._p), _dptr(v), _dptr(out))
        return out

    def row_A(self, un, p: int):
        un = self._vec(un)
        e = np.empty(7)
        self._lib.oracle_row_A(ctypes.byref(self._p), _dptr(un), int(p), _dptr(e))
        return e

    def rows_A(self, un):
        """(n, 7) entries of A_n: diagonal, then the -x, +x, -y, +y, -z, +z
        off-diagonals (0 where the neighbour lies outside the box)."""
        un = self._vec(un)
        e = np.empty((self.D.size, 7))
        self._lib.oracle_assemble_A(ctypes.byref(self._p), _dptr(un), _dptr(e))
        return e

    def norm_inf_A(self, un):
        un = self._vec(un)
        return self._lib.oracle_norm_inf_A(ctypes.byref(self._p), _dptr(un))

    def residual(self, un):
        un = self._vec(un)
        b = np.empty(self.shape)
        self._lib.oracle_residual(ctypes.byref(self._p), _dptr(un), _dptr(b))
        return b

    def phi1_action(self, un, b, tau, theta=0.5, stop_tol=1e-18, max_terms=200):
        """tau phi1(tau A) b; returns (x, s, m)."""
        un, b = self._vec(un), self._vec(b)
        x = np.empty(self.shape)
        s, m = ctypes.c_int(), ctypes.c_int()
        sch = _Schedule(theta, stop_tol, max_terms)
        rc = self._lib.oracle_phi1_action(ctypes.byref(self._p), _dptr(un), _dptr(b), float(tau),
                                          ctypes.byref(sch), _dptr(x), ctypes.byref(s),
                                          ctypes.byref(m))
        if rc != 0:
            raise RuntimeError(f"oracle_phi1_action failed ({rc})")
        return x, s.value, m.value

    def run(self, u0, tau, nsteps, theta=0.5, stop_tol=1e-18, max_terms=200, every=False):
        """nsteps steps from u0; returns (u, stats) or, with every=True, (list of u^n, stats)."""
        u = np.array(self._vec(u0), dtype=np.float64, copy=True)
        sch = _Schedule(theta, stop_tol, max_terms)
        stats = (_Stats * max(nsteps, 1))()
        states = [u.copy()] if every else None
        for t in range(nsteps):
            rc = self._lib.oracle_step(ctypes.byref(self._p), _dptr(u), float(tau),
                                       ctypes.byref(sch), ctypes.byref(stats[t]))
            if rc != 0:
                raise RuntimeError(f"oracle_step failed ({rc}) at step {t}")
            if every:
                states.append(u.copy())
        st = [{"mass": x.mass, "umin": x.umin, "umax": x.umax, "s": x.s, "m": x.m}
              for x in list(stats)[:nsteps]]
        return (states if every else u), st


def _problem_like(P, D):
    return Problem(D, h=P.h, rho=P.rho, op=P.op, scheme=P.scheme)


def vjp(P, u0, tau, nsteps, ubar_final, theta=0.5, stop_tol=1e-18, max_terms=200):
    """Reverse mode through nsteps oracle steps: given dJ/du_K, returns
    (dJ/du_0, dJ/drho, d/ds J(s D) at s = 1), every step's schedule frozen at its
    forward value.  All states are kept (small problems)."""
    lib = _load()
    states, _ = P.run(u0, tau, nsteps, theta, stop_tol, max_terms, every=True)
    sch = _Schedule(theta, stop_tol, max_terms)
    ubar = np.ascontiguousarray(np.array(ubar_final, dtype=np.float64).reshape(P.shape))
    g_rho, g_ds = ctypes.c_double(0.0), ctypes.c_double(0.0)
    for t in range(nsteps - 1, -1, -1):
        un = np.ascontiguousarray(states[t])
        out = np.empty(P.shape)
        rc = lib.oracle_step_adjoint(ctypes.byref(P._p), _dptr(un), float(tau), ctypes.byref(sch),
                                     _dptr(ubar), _dptr(out), ctypes.byref(g_rho), ctypes.byref(g_ds))
        if rc != 0:
            raise RuntimeError(f"oracle_step_adjoint failed ({rc})")
        ubar = out
    return ubar, g_rho.value, g_ds.value


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())
