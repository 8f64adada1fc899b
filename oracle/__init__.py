"""FP64 CPU oracle for homotopy-continuation path tracking (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``hc_oracle.cpp`` (plain C++,
complex double) through ctypes; it shares no code with the CUDA path.

Parity pins for every function here: ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hc_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Numeric status codes (the interface shared with the CUDA path by number).
FINITE, DIVERGED, FAIL_STEP, FAIL_MAXSTEPS, FAIL_NAN, SINGULAR, FAIL_REFINE = 1, 2, 3, 4, 5, 6, 7
REAL_BIT = 0x80

KIND_TOTAL_DEGREE, KIND_PARAMETER, KIND_COEFFICIENT = 0, 1, 2

# Order of the settings vector passed to the C++ side.
SETTINGS_ORDER = ("dt_min", "dt_max", "dt_init", "newton_tol", "max_newton", "max_steps",
                  "grow_after", "refine_tol", "refine_iters", "r_inf", "finite_tol",
                  "real_tol", "singular_cond", "max_first_corr", "endgame", "eg_s0",
                  "eg_ratio", "eg_tol", "eg_cmax", "eg_samples")

DEFAULT_SETTINGS = dict(dt_min=1e-6, dt_max=0.05, dt_init=0.01, newton_tol=1e-8,
                        max_newton=3, max_steps=100000, grow_after=3, refine_tol=1e-13,
                        refine_iters=8, r_inf=1e8, finite_tol=1e-10, real_tol=1e-8,
                        singular_cond=1e12, max_first_corr=0.1, endgame=0, eg_s0=0.1,
                        eg_ratio=0.5, eg_tol=1e-8, eg_cmax=8, eg_samples=40)


def build(force: bool = False) -> str:
    """Compile hc_oracle.cpp into liboracle.so (plain g++, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P, D, I, I64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
        lib.oracle_problem_new.restype = P
        lib.oracle_problem_new.argtypes = [I, I, P, P, P, I, P, I, I, D, D, P, P]
        lib.oracle_problem_free.argtypes = [P]
        lib.oracle_total_degree_paths.restype = I64
        lib.oracle_total_degree_paths.argtypes = [P]
        lib.oracle_start_point.argtypes = [P, I64, P]
        lib.oracle_eval.argtypes = [P, P, D, P, P, P]
        lib.oracle_solve.argtypes = [I, P, P, P]
        lib.oracle_solve.restype = I
        lib.oracle_rk4_step.argtypes = [P, P, D, D, P]
        lib.oracle_rk4_step.restype = I
        lib.oracle_newton_step.argtypes = [P, P, D, P]
        lib.oracle_newton_step.restype = I
        lib.oracle_track.argtypes = [P, I64, P, P, P, I, P, P, P, P, P, P]
        lib.oracle_hardware_threads.restype = I
        lib.oracle_backward_error.argtypes = [P, P]
        lib.oracle_backward_error.restype = D
        lib.oracle_cond1.argtypes = [P, P]
        lib.oracle_cond1.restype = D
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def hardware_threads() -> int:
    return int(_load().oracle_hardware_threads())


class OracleProblem:
    """A system plus its homotopy, held by the C++ oracle.

    kind = KIND_TOTAL_DEGREE: H = (1-t) gamma G + t F, G_i = x_i^{d_i} - 1.
    kind = KIND_PARAMETER:    H = F(x; (1-t) p0 + t p1).
    kind = KIND_COEFFICIENT:  H = sum_k ((1-t) c_k(p0) + t c_k(p1)) x^alpha_k, the
                              term coefficients c_k(p) interpolated (Sec. 6).
    """

    def __init__(self, system, kind=KIND_TOTAL_DEGREE, gamma=1.0 + 0j, p0=None, p1=None,
                 coef=None):
        self._lib = _load()
        self.n = int(system.n)
        self.kind = int(kind)
        coefs = np.ascontiguousarray(system.term_coef if coef is None else coef, dtype=np.complex128)
        self._keep = dict(
            eq=np.ascontiguousarray(system.term_eq, dtype=np.int32),
            coef=np.ascontiguousarray(coefs.view(np.float64)),
            exp=np.ascontiguousarray(system.term_exp, dtype=np.uint8),
            par=np.ascontiguousarray(system.term_param, dtype=np.int32),
            p0=None if p0 is None else np.ascontiguousarray(np.asarray(p0, np.complex128).view(np.float64)),
            p1=None if p1 is None else np.ascontiguousarray(np.asarray(p1, np.complex128).view(np.float64)),
        )
        k = self._keep
        self.h = self._lib.oracle_problem_new(
            self.n, int(system.n_terms), _ptr(k["eq"]), _ptr(k["coef"]), _ptr(k["exp"]),
            int(system.max_pfac), _ptr(k["par"]), int(system.n_params), self.kind,
            float(complex(gamma).real), float(complex(gamma).imag), _ptr(k["p0"]), _ptr(k["p1"]))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._lib.oracle_problem_free(h)
            self.h = None

    def total_degree_paths(self) -> int:
        return int(self._lib.oracle_total_degree_paths(self.h))

    def start_point(self, k: int) -> np.ndarray:
        x = np.zeros(self.n, np.complex128)
        self._lib.oracle_start_point(self.h, int(k), _ptr(x))
        return x

    def eval(self, x, t):
        x = np.ascontiguousarray(x, np.complex128)
        H = np.zeros(self.n, np.complex128)
        Ht = np.zeros(self.n, np.complex128)
        Hx = np.zeros((self.n, self.n), np.complex128)
        self._lib.oracle_eval(self.h, _ptr(x), float(t), _ptr(H), _ptr(Hx), _ptr(Ht))
        return H, Hx, Ht

    def rk4_step(self, x, t, dt):
        x = np.ascontiguousarray(x, np.complex128)
        y = np.zeros(self.n, np.complex128)
        rc = self._lib.oracle_rk4_step(self.h, _ptr(x), float(t), float(dt), _ptr(y))
        return y, rc == 0

    def newton_step(self, x, t):
        x = np.array(x, np.complex128)
        dn = ctypes.c_double(0.0)
        rc = self._lib.oracle_newton_step(self.h, _ptr(x), float(t), ctypes.byref(dn))
        return x, float(dn.value), rc == 0

    def backward_error(self, x) -> float:
        """max_i |F_i(x)| / sum_k |c_k| |x^alpha_k| at t = 1 (classification)."""
        x = np.ascontiguousarray(x, np.complex128)
        return float(self._lib.oracle_backward_error(self.h, _ptr(x)))

    def cond1(self, x) -> float:
        """1-norm condition number of dF/dx at t = 1 and the point x."""
        x = np.ascontiguousarray(x, np.complex128)
        return float(self._lib.oracle_cond1(self.h, _ptr(x)))

    def track(self, n_paths=None, start=None, path_ids=None, settings=None, threads=0):
        """Track paths; returns dict of numpy arrays (x, status, counts, be, cond, t)."""
        s = dict(DEFAULT_SETTINGS)
        if settings:
            s.update({k: v for k, v in settings.items() if k in DEFAULT_SETTINGS})
        svec = np.array([float(s[k]) for k in SETTINGS_ORDER], np.float64)
        if start is not None:
            start = np.ascontiguousarray(start, np.complex128).reshape(-1, self.n)
            n_paths = start.shape[0]
        elif path_ids is not None:
            path_ids = np.ascontiguousarray(path_ids, np.int64)
            n_paths = path_ids.shape[0]
        elif n_paths is None:
            n_paths = self.total_degree_paths()
        n_paths = int(n_paths)
        out = dict(x=np.zeros((n_paths, self.n), np.complex128),
                   status=np.zeros(n_paths, np.uint8),
                   counts=np.zeros((n_paths, 3), np.int32),
                   be=np.zeros(n_paths), cond=np.zeros(n_paths), t=np.zeros(n_paths))
        self._lib.oracle_track(self.h, n_paths, _ptr(start), _ptr(path_ids), _ptr(svec),
                               int(threads), _ptr(out["x"]), _ptr(out["status"]),
                               _ptr(out["counts"]), _ptr(out["be"]), _ptr(out["cond"]),
                               _ptr(out["t"]))
        return out


def solve(A, b):
    """Sec. 6 augmented-matrix LU solve of A x = b (complex double)."""
    A = np.ascontiguousarray(A, np.complex128)
    b = np.ascontiguousarray(b, np.complex128)
    n = b.shape[0]
    x = np.zeros(n, np.complex128)
    rc = _load().oracle_solve(n, _ptr(A), _ptr(b), _ptr(x))
    return x, rc == 0


def status_counts(status) -> dict:
    """Counts per class: finite, real, diverged, singular, failed."""
    st = np.asarray(status, np.uint8)
    base = st & 0x7F
    return dict(finite=int(np.sum(base == FINITE)),
                real=int(np.sum((base == FINITE) & ((st & REAL_BIT) != 0))),
                diverged=int(np.sum(base == DIVERGED)),
                singular=int(np.sum(base == SINGULAR)),
                failed=int(np.sum((base != FINITE) & (base != DIVERGED) & (base != SINGULAR))))
