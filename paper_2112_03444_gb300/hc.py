"""Thin ctypes binding of the C-ABI in include/hc.h (libhc.so).

Argument marshalling only: every step of the tracking path runs in the CUDA
kernels behind the C-ABI.  The library must have been built (``build.py``);
importing this module without it raises, there is no CPU fallback.

Same names as the C calls: ``create_problem``, ``track_batch``, ``poll``,
``destroy``, ``default_settings``; plus ``Problem`` / ``Batch`` wrappers that
accept numpy arrays (host) or torch CUDA tensors (device-resident).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2112_03444_gb300/build.py "
                      "(the tracker has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

# ---------------------------------------------------------------- constants
HC_OK, HC_PENDING = 0, 1
HC_ERR_INVALID, HC_ERR_OOM, HC_ERR_CUDA, HC_ERR_TIMEOUT = -1, -2, -3, -4
HC_ERR_NUMERIC, HC_ERR_BUSY, HC_ERR_UNSUPPORTED = -5, -6, -7
HC_TOTAL_DEGREE, HC_PARAMETER, HC_COEFFICIENT = 0, 1, 2
HC_PREC_FP64, HC_PREC_MIXED, HC_PREC_DF = 0, 1, 2
HC_DEVICE_PTRS, HC_BLOCKING_ADMIT = 1, 2
PATH_FINITE, PATH_DIVERGED, PATH_FAIL_STEP, PATH_FAIL_MAXSTEPS = 1, 2, 3, 4
PATH_FAIL_NAN, PATH_SINGULAR, PATH_FAIL_REFINE, PATH_REAL = 5, 6, 7, 0x80


class hc_settings(ctypes.Structure):
    _fields_ = [("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("dt_init", ctypes.c_double), ("newton_tol", ctypes.c_double),
                ("newton_tol_fp32", ctypes.c_double), ("max_first_corr", ctypes.c_double),
                ("refine_tol", ctypes.c_double), ("r_inf", ctypes.c_double),
                ("finite_tol", ctypes.c_double), ("real_tol", ctypes.c_double),
                ("singular_cond", ctypes.c_double), ("t_endgame", ctypes.c_double),
                ("dt_min_fp32", ctypes.c_double), ("max_first_corr_fp32", ctypes.c_double),
                ("max_steps_fp32", ctypes.c_int32), ("max_newton", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("grow_after", ctypes.c_int32), ("refine_iters", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("escalate", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("max_newton_ir", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("endgame", ctypes.c_int32),
                ("eg_cmax", ctypes.c_int32), ("eg_samples", ctypes.c_int32),
                ("retrack_precision", ctypes.c_int32), ("eg_s0", ctypes.c_double),
                ("eg_ratio", ctypes.c_double), ("eg_tol", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hc_problem_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_terms", ctypes.c_int32),
                ("term_eq", ctypes.c_void_p), ("term_coef", ctypes.c_void_p),
                ("term_exp", ctypes.c_void_p), ("max_pfac", ctypes.c_int32),
                ("term_param", ctypes.c_void_p), ("n_params", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("gamma", ctypes.c_double * 2),
                ("p0", ctypes.c_void_p), ("n_start", ctypes.c_int64),
                ("start", ctypes.c_void_p), ("settings", hc_settings),
                ("n_sym", ctypes.c_int32), ("sym_mask", ctypes.c_uint32 * 4)]


class hc_batch_desc(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("coef", ctypes.c_void_p), ("p1", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("x_out", ctypes.c_void_p),
                ("status_out", ctypes.c_void_p), ("steps_out", ctypes.c_void_p),
                ("be_out", ctypes.c_void_p), ("step_budget", ctypes.c_int64),
                ("n_subset", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("path_ids", ctypes.c_void_p)]


class hc_batch_result(ctypes.Structure):
    _fields_ = [("paths", ctypes.c_int64), ("finite", ctypes.c_int64),
                ("real", ctypes.c_int64), ("diverged", ctypes.c_int64),
                ("singular", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("escalated", ctypes.c_int64), ("steps_accepted", ctypes.c_int64),
                ("steps_rejected", ctypes.c_int64), ("newton_iters", ctypes.c_int64),
                ("esc_accepted", ctypes.c_int64), ("esc_rejected", ctypes.c_int64),
                ("esc_newton", ctypes.c_int64),
                ("device_ms", ctypes.c_double), ("track_ms", ctypes.c_double),
                ("escalate_ms", ctypes.c_double), ("untracked", ctypes.c_int64),
                ("steps_total", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_lib.hc_status_string.restype = ctypes.c_char_p
_lib.hc_status_string.argtypes = [ctypes.c_int32]
_lib.hc_last_error.restype = ctypes.c_char_p
_lib.hc_default_settings.restype = hc_settings
_lib.hc_create_problem.restype = ctypes.c_int32
_lib.hc_create_problem.argtypes = [ctypes.POINTER(hc_problem_desc), ctypes.POINTER(_P)]
_lib.hc_problem_paths.restype = ctypes.c_int64
_lib.hc_problem_paths.argtypes = [_P]
_lib.hc_track_batch.restype = ctypes.c_int32
_lib.hc_track_batch.argtypes = [_P, ctypes.POINTER(hc_batch_desc), ctypes.POINTER(_P)]
_lib.hc_poll.restype = ctypes.c_int32
_lib.hc_poll.argtypes = [_P, ctypes.c_int64, ctypes.POINTER(hc_batch_result)]
_lib.hc_destroy.restype = None
_lib.hc_destroy.argtypes = [_P]
_lib.hc_set_memory_cap.restype = ctypes.c_int32
_lib.hc_set_memory_cap.argtypes = [ctypes.c_int64]

_lib.hc_measure_fma_peak.restype = ctypes.c_int32
_lib.hc_measure_fma_peak.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]

class hc_problem_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("inputs_per_instance", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("paths", ctypes.c_int64), ("device_bytes_per_instance", ctypes.c_int64)]


class hc_server_config(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("max_batch_instances", ctypes.c_int32),
                ("max_device_bytes", ctypes.c_int64)]


class hc_request_info(ctypes.Structure):
    _fields_ = [("paths", ctypes.c_int64), ("finite", ctypes.c_int64), ("real", ctypes.c_int64),
                ("queue_us", ctypes.c_double), ("latency_us", ctypes.c_double),
                ("batch_instances", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class hc_tune_report(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int32), ("best", ctypes.c_int32),
                ("cached", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ms", ctypes.c_double * 16), ("finite", ctypes.c_int64 * 16),
                ("tried", hc_settings * 16)]


_lib.hc_autotune.restype = ctypes.c_int32
_lib.hc_autotune.argtypes = [_P, ctypes.POINTER(hc_batch_desc), ctypes.POINTER(hc_tune_report)]
_lib.hc_autotune_cached.restype = ctypes.c_int32
_lib.hc_autotune_cached.argtypes = [_P, ctypes.POINTER(hc_batch_desc), ctypes.c_char_p,
                                    ctypes.POINTER(hc_tune_report)]
_lib.hc_problem_query.restype = ctypes.c_int32
_lib.hc_problem_query.argtypes = [_P, ctypes.POINTER(hc_problem_info)]
_lib.hc_server_default_config.restype = hc_server_config
_lib.hc_server_create.restype = ctypes.c_int32
_lib.hc_server_create.argtypes = [ctypes.POINTER(hc_server_config), ctypes.POINTER(_P)]
_lib.hc_server_submit.restype = ctypes.c_int32
_lib.hc_server_submit.argtypes = [_P, _P, _P, ctypes.POINTER(ctypes.c_uint64)]
_lib.hc_server_wait.restype = ctypes.c_int32
_lib.hc_server_wait.argtypes = [_P, ctypes.c_uint64, ctypes.c_int64, _P, _P,
                                ctypes.POINTER(hc_request_info)]
_lib.hc_server_stats.restype = ctypes.c_int32
_lib.hc_server_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_int64 * 5)]

_lib.hc_plan_create.restype = ctypes.c_int32
_lib.hc_plan_create.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(_P)]
_lib.hc_plan_run.restype = ctypes.c_int32
_lib.hc_plan_run.argtypes = [_P, ctypes.POINTER(hc_batch_desc), ctypes.POINTER(_P)]

_lib.hc_track_dense_noalloc.restype = ctypes.c_int32
_lib.hc_track_dense_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(hc_settings), ctypes.c_int32, _P, _P, _P, _P,
                                        _P, _P]

EXPORTED = ("hc_status_string", "hc_last_error", "hc_default_settings", "hc_create_problem",
            "hc_problem_paths", "hc_problem_query", "hc_track_batch", "hc_poll", "hc_destroy",
            "hc_measure_fma_peak", "hc_track_dense_noalloc", "hc_server_default_config",
            "hc_server_create", "hc_server_submit", "hc_server_wait", "hc_server_stats",
            "hc_autotune", "hc_plan_create", "hc_plan_run", "hc_set_memory_cap",
            "hc_batched_solve", "hc_monodromy_solve", "hc_autotune_cached", "hc_evaluate",
            "hc_stream_create", "hc_stream_submit", "hc_stream_poll", "hc_stream_destroy")

_lib.hc_stream_create.restype = ctypes.c_int32
_lib.hc_stream_create.argtypes = [_P, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(_P)]
_lib.hc_stream_submit.restype = ctypes.c_int32
_lib.hc_stream_submit.argtypes = [_P, _P, ctypes.POINTER(ctypes.c_int64)]
_lib.hc_stream_poll.restype = ctypes.c_int32
_lib.hc_stream_poll.argtypes = [_P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P]
_lib.hc_stream_destroy.restype = ctypes.c_int32
_lib.hc_stream_destroy.argtypes = [_P]

_lib.hc_evaluate.restype = ctypes.c_int32
_lib.hc_evaluate.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P,
                             _P, _P, _P]


def problem_query(problem: int) -> dict:
    info = hc_problem_info()
    _check(_lib.hc_problem_query(problem, ctypes.byref(info)), "hc_problem_query")
    return {k: getattr(info, k) for k, _ in info._fields_}


class Server:
    """Continuous-batching server (hc_server_*): submit single instances of
    any number of problems; the library batches what is pending per problem
    and overlaps batches on n_streams streams under a device-memory cap."""

    def __init__(self, n_streams=None, max_batch_instances=None, max_device_bytes=None):
        cfg = _lib.hc_server_default_config()
        if n_streams is not None:
            cfg.n_streams = n_streams
        if max_batch_instances is not None:
            cfg.max_batch_instances = max_batch_instances
        if max_device_bytes is not None:
            cfg.max_device_bytes = max_device_bytes
        h = _P()
        _check(_lib.hc_server_create(ctypes.byref(cfg), ctypes.byref(h)), "hc_server_create")
        self.h = h.value

    def submit(self, problem, inp) -> int:
        a = np.ascontiguousarray(inp, np.complex128)
        rid = ctypes.c_uint64()
        _check(_lib.hc_server_submit(self.h, problem.h, a.ctypes.data, ctypes.byref(rid)),
               "hc_server_submit")
        return rid.value

    def wait(self, rid, problem, timeout_us=-1):
        x = np.zeros((problem.paths, problem.n), np.complex128)
        st = np.zeros(problem.paths, np.uint8)
        info = hc_request_info()
        code = _lib.hc_server_wait(self.h, rid, int(timeout_us), x.ctypes.data, st.ctypes.data,
                                   ctypes.byref(info))
        if code == HC_PENDING:
            return None
        _check(code, "hc_server_wait")
        return x, st, info.as_dict()

    def stats(self) -> dict:
        a = (ctypes.c_int64 * 5)()
        _check(_lib.hc_server_stats(self.h, ctypes.byref(a)), "hc_server_stats")
        return dict(done=a[0], batches=a[1], max_inflight_batches=a[2],
                    max_inflight_bytes=a[3], max_batch_instances=a[4])

    def close(self):
        if getattr(self, "h", None):
            destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def track_dense_noalloc(n, degree, gamma, settings, n_instances, coef, x_out, status_out,
                        steps_out, be_out=None, stream=None):
    """hc_track_dense_noalloc on device buffers (torch CUDA tensors); returns the status code.

    For callers that cannot allocate device memory while tracking: all scratch
    lives in the library's fixed device array.  Calls that overlap on the GPU
    race on that array; serialize them.
    """
    g = (ctypes.c_double * 2)(complex(gamma).real, complex(gamma).imag)
    if isinstance(settings, dict) or settings is None:
        settings = default_settings(**(settings or {}))
    return int(_lib.hc_track_dense_noalloc(int(n), int(degree), g, ctypes.byref(settings),
                                           int(n_instances), _addr(coef), _addr(x_out),
                                           _addr(status_out), _addr(steps_out), _addr(be_out),
                                           stream))


_lib.hc_batched_solve.restype = ctypes.c_int32
_lib.hc_batched_solve.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P,
                                  _P]


def batched_solve(A, b, x, info=None, stream=None) -> int:
    """hc_batched_solve on torch CUDA tensors: A [batch, n, n], b and x
    [batch, n], complex64 (FP32) or complex128 (FP64); info int32 [batch]."""
    batch, n = int(A.shape[0]), int(A.shape[-1])
    fp32 = 1 if str(A.dtype).endswith("complex64") else 0
    return int(_lib.hc_batched_solve(n, batch, fp32, _addr(A), _addr(b), _addr(x), _addr(info),
                                     stream))


class hc_monodromy_desc(ctypes.Structure):
    _fields_ = [("family", ctypes.c_void_p), ("x0", ctypes.c_void_p), ("p0", ctypes.c_void_p),
                ("seed", ctypes.c_uint64), ("stall_loops", ctypes.c_int32),
                ("max_loops", ctypes.c_int32), ("loops_per_round", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("max_solutions", ctypes.c_int64),
                ("out", ctypes.c_void_p)]


class hc_monodromy_info(ctypes.Structure):
    _fields_ = [("loops", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("paths_tracked", ctypes.c_int64), ("seconds", ctypes.c_double)]


_lib.hc_monodromy_solve.restype = ctypes.c_int32
_lib.hc_monodromy_solve.argtypes = [ctypes.POINTER(hc_monodromy_desc),
                                    ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(hc_monodromy_info)]


def monodromy_solve(system, x0, p0, seed=0, stall_loops=10, max_loops=400, loops_per_round=4,
                    max_solutions=100_000, symmetries=(), settings=None):
    """hc_monodromy_solve: (solutions [S, n] complex128, info dict)."""
    if isinstance(settings, dict) or settings is None:
        settings = default_settings(**(settings or {}))
    keep = [_host(system.term_eq, np.int32), _host(system.term_coef, np.complex128),
            _host(system.term_exp, np.uint8), _host(system.term_param, np.int32),
            _host(x0, np.complex128), _host(p0, np.complex128)]
    eq, cf, ex, pa, xa, pa0 = keep
    d = hc_problem_desc()
    d.n, d.n_terms = int(system.n), int(system.n_terms)
    d.term_eq, d.term_coef, d.term_exp = eq.ctypes.data, cf.ctypes.data, ex.ctypes.data
    d.max_pfac = int(system.max_pfac)
    d.term_param = pa.ctypes.data if pa.size else None
    d.n_params = int(system.n_params)
    d.kind = HC_PARAMETER
    d.settings = settings
    d.n_sym = len(symmetries)
    for k, m in enumerate(symmetries):
        d.sym_mask[k] = int(m)
    out = np.zeros((int(max_solutions), d.n), np.complex128)
    m = hc_monodromy_desc()
    m.family = ctypes.addressof(d)
    m.x0, m.p0 = xa.ctypes.data, pa0.ctypes.data
    m.seed, m.stall_loops, m.max_loops = int(seed), int(stall_loops), int(max_loops)
    m.loops_per_round, m.max_solutions, m.out = int(loops_per_round), int(max_solutions), \
        out.ctypes.data
    cnt = ctypes.c_int64()
    inf = hc_monodromy_info()
    _check(_lib.hc_monodromy_solve(ctypes.byref(m), ctypes.byref(cnt), ctypes.byref(inf)),
           "hc_monodromy_solve")
    return out[:cnt.value].copy(), {k: getattr(inf, k) for k, _ in inf._fields_}


def measure_fma_peak(fp64: bool, iters: int = 20000):
    """(FLOP/s, ms) of the device's FP32 or FP64 FMA pipe (own microbenchmark)."""
    f = ctypes.c_double()
    ms = ctypes.c_double()
    _check(_lib.hc_measure_fma_peak(int(bool(fp64)), int(iters), ctypes.byref(f), ctypes.byref(ms)),
           "hc_measure_fma_peak")
    return f.value, ms.value


class HCError(RuntimeError):
    def __init__(self, code, where):
        msg = _lib.hc_last_error().decode()
        super().__init__(f"{where}: {_lib.hc_status_string(code).decode()} ({code}) {msg}")
        self.code = code


def _check(code, where):
    if code not in (HC_OK, HC_PENDING):
        raise HCError(code, where)
    return code


def default_settings(**over) -> hc_settings:
    s = _lib.hc_default_settings()
    for k, v in over.items():
        setattr(s, k, v)
    return s


# ---------------------------------------------------------------- raw calls
def create_problem(desc: hc_problem_desc) -> int:
    h = _P()
    _check(_lib.hc_create_problem(ctypes.byref(desc), ctypes.byref(h)), "hc_create_problem")
    return h.value


def track_batch(problem: int, desc: hc_batch_desc) -> int:
    h = _P()
    _check(_lib.hc_track_batch(problem, ctypes.byref(desc), ctypes.byref(h)), "hc_track_batch")
    return h.value


def poll(batch: int, timeout_us: int = -1):
    """(code, result): HC_OK, HC_PENDING, or HC_ERR_TIMEOUT (done, step
    budget exhausted; result filled); other codes raise."""
    r = hc_batch_result()
    code = _lib.hc_poll(batch, int(timeout_us), ctypes.byref(r))
    if code != HC_ERR_TIMEOUT:
        _check(code, "hc_poll")
    return code, r


def set_memory_cap(max_device_bytes: int) -> None:
    """hc_set_memory_cap on the current device (0: no cap)."""
    _check(_lib.hc_set_memory_cap(int(max_device_bytes)), "hc_set_memory_cap")


def destroy(handle: int) -> None:
    if handle:
        _lib.hc_destroy(handle)


def problem_paths(problem: int) -> int:
    return int(_lib.hc_problem_paths(problem))


# ---------------------------------------------------------------- wrappers
def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _addr(a):
    """Address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Problem:
    """A polynomial system and its homotopy, encoded on the current device.

    system: an ``inputs.TermSystem``.  kind: HC_TOTAL_DEGREE (gamma) or
    HC_PARAMETER (p0, start).  settings: hc_settings or dict of overrides.
    symmetries: HC_PARAMETER sign masks (hc_problem_desc.sym_mask).
    """

    def __init__(self, system, kind=HC_TOTAL_DEGREE, gamma=1 + 0j, p0=None, start=None,
                 settings=None, symmetries=()):
        if isinstance(settings, dict) or settings is None:
            settings = default_settings(**(settings or {}))
        self.system = system
        self.n = int(system.n)
        self.kind = kind
        self._keep = [
            _host(system.term_eq, np.int32), _host(system.term_coef, np.complex128),
            _host(system.term_exp, np.uint8), _host(system.term_param, np.int32),
            None if p0 is None else _host(p0, np.complex128),
            None if start is None else _host(start, np.complex128),
        ]
        eq, cf, ex, pa, p0a, sa = self._keep
        d = hc_problem_desc()
        d.n = self.n
        d.n_terms = int(system.n_terms)
        d.term_eq = eq.ctypes.data
        d.term_coef = cf.ctypes.data
        d.term_exp = ex.ctypes.data
        d.max_pfac = int(system.max_pfac)
        d.term_param = pa.ctypes.data if pa.size else None
        d.n_params = int(system.n_params)
        d.kind = kind
        g = complex(gamma)
        d.gamma[0], d.gamma[1] = g.real, g.imag
        d.p0 = None if p0a is None else p0a.ctypes.data
        d.n_start = 0 if sa is None else int(sa.shape[0])
        d.start = None if sa is None else sa.ctypes.data
        d.settings = settings
        d.n_sym = len(symmetries)
        for k, m in enumerate(symmetries):
            d.sym_mask[k] = int(m)
        self.settings = settings
        self.h = create_problem(d)
        self.paths = problem_paths(self.h)

    def close(self):
        if getattr(self, "h", None):
            destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def _desc(self, n_instances, coef, p1, stream, x_out, status_out, steps_out, be_out, device,
              path_ids=None, step_budget=0, blocking=False):
        I, P, n = int(n_instances), self.paths, self.n
        if path_ids is not None:
            path_ids = _host(path_ids, np.int64).reshape(I, -1)
            P = path_ids.shape[1]
        if not device:
            x_out = np.zeros((I, P, n), np.complex128) if x_out is None else x_out
            status_out = np.zeros((I, P), np.uint8) if status_out is None else status_out
            steps_out = np.zeros((I, P, 3), np.int32) if steps_out is None else steps_out
            be_out = np.zeros((I, P), np.float64) if be_out is None else be_out
            if coef is not None and not hasattr(coef, "data_ptr"):
                coef = _host(coef, np.complex128)
            if p1 is not None and not hasattr(p1, "data_ptr"):
                p1 = _host(p1, np.complex128)
        b = hc_batch_desc()
        b.n_instances = I
        b.flags = (HC_DEVICE_PTRS if device else 0) | (HC_BLOCKING_ADMIT if blocking else 0)
        b.step_budget = int(step_budget)
        b.n_subset = 0 if path_ids is None else P
        b.path_ids = None if path_ids is None else path_ids.ctypes.data
        b.coef = _addr(coef)
        b.p1 = _addr(p1)
        b.stream = stream
        b.x_out = _addr(x_out)
        b.status_out = _addr(status_out)
        b.steps_out = _addr(steps_out)
        b.be_out = _addr(be_out)
        return b, dict(x=x_out, status=status_out, steps=steps_out, be=be_out, coef=coef, p1=p1,
                       path_ids=path_ids)

    def evaluate(self, x, t, instance=None, coef=None, p1=None, precision=HC_PREC_FP64):
        """H, dH/dx, dH/dt of the homotopy at points x [k][n] and times t [k]
        with the device evaluator (hc_evaluate); instance [k] indexes the rows
        of coef (total degree; None: the problem's coefficients) or p1
        (parameter families).  Returns (H [k][n], Hx [k][n][n], Ht [k][n])."""
        x = _host(np.atleast_2d(x), np.complex128)
        k = x.shape[0]
        t = _host(np.broadcast_to(np.asarray(t, np.float64), (k,)), np.float64)
        inst = _host(np.zeros(k) if instance is None else instance, np.int64)
        data = p1 if self.kind != HC_TOTAL_DEGREE else coef
        if data is not None:
            data = _host(np.atleast_2d(data), np.complex128)
        n_inst = 1 if data is None else data.shape[0]
        H = np.zeros((k, self.n), np.complex128)
        Hx = np.zeros((k, self.n, self.n), np.complex128)
        Ht = np.zeros((k, self.n), np.complex128)
        _check(_lib.hc_evaluate(self.h, int(precision), n_inst, _addr(data) if data is not None
                                else None, k, _addr(inst), _addr(x), _addr(t), _addr(H),
                                _addr(Hx), _addr(Ht)), "hc_evaluate")
        return H, Hx, Ht

    def track(self, n_instances=1, coef=None, p1=None, stream=None, device_out=None,
              x_out=None, status_out=None, steps_out=None, be_out=None, device=False,
              path_ids=None, step_budget=0, blocking=False):
        """Enqueue a batch; returns a Batch.  Host mode (default) allocates numpy
        outputs; with device=True pass torch CUDA tensors (inputs and outputs).
        path_ids [n_instances, k]: track only those starts (outputs hold k
        paths per instance); step_budget: hc_batch_desc.step_budget;
        blocking: HC_BLOCKING_ADMIT."""
        b, bufs = self._desc(n_instances, coef, p1, stream, x_out, status_out, steps_out, be_out,
                             device, path_ids, step_budget, blocking)
        h = track_batch(self.h, b)
        return Batch(h, self, bufs)

    def plan(self, n_instances=1):
        """A Plan: this batch size captured once as a CUDA graph (hc_plan_create)."""
        return Plan(self, n_instances)

    def autotune(self, n_instances=1, coef=None, p1=None, cache=None):
        """hc_autotune (or hc_autotune_cached with a cache file path) on a host
        sample batch; returns the report as a dict and keeps the chosen
        settings in the problem (and in self.settings)."""
        I, P, n = int(n_instances), self.paths, self.n
        bufs = dict(x=np.zeros((I, P, n), np.complex128), st=np.zeros((I, P), np.uint8),
                    steps=np.zeros((I, P, 3), np.int32))
        coef = None if coef is None else _host(coef, np.complex128)
        p1 = None if p1 is None else _host(p1, np.complex128)
        b = hc_batch_desc()
        b.n_instances = I
        b.coef = _addr(coef)
        b.p1 = _addr(p1)
        b.x_out, b.status_out, b.steps_out = (_addr(bufs[k]) for k in ("x", "st", "steps"))
        rep = hc_tune_report()
        if cache is None:
            _check(_lib.hc_autotune(self.h, ctypes.byref(b), ctypes.byref(rep)), "hc_autotune")
        else:
            _check(_lib.hc_autotune_cached(self.h, ctypes.byref(b), str(cache).encode(),
                                           ctypes.byref(rep)), "hc_autotune_cached")
        self.settings = rep.tried[rep.best]
        return dict(best=rep.best, cached=bool(rep.cached), ms=list(rep.ms[:rep.n_candidates]),
                    finite=list(rep.finite[:rep.n_candidates]),
                    tried=[dict(precision=rep.tried[i].precision, lanes=rep.tried[i].lanes,
                                block_threads=rep.tried[i].block_threads,
                                max_first_corr_fp32=rep.tried[i].max_first_corr_fp32)
                           for i in range(rep.n_candidates)])


class Plan:
    """hc_plan_create / hc_plan_run: replays one batch size of a problem as a
    CUDA graph over device buffers the plan owns."""

    def __init__(self, problem, n_instances):
        h = _P()
        _check(_lib.hc_plan_create(problem.h, int(n_instances), ctypes.byref(h)), "hc_plan_create")
        self.h = h.value
        self.problem = problem
        self.n_instances = int(n_instances)

    def run(self, coef=None, p1=None, stream=None, x_out=None, status_out=None, steps_out=None,
            be_out=None, device=False):
        """Enqueue one replay; returns a Batch (same outputs as Problem.track)."""
        sysm = self.problem.system
        for a, per in ((coef, sysm.n_terms), (p1, sysm.n_params)):
            if a is not None and int(np.prod(a.shape)) != self.n_instances * int(per):
                raise ValueError(f"input holds {int(np.prod(a.shape))} values, the plan takes "
                                 f"{self.n_instances} x {int(per)}")
        b, bufs = self.problem._desc(self.n_instances, coef, p1, stream, x_out, status_out,
                                     steps_out, be_out, device)
        h = _P()
        _check(_lib.hc_plan_run(self.h, ctypes.byref(b), ctypes.byref(h)), "hc_plan_run")
        return Batch(h.value, self.problem, bufs)

    def close(self):
        if getattr(self, "h", None):
            destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Batch:
    def __init__(self, h, problem, bufs):
        self.h = h
        self.problem = problem
        self.bufs = bufs
        self.result = None

    def poll(self, timeout_us=-1):
        code, r = poll(self.h, timeout_us)
        if code in (HC_OK, HC_ERR_TIMEOUT):
            self.result = r.as_dict()
            self.code = code
        return code

    def wait(self):
        self.poll(-1)
        return self

    @property
    def x(self):
        return self.bufs["x"]

    @property
    def status(self):
        return self.bufs["status"]

    @property
    def steps(self):
        return self.bufs["steps"]

    @property
    def be(self):
        return self.bufs["be"]

    def close(self):
        if getattr(self, "h", None):
            destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Stream:
    """Continuous admission into a resident tracking launch (hc_stream_*):
    submit(inputs) returns a ticket as soon as the instance is staged; its
    paths start as lane groups of the running launch free up.  poll(ticket)
    returns (x [paths][n], status [paths], steps [paths][3], be [paths]) or
    None while it is not done (timeout_us elapsed)."""

    def __init__(self, problem, slots=64, idle_us=20000):
        self.problem = problem
        h = _P()
        _check(_lib.hc_stream_create(problem.h, int(slots), int(idle_us), ctypes.byref(h)),
               "hc_stream_create")
        self.h = h.value
        self.paths = problem.paths

    def submit(self, coef=None, p1=None):
        data = p1 if self.problem.kind != HC_TOTAL_DEGREE else coef
        buf = None if data is None else _host(np.ravel(data), np.complex128)
        t = ctypes.c_int64()
        _check(_lib.hc_stream_submit(self.h, _addr(buf) if buf is not None else None,
                                     ctypes.byref(t)), "hc_stream_submit")
        return t.value

    def poll(self, ticket, timeout_us=-1):
        n = self.problem.n
        x = np.zeros((self.paths, n), np.complex128)
        st = np.zeros(self.paths, np.uint8)
        steps = np.zeros((self.paths, 3), np.int32)
        be = np.zeros(self.paths, np.float64)
        code = _lib.hc_stream_poll(self.h, int(ticket), int(timeout_us), _addr(x), _addr(st),
                                   _addr(steps), _addr(be))
        if code == HC_ERR_TIMEOUT:
            return None
        _check(code, "hc_stream_poll")
        return x, st, steps, be

    def close(self):
        if getattr(self, "h", None):
            _lib.hc_stream_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
