"""The C-ABI library loads, exports every declared symbol and validates its
inputs on the host (CPU only: no call here reaches the GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hc():
    from paper_2112_03444_gb300 import build
    build.build()
    from paper_2112_03444_gb300 import hc as mod
    return mod


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hc_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(hc):
    lib = ctypes.CDLL(hc.LIB_PATH)
    names = declared_functions()
    assert "hc_create_problem" in names and "hc_track_batch" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(hc.EXPORTED) | set(names)


def test_struct_layouts_match_header_sizes(hc):
    # hc_settings: 14 doubles + 10 int32, then 4 int32 + 3 doubles of the endgame
    assert ctypes.sizeof(hc.hc_settings) == 192
    assert ctypes.sizeof(hc.hc_batch_result) == 18 * 8
    assert ctypes.sizeof(hc.hc_batch_desc) == 4 + 4 + 7 * 8 + 8 + 4 + 4 + 8


def test_default_settings_and_strings(hc):
    s = hc.default_settings()
    assert s.dt_min == 1e-6 and s.dt_max == 0.05 and s.max_newton == 3
    assert s.precision == hc.HC_PREC_MIXED and s.newton_tol == 1e-8
    assert s.retrack_precision == hc.HC_PREC_DF
    assert hc._lib.hc_status_string(hc.HC_ERR_INVALID) == b"invalid argument"
    assert hc._lib.hc_status_string(12345) == b"unknown status"


def _desc(hc, system, **kw):
    keep = [np.ascontiguousarray(system.term_eq, np.int32),
            np.ascontiguousarray(system.term_coef, np.complex128),
            np.ascontiguousarray(system.term_exp, np.uint8)]
    d = hc.hc_problem_desc()
    d.n = system.n
    d.n_terms = system.n_terms
    d.term_eq, d.term_coef, d.term_exp = (k.ctypes.data for k in keep)
    d.kind = hc.HC_TOTAL_DEGREE
    d.gamma[0], d.gamma[1] = 1.0, 0.0
    d.settings = hc.default_settings()
    for k, v in kw.items():
        setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("field,value", [("n", 0), ("n", 33), ("n_terms", 0), ("kind", 7)])
def test_create_problem_rejects_bad_descriptors(hc, field, value):
    from paper_2112_03444_gb300 import inputs
    d, keep = _desc(hc, inputs.dense_system(3, 2, 0), **{field: value})
    h = ctypes.c_void_p(12345)
    rc = hc._lib.hc_create_problem(ctypes.byref(d), ctypes.byref(h))
    assert rc == hc.HC_ERR_INVALID
    assert h.value == 12345  # untouched on error


def test_create_problem_rejects_out_of_range_equation(hc):
    from paper_2112_03444_gb300 import inputs
    sys_ = inputs.dense_system(2, 2, 0)
    sys_.term_eq[3] = 5
    d, keep = _desc(hc, sys_)
    h = ctypes.c_void_p()
    assert hc._lib.hc_create_problem(ctypes.byref(d), ctypes.byref(h)) == hc.HC_ERR_INVALID


def test_create_problem_rejects_non_unit_gamma_and_nan(hc):
    from paper_2112_03444_gb300 import inputs
    sys_ = inputs.dense_system(2, 2, 0)
    d, keep = _desc(hc, sys_)
    d.gamma[0] = 2.0
    h = ctypes.c_void_p()
    assert hc._lib.hc_create_problem(ctypes.byref(d), ctypes.byref(h)) == hc.HC_ERR_INVALID
    sys_.term_coef[0] = complex(np.nan, 0)
    d, keep = _desc(hc, sys_)
    assert hc._lib.hc_create_problem(ctypes.byref(d), ctypes.byref(h)) == hc.HC_ERR_NUMERIC


def test_create_problem_rejects_bad_settings(hc):
    from paper_2112_03444_gb300 import inputs
    d, keep = _desc(hc, inputs.dense_system(2, 2, 0))
    d.settings.dt_min = -1.0
    h = ctypes.c_void_p()
    assert hc._lib.hc_create_problem(ctypes.byref(d), ctypes.byref(h)) == hc.HC_ERR_INVALID


def test_null_handles_are_rejected(hc):
    r = hc.hc_batch_result()
    assert hc._lib.hc_poll(None, 0, ctypes.byref(r)) == hc.HC_ERR_INVALID
    assert hc._lib.hc_problem_paths(None) == -1
    hc._lib.hc_destroy(None)  # no-op


@pytest.mark.parametrize("field,value", [("max_newton_ir", 0), ("max_newton_ir", 33),
                                         ("block_threads", 16), ("block_threads", 256),
                                         ("lanes", 16), ("endgame", 2), ("retrack_precision", 1),
                                         ("retrack_precision", 3), ("precision", 3)])
def test_create_problem_rejects_bad_iteration_limits(hc, field, value):
    from paper_2112_03444_gb300 import inputs
    d, keep = _desc(hc, inputs.dense_system(2, 2, 0))
    setattr(d.settings, field, value)
    h = ctypes.c_void_p()
    assert hc._lib.hc_create_problem(ctypes.byref(d), ctypes.byref(h)) == hc.HC_ERR_INVALID


def test_default_refinement_iterations(hc):
    s = hc.default_settings()
    assert s.max_newton_ir == 2 * s.max_newton and s.block_threads == 0


def test_plan_calls_reject_null_handles(hc):
    h = ctypes.c_void_p()
    assert hc._lib.hc_plan_create(None, 1, ctypes.byref(h)) == hc.HC_ERR_INVALID
    b = hc.hc_batch_desc()
    assert hc._lib.hc_plan_run(None, ctypes.byref(b), ctypes.byref(h)) == hc.HC_ERR_INVALID


def test_memory_cap_rejects_negative(hc):
    assert hc._lib.hc_set_memory_cap(-1) == hc.HC_ERR_INVALID


def test_batch_descriptor_defaults_are_zero(hc):
    b = hc.hc_batch_desc()
    assert b.step_budget == 0 and b.n_subset == 0 and b.reserved == 0 and not b.path_ids
