"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point that include/isdf.h declares, and
rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2404_09373_gb300 import isdf as B
from paper_2404_09373_gb300 import systems as S

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "isdf.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(isdf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("isdf_plan", "isdf_select_points", "isdf_fit", "isdf_coulomb", "isdf_exchange", "isdf_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = B.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(B.EXPORTED) == sorted(declared_functions())


def test_options_default():
    o = B.default_options()
    assert o.precision == 0 and o.tie_rel == 1e-9 and o.tie_abs == 1e-13 and o.reg_rel == 0.0


def _bad(system, **opt):
    with pytest.raises(B.IsdfError) as e:
        B.isdf_plan(system, B.default_options(**opt) if opt else None, stream=0)
    assert e.value.status == B.ISDF_ERR_ARG
    return e.value.message


def test_plan_rejects_invalid_systems_without_a_device():
    good = S.make_system((1, 1, 1), 0.0, None, ((8, 8, 8), (4, 4, 4)), (0.5,))
    s = dict(good)
    s["grids"] = np.array([[8, 8, 8], [8, 4, 4]])
    assert "decrease" in _bad(s)
    s = dict(good)
    s["grids"] = np.array([[9, 8, 8], [4, 4, 4]])
    assert "even" in _bad(s)
    s = dict(good)
    s["shell_l"] = good["shell_l"].copy()
    s["shell_l"][0] = 2
    assert "s and p" in _bad(s)
    s = dict(good)
    s["shell_exp"] = good["shell_exp"].copy()
    s["shell_exp"][3] = -1.0
    assert "exponent" in _bad(s)
    s = dict(good)
    s["level_min_exp"] = np.array([])
    with pytest.raises(Exception):
        B.isdf_plan(s, stream=0)
    s = dict(good)
    s["image_tol"] = 2.0
    assert "image_tol" in _bad(s)
    assert "precision" in _bad(good, precision=7)
    assert "prefilter" in _bad(good, prefilter=3)


def test_plan_rejects_non_orthorhombic_lattice():
    lib = B.load_library()
    good = S.make_system((1, 1, 1), 0.0, None, ((8, 8, 8),), ())
    xyz = np.ascontiguousarray(good["xyz"])
    sa = np.ascontiguousarray(good["shell_atom"], dtype=np.int32)
    sl = np.ascontiguousarray(good["shell_l"], dtype=np.int32)
    se = np.ascontiguousarray(good["shell_exp"])
    grid = np.array([8, 8, 8], dtype=np.int32)
    s = B.isdf_system()
    for i in range(9):
        s.lattice[i] = 0.0
    s.lattice[0] = s.lattice[4] = s.lattice[8] = 6.74
    s.lattice[1] = 0.5  # sheared cell
    s.natom = xyz.shape[0]
    s.xyz = xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s.nshell = se.shape[0]
    s.shell_atom = sa.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    s.shell_l = sl.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    s.shell_exp = se.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s.nlevel = 1
    s.grid = grid.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    s.level_min_exp = None
    s.image_tol = 1e-10
    h = ctypes.c_void_p()
    st = lib.isdf_plan(ctypes.byref(s), None, None, ctypes.byref(h))
    assert st == B.ISDF_ERR_ARG and h.value is None
    assert b"diagonal" in lib.isdf_last_error(None)


def test_null_plan_calls_are_rejected():
    lib = B.load_library()
    piv = np.zeros(4, dtype=np.int64)
    n = ctypes.c_int(0)
    assert lib.isdf_select_points(None, 4, 0.0, None, 0, piv.ctypes.data, None, ctypes.byref(n)) == B.ISDF_ERR_ARG
    assert lib.isdf_fit(None, piv.ctypes.data, 4) == B.ISDF_ERR_ARG
    assert lib.isdf_coulomb(None, None) == B.ISDF_ERR_ARG
    assert lib.isdf_get_size(None, 0) == 0
    lib.isdf_destroy(None)


@pytest.mark.parametrize("slices,accepted", [(4, False), (5, True), (6, True), (7, True), (8, True), (9, False)])
def test_gemm_digit_counts(slices, accepted):
    """isdf_gemm_f64 takes 5 to 8 digits; the argument check comes before the
    device-pointer check, so host buffers show which counts pass it."""
    lib = B.load_library()
    a = np.zeros((4, 4))
    st = lib.isdf_gemm_f64(a.ctypes.data, a.ctypes.data, a.ctypes.data, 4, 4, 4, 4, 4, 4, 1.0, slices, 1, None)
    assert st == B.ISDF_ERR_ARG
    msg = lib.isdf_last_error(None)
    if accepted:
        assert b"device pointers" in msg
    else:
        assert b"invalid arguments" in msg


@pytest.mark.parametrize("reps,eps", [((1, 1, 1), 1e-8), ((2, 2, 1), 1e-8), ((1, 2, 3), 1e-3), ((2, 2, 2), 0.5),
                                      ((1, 1, 1), 1e-14)])
def test_grids_for_threshold_match_the_oracle(reps, eps):
    """Host logic of the library: the threshold-driven grid of every level
    (Section III, Eq. 6) equals the oracle's, bit for bit."""
    from oracle import isdf as O
    from paper_2404_09373_gb300 import isdf as B
    from paper_2404_09373_gb300 import systems as S

    sysd = S.make_system(reps, 0.0, None, ((8, 8, 8), (4, 4, 4), (2, 2, 2)), S.LEVEL_EDGES_3)
    np.testing.assert_array_equal(B.isdf_grids_for_threshold(sysd, eps), O.grids_for_threshold(sysd, eps))
    two = S.make_system(reps, 0.0, None, ((8, 8, 8), (4, 4, 4)), (0.5,), s_exps=(0.3, 2.0), p_exps=(0.7,))
    np.testing.assert_array_equal(B.isdf_grids_for_threshold(two, eps), O.grids_for_threshold(two, eps))


def test_grids_for_threshold_rejects_bad_thresholds():
    from paper_2404_09373_gb300 import isdf as B
    from paper_2404_09373_gb300 import systems as S

    sysd = S.make_system((1, 1, 1), 0.0, None, ((8, 8, 8),), ())
    for eps in (0.0, 1.0, -1e-3, float("nan")):
        with pytest.raises(B.IsdfError) as e:
            B.isdf_grids_for_threshold(sysd, eps)
        assert e.value.status == B.ISDF_ERR_ARG
