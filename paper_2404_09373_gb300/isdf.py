"""Thin Python binding of the C ABI in ``include/isdf.h`` (argument marshalling only).

Every computation runs in ``libisdf.so``'s CUDA kernels.  Arrays may be NumPy
arrays (host) or torch tensors (host or CUDA); they are passed to the library
as raw pointers and the library tells host from device memory itself.  If the
shared library is missing it is built from ``csrc/`` with nvcc; if that is not
possible, loading fails with an exception (there is no other code path).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int64, c_void_p

import numpy as np

from . import build as _build

PIVOT_SHIFT = 40

ISDF_OK, ISDF_ERR_ARG, ISDF_ERR_OOM, ISDF_ERR_NOT_PD, ISDF_ERR_CUDA, ISDF_ERR_CUFFT, ISDF_ERR_TIMEOUT, ISDF_ERR_STATE = range(8)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_OOM", "ERR_NOT_PD", "ERR_CUDA", "ERR_CUFFT", "ERR_TIMEOUT", "ERR_STATE"]
GET_NBASIS, GET_NIP_LEVEL, GET_PIVOTS, GET_XL, GET_XN, GET_V, GET_XI_LEVEL0 = 0, 1, 2, 3, 4, 5, 6
GET_PHI_LEVEL0 = 10
GET_NPOINTS, GET_FIT_RESIDUAL, GET_SELECT_STATS, GET_V_COARSE = 20, 21, 22, 23
GET_LOCAL_BOX, GET_LOCAL_NIP = 24, 25
LOCAL_ATOM_SHIFT = 24  # local pivot code on level 0: (atom << 24) | box index
# element type written by isdf_get for each selector (float64 otherwise)
_GET_DTYPE = {GET_NBASIS: np.int32, GET_NIP_LEVEL: np.int32, GET_PIVOTS: np.int64, GET_NPOINTS: np.int64,
              GET_LOCAL_NIP: np.int32,
              GET_SELECT_STATS: np.int64}

EXPORTED = [
    "isdf_options_default",
    "isdf_plan",
    "isdf_select_points",
    "isdf_fit",
    "isdf_coulomb",
    "isdf_exchange",
    "isdf_get_size",
    "isdf_get",
    "isdf_last_error",
    "isdf_destroy",
    "isdf_profile_json",
    "isdf_kernel_launches",
    "isdf_gemm_f64",
    "isdf_mlp_num_params",
    "isdf_features",
    "isdf_mlp_train_step",
    "isdf_mlp_score",
    "isdf_propose",
    "isdf_propose_residual",
    "isdf_gemm_f64_noalloc",
    "isdf_gemm_f64_noalloc_capacity",
    "isdf_rfft3",
    "isdf_grids_for_threshold",
    "isdf_exchange_occ",
    "isdf_save",
    "isdf_load",
    "isdf_plan_batch",
    "isdf_exchange_graph",
    "isdf_exchange_graph_run",
    "isdf_exchange_graph_destroy",
    "isdf_autotune_table",
    "isdf_release_fit",
]


class isdf_system(ctypes.Structure):
    _fields_ = [
        ("lattice", c_double * 9),
        ("natom", c_int),
        ("xyz", POINTER(c_double)),
        ("nshell", c_int),
        ("shell_atom", POINTER(c_int)),
        ("shell_l", POINTER(c_int)),
        ("shell_exp", POINTER(c_double)),
        ("nlevel", c_int),
        ("grid", POINTER(c_int)),
        ("level_min_exp", POINTER(c_double)),
        ("image_tol", c_double),
    ]


class isdf_options(ctypes.Structure):
    _fields_ = [
        ("precision", c_int),
        ("tie_rel", c_double),
        ("tie_abs", c_double),
        ("reg_rel", c_double),
        ("col_batch", c_int),
        ("timeout_ms", c_int),
        ("prefilter", c_int),
        ("profile", c_int),
        ("select_block", c_int),
        ("coarse_sinc", c_int),
        ("local_grids", c_int),
        ("local_eps_r", c_double),
        ("local_tol", c_double),
        ("local_cap", c_int),
    ]


class IsdfError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {message}")
        self.status = status
        self.message = message


_lib = None


def load_library(build_if_missing: bool = True):
    """Load libisdf.so (building it first if needed).  Raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build_library()
    if not os.path.exists(path):
        raise RuntimeError(f"libisdf.so not found at {path}; build it with paper_2404_09373_gb300.build")
    lib = ctypes.CDLL(path)
    lib.isdf_options_default.argtypes = [POINTER(isdf_options)]
    lib.isdf_options_default.restype = None
    lib.isdf_plan.argtypes = [POINTER(isdf_system), POINTER(isdf_options), c_void_p, POINTER(c_void_p)]
    lib.isdf_plan.restype = c_int
    lib.isdf_select_points.argtypes = [c_void_p, c_int, c_double, c_void_p, c_int64, c_void_p, c_void_p,
                                       POINTER(c_int)]
    lib.isdf_select_points.restype = c_int
    lib.isdf_fit.argtypes = [c_void_p, c_void_p, c_int]
    lib.isdf_fit.restype = c_int
    lib.isdf_coulomb.argtypes = [c_void_p, c_void_p]
    lib.isdf_coulomb.restype = c_int
    lib.isdf_exchange.argtypes = [c_void_p, c_void_p, c_int, c_void_p, POINTER(c_double)]
    lib.isdf_exchange.restype = c_int
    lib.isdf_get_size.argtypes = [c_void_p, c_int]
    lib.isdf_get_size.restype = c_int64
    lib.isdf_get.argtypes = [c_void_p, c_int, c_void_p]
    lib.isdf_get.restype = c_int
    lib.isdf_last_error.argtypes = [c_void_p]
    lib.isdf_last_error.restype = ctypes.c_char_p
    lib.isdf_destroy.argtypes = [c_void_p]
    lib.isdf_destroy.restype = None
    lib.isdf_profile_json.argtypes = [c_void_p]
    lib.isdf_profile_json.restype = ctypes.c_char_p
    lib.isdf_kernel_launches.argtypes = []
    lib.isdf_kernel_launches.restype = c_int64
    lib.isdf_gemm_f64.argtypes = [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int64, c_int64, c_int64,
                                  c_double, c_int, c_int, c_void_p]
    lib.isdf_gemm_f64.restype = c_int
    lib.isdf_mlp_num_params.argtypes = []
    lib.isdf_mlp_num_params.restype = c_int
    lib.isdf_features.argtypes = [c_void_p, c_void_p]
    lib.isdf_features.restype = c_int
    lib.isdf_mlp_train_step.argtypes = [c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float, c_void_p, c_void_p,
                                        c_void_p, c_int64, POINTER(ctypes.c_float), c_void_p, c_void_p]
    lib.isdf_mlp_train_step.restype = c_int
    lib.isdf_mlp_score.argtypes = [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]
    lib.isdf_mlp_score.restype = c_int
    lib.isdf_propose.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    lib.isdf_propose.restype = c_int
    lib.isdf_propose_residual.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.isdf_propose_residual.restype = c_int
    lib.isdf_rfft3.argtypes = [c_void_p, c_int, c_int, c_int, c_int64, c_void_p, c_void_p]
    lib.isdf_rfft3.restype = c_int
    lib.isdf_gemm_f64_noalloc.argtypes = [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int64, c_int64,
                                          c_int64, c_double, c_int, c_void_p]
    lib.isdf_gemm_f64_noalloc.restype = c_int
    lib.isdf_plan_batch.argtypes = [POINTER(isdf_system), c_int, POINTER(isdf_options), c_void_p, c_void_p]
    lib.isdf_plan_batch.restype = c_int
    lib.isdf_exchange_graph.argtypes = [c_void_p, c_int, c_void_p, c_int, c_void_p, POINTER(c_void_p)]
    lib.isdf_exchange_graph.restype = c_int
    lib.isdf_exchange_graph_run.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    lib.isdf_exchange_graph_run.restype = c_int
    lib.isdf_exchange_graph_destroy.argtypes = [c_void_p]
    lib.isdf_exchange_graph_destroy.restype = None
    lib.isdf_autotune_table.argtypes = []
    lib.isdf_autotune_table.restype = ctypes.c_char_p
    lib.isdf_save.argtypes = [c_void_p, ctypes.c_char_p]
    lib.isdf_save.restype = c_int
    lib.isdf_release_fit.argtypes = [c_void_p]
    lib.isdf_release_fit.restype = c_int
    lib.isdf_load.argtypes = [c_void_p, ctypes.c_char_p]
    lib.isdf_load.restype = c_int
    lib.isdf_exchange_occ.argtypes = [c_void_p, c_void_p, c_int, c_void_p, POINTER(c_double)]
    lib.isdf_exchange_occ.restype = c_int
    lib.isdf_grids_for_threshold.argtypes = [POINTER(isdf_system), c_double, POINTER(c_int)]
    lib.isdf_grids_for_threshold.restype = c_int
    lib.isdf_gemm_f64_noalloc_capacity.argtypes = []
    lib.isdf_gemm_f64_noalloc_capacity.restype = c_int64
    _lib = lib
    return lib


def _addr(x, dtype):
    """Raw pointer of a C-contiguous numpy array or torch tensor of ``dtype``."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"expected a C-contiguous {np.dtype(dtype)} array")
        return x.ctypes.data
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        tmap = {np.dtype(np.float64): torch.float64, np.dtype(np.int64): torch.int64, np.dtype(np.int32): torch.int32}
        if x.dtype != tmap[np.dtype(dtype)] or not x.is_contiguous():
            raise ValueError(f"expected a contiguous {np.dtype(dtype)} tensor")
        return x.data_ptr()
    raise TypeError("expected a numpy array or a torch tensor")


def _default_stream():
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return 0


def default_options(**kw):
    lib = load_library()
    o = isdf_options()
    lib.isdf_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Plan:
    """Owner of an ``isdf_plan_t``; destroyed with ``close()`` or on collection."""

    def __init__(self, handle, lib, system, options=None):
        self.handle = handle
        self._lib = lib
        self.system = system
        self.options = options

    def close(self):
        if self.handle:
            self._lib.isdf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != ISDF_OK:
            raise IsdfError(st, self._lib.isdf_last_error(self.handle).decode())


def _system_struct(system: dict, need_grid=True):
    """isdf_system for a system dict; returns (struct, arrays kept alive)."""
    edges = np.asarray(system["edges"], dtype=np.float64)
    xyz = np.ascontiguousarray(system["xyz"], dtype=np.float64)
    sa = np.ascontiguousarray(system["shell_atom"], dtype=np.int32)
    sl = np.ascontiguousarray(system["shell_l"], dtype=np.int32)
    se = np.ascontiguousarray(system["shell_exp"], dtype=np.float64)
    lme = np.ascontiguousarray(system["level_min_exp"], dtype=np.float64)
    if need_grid:
        grid = np.ascontiguousarray(system["grids"], dtype=np.int32).reshape(-1, 3)
    else:
        grid = np.zeros((lme.size + 1, 3), dtype=np.int32)
    s = isdf_system()
    for i in range(9):
        s.lattice[i] = 0.0
    for a in range(3):
        s.lattice[4 * a] = float(edges[a])
    s.natom = xyz.shape[0]
    s.xyz = xyz.ctypes.data_as(POINTER(c_double))
    s.nshell = se.shape[0]
    s.shell_atom = sa.ctypes.data_as(POINTER(c_int))
    s.shell_l = sl.ctypes.data_as(POINTER(c_int))
    s.shell_exp = se.ctypes.data_as(POINTER(c_double))
    s.nlevel = grid.shape[0]
    s.grid = grid.ctypes.data_as(POINTER(c_int))
    s.level_min_exp = lme.ctypes.data_as(POINTER(c_double)) if lme.size else None
    s.image_tol = float(system["image_tol"])
    return s, (xyz, sa, sl, se, grid, lme)


def isdf_plan(system: dict, options=None, stream=None) -> Plan:
    lib = load_library()
    if options is None:
        options = default_options()
    elif isinstance(options, dict):
        options = default_options(**options)
    s, keep = _system_struct(system)
    h = c_void_p()
    st = lib.isdf_plan(ctypes.byref(s), ctypes.byref(options), c_void_p(_default_stream() if stream is None else stream),
                       ctypes.byref(h))
    if st != ISDF_OK:
        raise IsdfError(st, lib.isdf_last_error(None).decode())
    return Plan(h.value, lib, system, options)


def isdf_plan_batch(systems, options=None, streams=None):
    """Plans for many cells; the basis of all cells and levels is evaluated by
    one launch of each basis kernel.  Returns a list of Plan."""
    lib = load_library()
    if options is None:
        options = default_options()
    elif isinstance(options, dict):
        options = default_options(**options)
    n = len(systems)
    arr = (isdf_system * n)()
    keep = []
    for i, sysd in enumerate(systems):
        st_, k = _system_struct(sysd)
        arr[i] = st_
        keep.append(k)
    sp = None
    if streams is not None:
        sp = (c_void_p * n)(*[c_void_p(int(x)) for x in streams])
    out = (c_void_p * n)()
    st = lib.isdf_plan_batch(arr, n, ctypes.byref(options), sp, out)
    if st != ISDF_OK:
        raise IsdfError(st, lib.isdf_last_error(None).decode())
    return [Plan(out[i], lib, systems[i], options) for i in range(n)]


class ExchangeGraph:
    """One CUDA graph holding the exchange builds of several fitted plans."""

    def __init__(self, plans, n_occ, occ=False, stream=None):
        self._lib = load_library()
        self.plans = list(plans)
        self.n = [int(x) for x in n_occ]
        self.occ = bool(occ)
        hp = (c_void_p * len(self.plans))(*[c_void_p(p.handle) for p in self.plans])
        nn = (c_int * len(self.plans))(*self.n)
        h = c_void_p()
        st = self._lib.isdf_exchange_graph(hp, len(self.plans), nn, int(self.occ),
                                           c_void_p(_default_stream() if stream is None else stream), ctypes.byref(h))
        if st != ISDF_OK:
            raise IsdfError(st, self._lib.isdf_last_error(None).decode())
        self.handle = h.value

    def run(self, Cs, outs=None):
        """Replay with orbitals Cs[i]; returns (outputs, E_x list).  Outputs are
        NumPy arrays unless ``outs`` (arrays or tensors) are given."""
        m = len(self.plans)
        Cs = [np.ascontiguousarray(C, dtype=np.float64) if isinstance(C, np.ndarray) else C for C in Cs]
        if outs is None:
            outs = [np.zeros((p.system_nfun, n) if self.occ else (p.system_nfun, p.system_nfun))
                    for p, n in zip(self._nfun_views(), self.n)]
        cp = (c_void_p * m)(*[c_void_p(_addr(C, np.float64)) for C in Cs])
        op = (c_void_p * m)(*[c_void_p(_addr(o, np.float64)) for o in outs])
        ex = (c_double * m)()
        st = self._lib.isdf_exchange_graph_run(self.handle, cp, op, ex)
        if st != ISDF_OK:
            raise IsdfError(st, self._lib.isdf_last_error(None).decode())
        return outs, list(ex)

    def _nfun_views(self):
        from types import SimpleNamespace

        return [SimpleNamespace(system_nfun=int(sum(1 if l == 0 else 3 for l in p.system["shell_l"])))
                for p in self.plans]

    def close(self):
        if self.handle:
            self._lib.isdf_exchange_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def isdf_grids_for_threshold(system: dict, eps_K: float):
    """Grid points per axis of every level from the accuracy threshold eps_K
    (host computation in the library).  Returns an int array (nlevel, 3)."""
    lib = load_library()
    s, keep = _system_struct(system, need_grid=False)
    out = np.zeros((s.nlevel, 3), dtype=np.int32)
    st = lib.isdf_grids_for_threshold(ctypes.byref(s), c_double(eps_K), out.ctypes.data_as(POINTER(c_int)))
    if st != ISDF_OK:
        raise IsdfError(st, lib.isdf_last_error(None).decode())
    return out


def isdf_select_points(plan: Plan, nip: int, tol: float = 0.0, cand=None, piv_out=None, dval_out=None):
    """Returns (pivot codes, pivot values) -- numpy unless outputs are given.
    With options.local_grids the atoms' local pivots come first and the
    outputs must hold nip + natom * local_cap values."""
    size = nip
    if plan.options is not None and plan.options.local_grids:
        size += len(plan.system["xyz"]) * int(plan.options.local_cap)
    piv = np.zeros(size, dtype=np.int64) if piv_out is None else piv_out
    dv = np.zeros(size, dtype=np.float64) if dval_out is None else dval_out
    cptr = None
    ncand = 0
    if cand is not None:
        cand = cand if not isinstance(cand, np.ndarray) else np.ascontiguousarray(cand, dtype=np.int64)
        cptr = _addr(cand, np.int64)
        ncand = int(cand.shape[0])
    nfound = c_int(0)
    st = plan._lib.isdf_select_points(plan.handle, int(nip), float(tol), cptr, ncand, _addr(piv, np.int64),
                                      _addr(dv, np.float64), ctypes.byref(nfound))
    plan._check(st)
    return piv[: nfound.value], dv[: nfound.value]


def isdf_fit(plan: Plan, piv):
    if isinstance(piv, np.ndarray):
        piv = np.ascontiguousarray(piv, dtype=np.int64)
    plan._check(plan._lib.isdf_fit(plan.handle, _addr(piv, np.int64), int(piv.shape[0])))


def isdf_coulomb(plan: Plan, V_out=None):
    plan._check(plan._lib.isdf_coulomb(plan.handle, _addr(V_out, np.float64)))
    return V_out


def isdf_exchange(plan: Plan, C, K_out=None):
    """Returns (K, E_x); K is ``K_out`` or a new numpy array."""
    if isinstance(C, np.ndarray):
        C = np.ascontiguousarray(C, dtype=np.float64)
    N = int(C.shape[0])
    K = np.zeros((N, N)) if K_out is None else K_out
    ex = c_double(0.0)
    plan._check(plan._lib.isdf_exchange(plan.handle, _addr(C, np.float64), int(C.shape[1]), _addr(K, np.float64),
                                        ctypes.byref(ex)))
    return K, ex.value


def isdf_exchange_occ(plan: Plan, C, KC_out=None):
    """occ-RI output K C (N x n) and E_x, without forming K."""
    if isinstance(C, np.ndarray):
        C = np.ascontiguousarray(C, dtype=np.float64)
    N, n = int(C.shape[0]), int(C.shape[1])
    KC = np.zeros((N, n)) if KC_out is None else KC_out
    ex = c_double(0.0)
    plan._check(plan._lib.isdf_exchange_occ(plan.handle, _addr(C, np.float64), n, _addr(KC, np.float64),
                                            ctypes.byref(ex)))
    return KC, ex.value


def isdf_autotune_table():
    """Split-K choices the library measured so far (list of dicts)."""
    import json

    return json.loads(load_library().isdf_autotune_table().decode())


def isdf_release_fit(plan: Plan):
    """Free the buffers the exchange build does not read (after isdf_coulomb)."""
    plan._check(plan._lib.isdf_release_fit(plan.handle))


def isdf_save(plan: Plan, path):
    """Write the pivots, X^L, X^N and V of a plan (after isdf_coulomb)."""
    plan._check(plan._lib.isdf_save(plan.handle, os.fsencode(path)))


def isdf_load(plan: Plan, path):
    """Read a checkpoint into a plan of the same system; exchange builds follow."""
    plan._check(plan._lib.isdf_load(plan.handle, os.fsencode(path)))


def isdf_get(plan: Plan, what: int, dst=None):
    n = int(plan._lib.isdf_get_size(plan.handle, what))
    if n == 0:
        raise IsdfError(ISDF_ERR_STATE, "not available")
    dtype = _GET_DTYPE.get(what, np.float64)
    if dst is None:
        dst = np.zeros(n, dtype=dtype)
    if isinstance(dst, np.ndarray):
        if dst.dtype != dtype or dst.size < n:
            raise ValueError(f"isdf_get({what}) needs {n} elements of {np.dtype(dtype)}")
    elif dst.numel() < n:
        raise ValueError(f"isdf_get({what}) needs {n} elements")
    dtype = dst.dtype if isinstance(dst, np.ndarray) else None
    plan._check(plan._lib.isdf_get(plan.handle, what, _addr(dst, dtype) if dtype is not None else dst.data_ptr()))
    return dst


def isdf_destroy(plan: Plan):
    plan.close()


def isdf_profile_json(plan: Plan) -> dict:
    import json

    return json.loads(plan._lib.isdf_profile_json(plan.handle).decode())


def isdf_gemm_f64(A, B, C, alpha=1.0, slices=5, splits=1, stream=None):
    """C = alpha A B^T on the tensor cores (torch CUDA float64 tensors, row-major)."""
    lib = load_library()
    M, K = A.shape
    N = B.shape[0]
    st = lib.isdf_gemm_f64(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, A.stride(0), B.stride(0), C.stride(0),
                           float(alpha), int(slices), int(splits),
                           c_void_p(_default_stream() if stream is None else stream))
    if st != ISDF_OK:
        raise IsdfError(st, lib.isdf_last_error(None).decode())
    return C


def _dptr(t):
    return None if t is None else t.data_ptr()


def isdf_features(plan: Plan, out=None):
    """Features (npoints x 8 float32): numpy unless a torch CUDA tensor is given."""
    n = int(isdf_get(plan, GET_NPOINTS)[0])
    if out is None:
        out = np.zeros((n, 8), dtype=np.float32)
        plan._check(plan._lib.isdf_features(plan.handle, out.ctypes.data))
    else:
        if out.numel() < 8 * n:
            raise ValueError(f"features need {n} x 8 floats")
        plan._check(plan._lib.isdf_features(plan.handle, out.data_ptr()))
    return out


def isdf_mlp_train_step(params, m, v, step, lr, X, y, w, grad_out=None, stream=None):
    """One Adam step (torch CUDA float32 tensors).  Returns the loss before the step."""
    lib = load_library()
    loss = ctypes.c_float(0.0)
    st = lib.isdf_mlp_train_step(params.data_ptr(), _dptr(m), _dptr(v), int(step), float(lr), X.data_ptr(),
                                 y.data_ptr(), w.data_ptr(), int(X.shape[0]), ctypes.byref(loss), _dptr(grad_out),
                                 c_void_p(_default_stream() if stream is None else stream))
    if st != ISDF_OK:
        raise IsdfError(st, lib.isdf_last_error(None).decode())
    return loss.value


def isdf_mlp_score(params, X, out, stream=None):
    lib = load_library()
    st = lib.isdf_mlp_score(params.data_ptr(), X.data_ptr(), int(X.shape[0]), out.data_ptr(),
                            c_void_p(_default_stream() if stream is None else stream))
    if st != ISDF_OK:
        raise IsdfError(st, lib.isdf_last_error(None).decode())
    return out


def isdf_propose(plan: Plan, params, quota):
    """Per-level quotas (sequence of nlevel ints) -> candidate pivot codes."""
    q = np.ascontiguousarray(quota, dtype=np.int64)
    out = np.zeros(int(q.sum()), dtype=np.int64)
    plan._check(plan._lib.isdf_propose(plan.handle, params.data_ptr(), q.ctypes.data, out.ctypes.data))
    return out


def isdf_propose_residual(plan: Plan, quota):
    """After isdf_fit: per level the quota[l] points with the largest fit residual (pivot codes)."""
    q = np.ascontiguousarray(quota, dtype=np.int64)
    out = np.zeros(int(q.sum()), dtype=np.int64)
    plan._check(plan._lib.isdf_propose_residual(plan.handle, q.ctypes.data, out.ctypes.data))
    return out


def isdf_rfft3(f, S=None, stream=None):
    """Half spectra of a batch of real grids (torch CUDA float64, shape (b, nz, ny, nx))
    -> complex128 tensor (b, nz, ny, nx/2+1), computed by the library's double-float transform."""
    import torch

    b, nz, ny, nx = f.shape
    if S is None:
        S = torch.empty((b, nz, ny, nx // 2 + 1), dtype=torch.complex128, device=f.device)
    lib = load_library()
    st = lib.isdf_rfft3(f.data_ptr(), nx, ny, nz, b, S.data_ptr(),
                        c_void_p(_default_stream() if stream is None else stream))
    if st != ISDF_OK:
        raise IsdfError(st, lib.isdf_last_error(None).decode())
    return S


def isdf_kernel_launches() -> int:
    return int(load_library().isdf_kernel_launches())
