"""Thin ctypes binding of libslqr (include/slqr.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libslqr.so.  There is no fallback: if the library is missing or does
not load, importing this module raises.  Build it with
``python -m paper_2506_09463_gb300.build`` (or ``__graft_entry__.build()``).

Pointers are passed as Python ints (device addresses, e.g. ``tensor.data_ptr()``)
and streams as ints (``torch.cuda.current_stream().cuda_stream``; 0 = legacy
default stream).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

# SLQR_CHECKED=1 loads the checked build (build(checked=True)) instead
LIB_PATH = _build.LIB_PATH_CHECKED if os.environ.get("SLQR_CHECKED") == "1" else _build.LIB_PATH

SLQR_OK = 0
SLQR_PENDING = 1
SLQR_EINVAL = -1
SLQR_ENOMEM = -2
SLQR_ECUDA = -3
SLQR_ETIMEOUT = -4
SLQR_ERANK = -5
SLQR_EBUSY = -6
SLQR_ENOTFOUND = -7

STATUS_NAMES = {
    -8: "SLQR_ENOCONV", 2: "SLQR_FALLBACK", -9: "SLQR_ECHECK",
    SLQR_OK: "SLQR_OK", SLQR_PENDING: "SLQR_PENDING", SLQR_EINVAL: "SLQR_EINVAL",
    SLQR_ENOMEM: "SLQR_ENOMEM", SLQR_ECUDA: "SLQR_ECUDA", SLQR_ETIMEOUT: "SLQR_ETIMEOUT",
    SLQR_ERANK: "SLQR_ERANK", SLQR_EBUSY: "SLQR_EBUSY", SLQR_ENOTFOUND: "SLQR_ENOTFOUND",
}

SLQR_ENOCONV = -8
SLQR_FALLBACK = 2
SLQR_ECHECK = -9
SLQR_REFINE_AUTO, SLQR_REFINE_BJORCK, SLQR_REFINE_GMRES, SLQR_REFINE_FP64 = 0, 1, 2, 3
SLQR_REQ_FACTOR, SLQR_REQ_SOLVE, SLQR_REQ_FACTOR_SOLVE, SLQR_REQ_RELEASE = 1, 2, 3, 4


class SlqrRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("m", ctypes.c_int), ("n", ctypes.c_int),
                ("lda", ctypes.c_int), ("A", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("handle", ctypes.c_uint64), ("prec", ctypes.c_int),
                ("structure", ctypes.c_int)]


class SlqrMixedOpts(ctypes.Structure):
    _fields_ = [("refine", ctypes.c_int), ("max_sweeps", ctypes.c_int), ("tol", ctypes.c_double),
                ("gmres_max_iters", ctypes.c_int), ("gmres_restart", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("fp64_fallback", ctypes.c_int),
                ("structure", ctypes.c_int)]


class SlqrMixedInfo(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("sweeps", ctypes.c_int), ("gmres_steps", ctypes.c_int),
                ("gmres_iters", ctypes.c_int), ("err", ctypes.c_double),
                ("kappa_est", ctypes.c_double)]


class SlqrResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("handle", ctypes.c_uint64),
                ("residual_norm", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("err", ctypes.c_double)]


# (name, restype, argtypes) of every entry point declared in include/slqr.h
_c_int, _c_size, _vp, _dbl = ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_double
SIGNATURES = [
    ("slqr_create", _c_int, [ctypes.POINTER(_vp), _c_int, _c_size]),
    ("slqr_destroy", None, [_vp]),
    ("slqr_last_error", ctypes.c_char_p, [_vp]),
    ("slqr_sync", _c_int, [_vp, _vp]),
    ("slqr_check_bounded_wait", _c_int, [_vp, ctypes.c_uint, _vp]),
    ("slqr_set_spin_limit", _c_int, [_vp, ctypes.c_uint]),
    ("slqr_is_checked", _c_int, []),
    ("slqr_check_selftest", _c_int, [_vp]),
    ("slqr_panel_width", _c_int, [_c_int, _c_int]),
    ("slqr_wy_size", _c_size, [_c_int, _c_int]),
    ("slqr_max_rows", _c_int, []),
    ("slqr_set_tuning", None, [_c_int, _c_int]),
    ("slqr_set_panel_cluster", _c_int, [_c_int]),
    ("slqr_get_panel_cluster", _c_int, []),
    ("slqr_set_panel_cluster_variant", _c_int, [_c_int]),
    ("slqr_set_fused_lookahead", _c_int, [_c_int]),
    ("slqr_get_fused_lookahead", _c_int, []),
    ("slqr_autotune", _c_int, [_vp, _c_int, _c_int, ctypes.POINTER(_dbl), ctypes.POINTER(_c_int),
                               ctypes.POINTER(_c_int)]),
    ("slqr_factor", _c_int, [_vp, _c_int, _c_int, _vp, _c_int, _vp, _vp, _vp]),
    ("slqr_apply_qt", _c_int, [_vp, _c_int, _c_int, _vp, _c_int, _vp, _vp, _c_int, _vp, _c_int, _vp]),
    ("slqr_solve_r", _c_int, [_vp, _c_int, _vp, _c_int, _c_int, _vp, _c_int, _vp]),
    ("slqr_factor_stacked", _c_int, [_vp, _c_int, _c_int, _vp, _c_int, _vp, _vp, _vp]),
    ("slqr_apply_qt_stacked", _c_int, [_vp, _c_int, _c_int, _vp, _c_int, _vp, _vp, _c_int, _vp,
                                       _c_int, _vp]),
    ("slqr_profile", _c_int, [_vp, _c_int]),
    ("slqr_profile_read", _c_int, [_vp, _c_int, ctypes.POINTER(_dbl),
                                   ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_dbl)]),
    ("slqr_launch_count", ctypes.c_longlong, [_vp]),
    ("slqr_measure_peak", _c_int, [_vp, _c_int, ctypes.POINTER(_dbl)]),
    ("slqr_factor_noalloc", _c_int, [_c_int, _c_int, _vp, _c_int, _vp, _vp, _vp, _vp]),
    ("slqr_batch_factor", _c_int, [_vp, _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                   ctypes.POINTER(_vp), ctypes.POINTER(_c_int),
                                   ctypes.POINTER(_vp), ctypes.POINTER(_vp), _c_int, _vp, _vp,
                                   _vp]),
    ("slqr_batch_max_rows", _c_int, []),
    ("slqr_batch_classes", _c_int, []),
    ("slqr_batch_class_rows", _c_int, [_c_int]),
    ("slqr_batch_set_tuning", _c_int, [_c_int, _c_int, _c_int, _c_int, _c_int]),
    ("slqr_batch_get_tuning", _c_int, [_c_int, _c_int, ctypes.POINTER(_c_int),
                                       ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    ("slqr_batch_autotune", _c_int, [_vp, _c_int, _c_int, ctypes.POINTER(_c_int),
                                     ctypes.POINTER(_c_int), _c_int, ctypes.POINTER(_c_int),
                                     ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                     ctypes.POINTER(_dbl)]),
    ("slqr_batch_plan_create", _c_int, [_vp, _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                        ctypes.POINTER(_c_int), ctypes.POINTER(_vp),
                                        ctypes.POINTER(_c_int), ctypes.POINTER(_vp),
                                        ctypes.POINTER(_vp), _c_int, _vp, _vp,
                                        ctypes.POINTER(_vp)]),
    ("slqr_batch_plan_launch", _c_int, [_vp, _vp]),
    ("slqr_batch_plan_destroy", None, [_vp]),
    ("slqr_batch_factor_stacked", _c_int, [_vp, _c_int, ctypes.POINTER(_c_int),
                                           ctypes.POINTER(_c_int), ctypes.POINTER(_vp),
                                           ctypes.POINTER(_c_int), ctypes.POINTER(_vp),
                                           ctypes.POINTER(_vp), _c_int, _vp, _vp, _vp]),
    ("slqr_submit", _c_int, [_vp, ctypes.POINTER(SlqrRequest), ctypes.POINTER(ctypes.c_uint64)]),
    ("slqr_poll", _c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(SlqrResult)]),
    ("slqr_server_bytes_in_use", _c_size, [_vp]),
    ("slqr_lstsq_mixed", _c_int, [_vp, _c_int, _c_int, _vp, _c_int, _vp, _vp, _c_int, _c_int, _dbl,
                                  ctypes.POINTER(_c_int), ctypes.POINTER(_dbl), _vp]),
    ("slqr_lstsq_mixed_ex", _c_int, [_vp, _c_int, _c_int, _vp, _c_int, _vp, _vp, _c_int,
                                     ctypes.POINTER(SlqrMixedOpts), ctypes.POINTER(SlqrMixedInfo),
                                     _vp]),
    ("slqr_noalloc_max_rows", _c_int, []),
    ("slqr_noalloc_max_cols", _c_int, []),
]

KERNEL_PANEL, KERNEL_VTX, KERNEL_TW, KERNEL_UPD, KERNEL_WY_REBUILD, KERNEL_TRSM, KERNEL_BATCH = \
    range(7)
KERNEL_NAMES = ["panel", "vtx", "tw", "upd", "wy_rebuild", "trsm", "batch"]
SLQR_FP64 = 0
SLQR_FP32 = 1
SLQR_TF32 = 2
SLQR_BF16X3 = 3
SLQR_DENSE = 0
SLQR_STACKED = 1


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH} missing); run "
            "`python -m paper_2506_09463_gb300.build` first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


class SlqrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def slqr_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    ctx = _vp()
    st = _lib.slqr_create(ctypes.byref(ctx), device, hbm_budget_bytes)
    if st != SLQR_OK:
        raise SlqrError(st, f"slqr_create(device={device}) failed")
    return ctx.value


def slqr_destroy(ctx: int) -> None:
    _lib.slqr_destroy(ctx)


def slqr_last_error(ctx: int) -> str:
    return _lib.slqr_last_error(ctx).decode()


def slqr_sync(ctx: int, stream: int = 0) -> int:
    return _lib.slqr_sync(ctx, stream)


def slqr_panel_width(m: int, n: int) -> int:
    return _lib.slqr_panel_width(m, n)


def slqr_wy_size(m: int, n: int) -> int:
    return _lib.slqr_wy_size(m, n)


def slqr_max_rows() -> int:
    return _lib.slqr_max_rows()


def slqr_set_tuning(panel_width: int = 0, panel_rows_min: int = 0) -> None:
    _lib.slqr_set_tuning(panel_width, panel_rows_min)


def slqr_is_checked() -> bool:
    return bool(_lib.slqr_is_checked())


def slqr_check_selftest(ctx: int) -> int:
    return _lib.slqr_check_selftest(ctx)


def slqr_set_panel_cluster(ctas: int = 0) -> int:
    return _lib.slqr_set_panel_cluster(ctas)


def slqr_get_panel_cluster() -> int:
    return _lib.slqr_get_panel_cluster()


def slqr_set_panel_cluster_variant(variant: int = 0) -> int:
    return _lib.slqr_set_panel_cluster_variant(variant)


def slqr_set_fused_lookahead(enable: int = 1) -> int:
    return _lib.slqr_set_fused_lookahead(enable)


def slqr_get_fused_lookahead() -> int:
    return _lib.slqr_get_fused_lookahead()


def slqr_autotune(ctx, m, n):
    """Returns (status, best_ms, panel_width, rows_min) and keeps that tuning."""
    ms, w, r = _dbl(), _c_int(), _c_int()
    st = _lib.slqr_autotune(ctx, m, n, ctypes.byref(ms), ctypes.byref(w), ctypes.byref(r))
    return st, ms.value, w.value, r.value


def slqr_check_bounded_wait(ctx, polls, stream=None) -> int:
    return _lib.slqr_check_bounded_wait(ctx, polls, stream)


def slqr_set_spin_limit(ctx, polls: int) -> int:
    return _lib.slqr_set_spin_limit(ctx, polls)


def slqr_factor(ctx, m, n, A, lda, up, wy, stream) -> int:
    return _lib.slqr_factor(ctx, m, n, A, lda, up, wy, stream)


def slqr_apply_qt(ctx, m, n, A, lda, up, wy, nrhs, B, ldb, stream) -> int:
    return _lib.slqr_apply_qt(ctx, m, n, A, lda, up, wy, nrhs, B, ldb, stream)


def slqr_solve_r(ctx, n, A, lda, nrhs, B, ldb, stream) -> int:
    return _lib.slqr_solve_r(ctx, n, A, lda, nrhs, B, ldb, stream)


def slqr_factor_stacked(ctx, n, m_eq, A, lda, up, wy, stream) -> int:
    return _lib.slqr_factor_stacked(ctx, n, m_eq, A, lda, up, wy, stream)


def slqr_apply_qt_stacked(ctx, n, m_eq, A, lda, up, wy, nrhs, B, ldb, stream) -> int:
    return _lib.slqr_apply_qt_stacked(ctx, n, m_eq, A, lda, up, wy, nrhs, B, ldb, stream)


def slqr_profile(ctx: int, enable: bool) -> int:
    return _lib.slqr_profile(ctx, 1 if enable else 0)


def slqr_profile_read(ctx: int, kernel: int):
    """(ms, launches, flops) recorded for one kernel family."""
    ms, n, fl = _dbl(), ctypes.c_longlong(), _dbl()
    st = _lib.slqr_profile_read(ctx, kernel, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl))
    check(ctx, st, "slqr_profile_read")
    return ms.value, n.value, fl.value


SLQR_PEAK_FP64_FMA, SLQR_PEAK_TF32_TC = 0, 1


def slqr_measure_peak(ctx, kind: int):
    """Returns (status, TFLOP/s) of the device's FP64 FMA or TF32 tensor-core probe."""
    v = _dbl()
    st = _lib.slqr_measure_peak(ctx, kind, ctypes.byref(v))
    return st, v.value


def slqr_launch_count(ctx: int) -> int:
    return _lib.slqr_launch_count(ctx)


def _int_array(values):
    return (_c_int * len(values))(*[int(v) for v in values])


def _ptr_array(values):
    return (_vp * len(values))(*[v if v else None for v in values])


def slqr_batch_factor(ctx, m_list, n_list, A_ptrs, lda_list, up_ptrs, b_ptrs, prec, status,
                      err, stream) -> int:
    """Host lists of sizes and of device pointers; status / err device pointers or None."""
    count = len(m_list)
    return _lib.slqr_batch_factor(
        ctx, count, _int_array(m_list), _int_array(n_list), _ptr_array(A_ptrs),
        _int_array(lda_list), _ptr_array(up_ptrs) if up_ptrs is not None else None,
        _ptr_array(b_ptrs) if b_ptrs is not None else None, prec, status, err, stream)


def slqr_batch_max_rows() -> int:
    return _lib.slqr_batch_max_rows()


def slqr_batch_classes() -> int:
    return _lib.slqr_batch_classes()


def slqr_batch_class_rows(m_class: int) -> int:
    return _lib.slqr_batch_class_rows(m_class)


def slqr_batch_set_tuning(prec: int, m_class: int, panel_width: int, tile_cols: int,
                          resident: int = 0) -> int:
    return _lib.slqr_batch_set_tuning(prec, m_class, panel_width, tile_cols, resident)


def slqr_batch_get_tuning(prec: int, m_class: int):
    """Returns (status, panel_width, tile_cols, resident)."""
    nb, tc, rs = _c_int(), _c_int(), _c_int()
    st = _lib.slqr_batch_get_tuning(prec, m_class, ctypes.byref(nb), ctypes.byref(tc),
                                    ctypes.byref(rs))
    return st, nb.value, tc.value, rs.value


def slqr_batch_autotune(ctx, prec: int, m_list=None, n_list=None, sample: int = 0):
    """Returns (status, [(panel_width, tile_cols, resident) per size class],
    (ms_before, ms_after))."""
    k = _lib.slqr_batch_classes()
    nb, tc, rs, ms = (_c_int * k)(), (_c_int * k)(), (_c_int * k)(), (_dbl * 2)()
    count = len(m_list) if m_list is not None else 0
    m_arr = _int_array(m_list) if count else None
    n_arr = _int_array(n_list) if count else None
    st = _lib.slqr_batch_autotune(ctx, prec, count, m_arr, n_arr, sample, nb, tc, rs, ms)
    return st, [(nb[i], tc[i], rs[i]) for i in range(k)], (ms[0], ms[1])


BATCH_SETTINGS = [(8, 32), (8, 64), (16, 16), (16, 32), (16, 64), (32, 16), (32, 32), (32, 64)]


def slqr_batch_plan_create(ctx, m_list, n_list, ntop_list, A_ptrs, lda_list, up_ptrs, b_ptrs,
                           prec, status, err):
    """Returns (status, plan handle).  ntop_list may be None (all dense)."""
    count = len(m_list)
    plan = _vp()
    st = _lib.slqr_batch_plan_create(
        ctx, count, _int_array(m_list), _int_array(n_list),
        _int_array(ntop_list) if ntop_list is not None else None, _ptr_array(A_ptrs),
        _int_array(lda_list), _ptr_array(up_ptrs) if up_ptrs is not None else None,
        _ptr_array(b_ptrs) if b_ptrs is not None else None, prec, status, err,
        ctypes.byref(plan))
    return st, plan.value


def slqr_batch_plan_launch(plan, stream) -> int:
    return _lib.slqr_batch_plan_launch(plan, stream)


def slqr_batch_plan_destroy(plan) -> None:
    _lib.slqr_batch_plan_destroy(plan)


def slqr_batch_factor_stacked(ctx, n_list, meq_list, A_ptrs, lda_list, up_ptrs, b_ptrs, prec,
                              status, err, stream) -> int:
    """As slqr_batch_factor for stacked [L^T; C] problems of n + m_eq rows."""
    count = len(n_list)
    return _lib.slqr_batch_factor_stacked(
        ctx, count, _int_array(n_list), _int_array(meq_list), _ptr_array(A_ptrs),
        _int_array(lda_list), _ptr_array(up_ptrs) if up_ptrs is not None else None,
        _ptr_array(b_ptrs) if b_ptrs is not None else None, prec, status, err, stream)


def slqr_submit(ctx, req: SlqrRequest):
    """Returns (status, ticket)."""
    t = ctypes.c_uint64()
    st = _lib.slqr_submit(ctx, ctypes.byref(req), ctypes.byref(t))
    return st, t.value


def slqr_poll(ctx, ticket: int):
    """Returns (status, SlqrResult): SLQR_PENDING until the request is done."""
    out = SlqrResult()
    st = _lib.slqr_poll(ctx, ticket, ctypes.byref(out))
    return st, out


def slqr_lstsq_mixed(ctx, m, n, A, lda, b, x, prec, max_iter, tol, stream):
    """Returns (status, iterations, last relative step)."""
    it, err = _c_int(), _dbl()
    st = _lib.slqr_lstsq_mixed(ctx, m, n, A, lda, b, x, prec, max_iter, tol, ctypes.byref(it),
                               ctypes.byref(err), stream)
    return st, it.value, err.value


def slqr_lstsq_mixed_ex(ctx, m, n, A, lda, b, x, prec, stream, refine=SLQR_REFINE_AUTO,
                        max_sweeps=0, tol=0.0, gmres_max_iters=0, gmres_restart=0,
                        gmres_tol=0.0, fp64_fallback=0, structure=0):
    """Returns (status, info) with info a dict of the SlqrMixedInfo fields."""
    opts = SlqrMixedOpts(refine, max_sweeps, tol, gmres_max_iters, gmres_restart, gmres_tol,
                         fp64_fallback, structure)
    info = SlqrMixedInfo()
    st = _lib.slqr_lstsq_mixed_ex(ctx, m, n, A, lda, b, x, prec, ctypes.byref(opts),
                                  ctypes.byref(info), stream)
    return st, {f: getattr(info, f) for f, _ in SlqrMixedInfo._fields_}


def slqr_server_bytes_in_use(ctx) -> int:
    return _lib.slqr_server_bytes_in_use(ctx)


def slqr_factor_noalloc(m, n, A, lda, up, wy, status, stream) -> int:
    """Allocation-free factorization (no context; fixed-size library scratch)."""
    return _lib.slqr_factor_noalloc(m, n, A, lda, up, wy, status, stream)


def slqr_noalloc_max_rows() -> int:
    return _lib.slqr_noalloc_max_rows()


def slqr_noalloc_max_cols() -> int:
    return _lib.slqr_noalloc_max_cols()


def check(ctx: int, status: int, what: str) -> None:
    """Raise SlqrError for a negative status, with the context's message."""
    if status < 0:
        raise SlqrError(status, f"{what}: {slqr_last_error(ctx)}")
