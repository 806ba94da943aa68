"""Python binding of the tile_chol C ABI (include/tile_chol.h): argument marshalling only.

Every function keeps the C name and forwards to ``libtile_chol.so``; all arithmetic runs
in the library's CUDA kernels.  Matrix arguments may be torch tensors (CUDA or CPU) or
numpy arrays; the library itself decides whether a pointer is host or device memory.
A missing or unloadable library raises ``RuntimeError``: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "TC_FP64", "TC_FP32", "TC_FP16", "TC_FP8", "TC_OK", "TileCholError", "tc_config", "tc_stats",
    "lib", "tc_config_default", "tc_create", "tc_destroy", "tc_last_error", "tc_matern_tiles",
    "tile_chol_precision_map", "tile_chol_factor", "tile_chol_factor_ooc", "tile_chol_solve", "tile_chol_logdet",
    "tile_chol_loglik", "tile_chol_loglik_refined", "tile_chol_loglik_solved", "tile_chol_get_factor", "tile_chol_precision_map_noalloc", "tile_chol_factor_batched",
    "tile_chol_solve_batched", "tile_chol_loglik_batched", "Handle", "ntiles",
    "tile_count", "tc_set_wait_limit", "tile_chol_get_factor_batched",
]

TC_FP64, TC_FP32, TC_FP16, TC_FP8 = 0, 1, 2, 3
TC_OK = 0
TC_ERR_ARG, TC_ERR_STATE, TC_ERR_CUDA, TC_ERR_OOM, TC_ERR_TIMEOUT, TC_ERR_HOSTMEM, TC_ERR_UNSUPPORTED = (
    -1, -2, -100, -101, -102, -103, -104)
ERRORS = {-1: "TC_ERR_ARG", -2: "TC_ERR_STATE", -100: "TC_ERR_CUDA", -101: "TC_ERR_OOM",
          -102: "TC_ERR_TIMEOUT", -103: "TC_ERR_HOSTMEM", -104: "TC_ERR_UNSUPPORTED"}

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtile_chol.so")


class TileCholError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class tc_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("ooc", ctypes.c_int),
                ("device_cap_bytes", ctypes.c_int64), ("prefetch_depth", ctypes.c_int),
                ("lookahead", ctypes.c_int), ("fp64_mode", ctypes.c_int), ("ooc_eviction", ctypes.c_int),
                ("fp32_updates", ctypes.c_int), ("wait_limit_us", ctypes.c_int),
                ("wait_test", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class tc_stats(ctypes.Structure):
    _fields_ = [("t_ms", ctypes.c_double), ("flops", ctypes.c_double), ("update_flops", ctypes.c_double * 4),
                ("trsm_flops", ctypes.c_double), ("potrf_flops", ctypes.c_double),
                ("tiles", ctypes.c_int64 * 4), ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
                ("cache_hits", ctypes.c_int64), ("cache_misses", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("refine_iters", ctypes.c_int), ("berr", ctypes.c_double),
                ("info", ctypes.c_int), ("ooc", ctypes.c_int),
                ("t_update_ms", ctypes.c_double * 4), ("t_potrf_ms", ctypes.c_double),
                ("t_trsm_ms", ctypes.c_double), ("t_convert_ms", ctypes.c_double),
                ("update_launches", ctypes.c_int64 * 4), ("tensor_flops", ctypes.c_double * 4)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


_lib = None


def lib() -> ctypes.CDLL:
    """Load libtile_chol.so (built by ``paper_2410_09819_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: run paper_2410_09819_gb300.build.build() first")
    L = ctypes.CDLL(_LIB_PATH)
    vp, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    H = ctypes.c_void_p
    sig = {
        "tc_config_default": (None, [ctypes.POINTER(tc_config)]),
        "tc_create": (ci, [ctypes.POINTER(H), ctypes.POINTER(tc_config)]),
        "tc_destroy": (None, [H]),
        "tc_last_error": (ctypes.c_char_p, [H]),
        "tc_set_wait_limit": (ci, [H, ci, ci]),
        "tc_matern_tiles": (ci, [H, i64, ci, vp, cd, cd, cd, cd, vp]),
        "tile_chol_precision_map": (ci, [H, i64, ci, vp, cd, ci, ci, vp, vp]),
        "tile_chol_factor": (ci, [H, i64, ci, vp, vp, ctypes.POINTER(tc_stats)]),
        "tile_chol_factor_ooc": (ci, [H, i64, ci, vp, vp, ctypes.POINTER(tc_stats)]),
        "tile_chol_factor_mapped": (ci, [H, i64, ci, vp, cd, ci, ci, vp, ctypes.POINTER(tc_stats)]),
        "tile_chol_solve": (ci, [H, ci, vp, i64, vp, i64, ci, cd, ctypes.POINTER(tc_stats)]),
        "tile_chol_logdet": (ci, [H, ctypes.POINTER(cd)]),
        "tile_chol_loglik": (ci, [H, vp, ctypes.POINTER(cd)]),
        "tile_chol_get_factor": (ci, [H, vp]),
        "tile_chol_get_factor_batched": (ci, [H, ci, vp]),
        "tile_chol_loglik_refined": (ci, [H, vp, ci, cd, ctypes.POINTER(cd), ctypes.POINTER(cd)]),
        "tile_chol_loglik_solved": (ci, [H, vp, vp, ctypes.POINTER(cd)]),
        "tile_chol_precision_map_noalloc": (ci, [i64, ci, vp, cd, ci, ci, vp, vp]),
        "tile_chol_factor_batched": (ci, [H, ci, vp, ci, vp, vp, vp, vp, ctypes.POINTER(tc_stats)]),
        "tile_chol_solve_batched": (ci, [H, ci, vp, vp, ci, cd, vp, ctypes.POINTER(tc_stats)]),
        "tile_chol_loglik_batched": (ci, [H, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(x) -> int | None:
    """Address of a torch tensor / numpy array / int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"] and not x.flags["F_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)!r}")


def _need(x, kind: str, count: int | None, what: str) -> None:
    """Reject a torch tensor or numpy array of the wrong element type, or with fewer than
    ``count`` elements, before the library reads or writes through its address (the C ABI sees
    only a pointer).  Raw integer addresses and None pass through unchecked."""
    if x is None or isinstance(x, int):
        return
    if hasattr(x, "data_ptr"):
        dt, size = str(x.dtype).replace("torch.", ""), x.numel()
    elif isinstance(x, np.ndarray):
        dt, size = str(x.dtype), x.size
    else:
        return                                  # _ptr rejects other buffer types
    if dt != kind:
        raise TileCholError(-1, f"{what} must hold {kind} elements, not {dt}")
    if count is not None and size < count:
        raise TileCholError(-1, f"{what} needs at least {count} elements, has {size}")


def _need_tiles(n, b, A_tiles, map_=None, what="A_tiles"):
    """The packed lower tiles (T b^2 doubles) and a precision map (Nt^2 bytes) of order n, tile b;
    sizes are checked only for n, b the library accepts at all (it reports the rest itself)."""
    ok = isinstance(n, (int, np.integer)) and isinstance(b, (int, np.integer)) and n >= 1 and b >= 1
    _need(A_tiles, "float64", tile_count(n, b) * b * b if ok else None, what)
    _need(map_, "uint8", ntiles(n, b) ** 2 if ok else None, "map")


def _check(h, rc: int, allow_positive: bool = False) -> int:
    if rc == TC_OK or (allow_positive and rc > 0):
        return rc
    msg = lib().tc_last_error(h).decode() if h else ""
    raise TileCholError(rc, msg)


def ntiles(n: int, b: int) -> int:
    return -(-n // b)


def tile_count(n: int, b: int) -> int:
    nt = ntiles(n, b)
    return nt * (nt + 1) // 2


def tc_config_default() -> tc_config:
    cfg = tc_config()
    lib().tc_config_default(ctypes.byref(cfg))
    return cfg


def tc_create(cfg: tc_config | None = None):
    h = ctypes.c_void_p()
    rc = lib().tc_create(ctypes.byref(h), ctypes.byref(cfg) if cfg is not None else None)
    if rc != TC_OK:
        raise TileCholError(rc, "tc_create failed")
    return h


def tc_destroy(h) -> None:
    lib().tc_destroy(h)


def tc_last_error(h) -> str:
    return lib().tc_last_error(h).decode()


def tc_set_wait_limit(h, wait_limit_us: int, wait_test: int = 0) -> None:
    _check(h, lib().tc_set_wait_limit(h, wait_limit_us, wait_test))


def tc_matern_tiles(h, n, b, points, sigma2, range_a, nu, nugget, A_tiles) -> None:
    _need(points, "float64", 2 * n if isinstance(n, (int, np.integer)) and n >= 1 else None, "points")
    _need_tiles(n, b, A_tiles)
    _check(h, lib().tc_matern_tiles(h, n, b, _ptr(points), sigma2, range_a, nu, nugget, _ptr(A_tiles)))


def tile_chol_precision_map(h, n, b, A_tiles, eps_high, band, prec_set, map_out, norms_out=None) -> None:
    _need_tiles(n, b, A_tiles, map_out)
    if isinstance(n, (int, np.integer)) and isinstance(b, (int, np.integer)) and n >= 1 and b >= 1:
        _need(norms_out, "float64", ntiles(n, b) ** 2 + 1, "norms_out")
    _check(h, lib().tile_chol_precision_map(h, n, b, _ptr(A_tiles), eps_high, band, prec_set,
                                            _ptr(map_out), _ptr(norms_out)))


def tile_chol_factor(h, n, b, A_tiles, map=None, stats: tc_stats | None = None) -> int:
    """Returns 0, or the 1-based column of a non-positive pivot (matrix not SPD)."""
    _need_tiles(n, b, A_tiles, map)
    return _check(h, lib().tile_chol_factor(h, n, b, _ptr(A_tiles), _ptr(map),
                                            ctypes.byref(stats) if stats is not None else None),
                  allow_positive=True)


def tile_chol_factor_mapped(h, n, b, A_tiles, eps_high, band, prec_set, map_out,
                            stats: tc_stats | None = None) -> int:
    """Precision map and factor on one device copy of A (a host A crosses the link once).
    Returns 0, or the 1-based column of a non-positive pivot."""
    _need_tiles(n, b, A_tiles, map_out)
    return _check(h, lib().tile_chol_factor_mapped(h, n, b, _ptr(A_tiles), eps_high, band, prec_set, _ptr(map_out),
                                                   ctypes.byref(stats) if stats is not None else None),
                  allow_positive=True)


def tile_chol_factor_ooc(h, n, b, A_tiles, map=None, stats: tc_stats | None = None) -> int:
    """Out-of-core factor: A_tiles (host) is overwritten by L.  Returns 0 or the failing column."""
    _need_tiles(n, b, A_tiles, map)
    return _check(h, lib().tile_chol_factor_ooc(h, n, b, _ptr(A_tiles), _ptr(map),
                                                ctypes.byref(stats) if stats is not None else None),
                  allow_positive=True)


def tile_chol_solve(h, nrhs, B, ldb, X, ldx, max_refine=0, target_berr=0.0, stats: tc_stats | None = None) -> None:
    _need(B, "float64", None, "B")
    _need(X, "float64", None, "X")
    _check(h, lib().tile_chol_solve(h, nrhs, _ptr(B), ldb, _ptr(X), ldx, max_refine, target_berr,
                                    ctypes.byref(stats) if stats is not None else None))


def tile_chol_logdet(h) -> float:
    out = ctypes.c_double()
    _check(h, lib().tile_chol_logdet(h, ctypes.byref(out)))
    return out.value


def tile_chol_loglik(h, y=None) -> float:
    out = ctypes.c_double()
    _need(y, "float64", None, "y")
    _check(h, lib().tile_chol_loglik(h, _ptr(y), ctypes.byref(out)))
    return out.value


def tile_chol_loglik_refined(h, y, max_refine=5, target_berr=1e-14):
    """Eq. 1 with y^T Sigma^{-1} y from a refined solve.  Returns (loglik, backward error)."""
    out, be = ctypes.c_double(), ctypes.c_double()
    _need(y, "float64", None, "y")
    _check(h, lib().tile_chol_loglik_refined(h, _ptr(y), max_refine, target_berr, ctypes.byref(out), ctypes.byref(be)))
    return out.value, be.value


def tile_chol_loglik_solved(h, y, x) -> float:
    """Eq. 1 with y^T Sigma^{-1} y = y^T x, x the solution of Sigma x = y from tile_chol_solve."""
    out = ctypes.c_double()
    _need(y, "float64", None, "y")
    _need(x, "float64", None, "x")
    _check(h, lib().tile_chol_loglik_solved(h, _ptr(y), _ptr(x), ctypes.byref(out)))
    return out.value


def tile_chol_get_factor(h, L_tiles) -> None:
    _need(L_tiles, "float64", None, "L_tiles")
    _check(h, lib().tile_chol_get_factor(h, _ptr(L_tiles)))


def tile_chol_get_factor_batched(h, index: int, L_tiles) -> None:
    _need(L_tiles, "float64", None, "L_tiles")
    _check(h, lib().tile_chol_get_factor_batched(h, index, _ptr(L_tiles)))


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))(*[_ptr(x) for x in items])
    return arr


def tile_chol_factor_batched(h, ns, b, A_list, maps=None, stats: tc_stats | None = None):
    """Factor every A_list[i] (order ns[i], tile b).  Returns (rc, info list, logdet list)."""
    count = len(ns)
    n_arr = (ctypes.c_int64 * count)(*ns)
    a_arr = _ptr_array(A_list)
    m_arr = _ptr_array(maps) if maps is not None else None
    info = (ctypes.c_int * count)()
    ld = (ctypes.c_double * count)()
    rc = lib().tile_chol_factor_batched(h, count, ctypes.cast(n_arr, ctypes.c_void_p), b,
                                        ctypes.cast(a_arr, ctypes.c_void_p),
                                        ctypes.cast(m_arr, ctypes.c_void_p) if m_arr is not None else None,
                                        ctypes.cast(info, ctypes.c_void_p), ctypes.cast(ld, ctypes.c_void_p),
                                        ctypes.byref(stats) if stats is not None else None)
    _check(h, rc, allow_positive=True)
    return rc, list(info), list(ld)


def tile_chol_solve_batched(h, nrhs, B_list, X_list, max_refine=0, target_berr=0.0,
                            stats: tc_stats | None = None):
    """Returns the per-matrix backward errors."""
    count = len(B_list)
    berr = (ctypes.c_double * count)()
    _check(h, lib().tile_chol_solve_batched(h, nrhs, ctypes.cast(_ptr_array(B_list), ctypes.c_void_p),
                                            ctypes.cast(_ptr_array(X_list), ctypes.c_void_p), max_refine,
                                            target_berr, ctypes.cast(berr, ctypes.c_void_p),
                                            ctypes.byref(stats) if stats is not None else None))
    return list(berr)


def tile_chol_loglik_batched(h, y_list, count=None):
    count = len(y_list) if y_list is not None else count
    out = (ctypes.c_double * count)()
    _check(h, lib().tile_chol_loglik_batched(
        h, ctypes.cast(_ptr_array(y_list), ctypes.c_void_p) if y_list is not None else None,
        ctypes.cast(out, ctypes.c_void_p)))
    return list(out)


def tile_chol_precision_map_noalloc(n, b, A_tiles, eps_high, band, prec_set, map_out, stream=None) -> None:
    """Precision map into a caller-owned device buffer without any allocation (see the header)."""
    _need_tiles(n, b, A_tiles, map_out)
    rc = lib().tile_chol_precision_map_noalloc(n, b, _ptr(A_tiles), eps_high, band, prec_set, _ptr(map_out),
                                               stream)
    if rc != TC_OK:
        why = ("arguments out of range (the allocation-free path takes at most 256 tiles per column)"
               if rc == -1 else "CUDA error")
        raise TileCholError(rc, f"tile_chol_precision_map_noalloc: {why}")


class Handle:
    """Context manager owning one tc_handle."""

    def __init__(self, device: int = 0, stream: int | None = None, **cfg_fields):
        cfg = tc_config_default()
        cfg.device = device
        if stream is not None:
            cfg.stream = stream
        for k, v in cfg_fields.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.h = tc_create(cfg)

    def close(self) -> None:
        if self.h:
            tc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass
