"""Python binding of the C ABI in include/tpcamg.h (argument marshalling only).

Every step of the solver runs inside libtpcamg.so (host setup in C++, every solve step in
CUDA kernels for sm_103a). This module only loads the library, converts arguments and
passes device pointers (``torch.Tensor.data_ptr()``) and CUDA streams through. There is no
CPU fallback: if the library is missing, loading fails with an error.

Functions carry the C names (``tpc_setup``, ``tpc_solve``, ...); ``Solver`` is a small
convenience wrapper around a handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtpcamg.so")

TPC_OK, TPC_ENOTCONV = 0, 1
TPC_EINVAL, TPC_ENOMEM, TPC_ECUDA, TPC_ESINGULAR, TPC_ENOTSUP, TPC_EDIVERGED = -1, -2, -3, -4, -5, -6
TPC_ESYNC = -7
TPC_BATCH_AUTO, TPC_BATCH_COOPERATIVE, TPC_BATCH_THREE_PASS = 0, 1, 2
TPC_SPD, TPC_NONSYM, TPC_WEAKLY = 0, 1, 2
TPC_FP64, TPC_MIXED = 0, 1
TPC_TRANSFER_PAPER, TPC_TRANSFER_GEOMETRIC = 0, 1
TPC_OUTER_VCYCLE, TPC_OUTER_FGMRES = 0, 1

EXPORTED = ["tpc_default_params", "tpc_setup", "tpc_solve", "tpc_solve_batch", "tpc_solve_host",
            "tpc_batch_create", "tpc_batch_create_2d", "tpc_batch_solve",
            "tpc_tune_get", "tpc_tune_set", "tpc_tune_reset", "tpc_batch_groups", "tpc_batch_set_product_mode",
            "tpc_batch_grouped_instances", "tpc_batch_destroy", "tpc_grid_wait_selftest",
            "tpc_apply",
            "tpc_apply_f32",
            "tpc_vcycle", "tpc_level_size", "tpc_finest_level", "tpc_coarsest_level",
            "tpc_export_level", "tpc_host_hierarchy", "tpc_time_level_kernels",
            "tpc_time_level_kernels_f32", "tpc_kernel_launches", "tpc_last_solve_cycles",
            "tpc_residual", "tpc_uses_box_residual",
            "tpc_apply_noalloc",
            "tpc_bdf4_coefficients", "tpc_collocation_rhs", "tpc_bdf4_step",
            "tpc_host_dense_level",
            "tpc_destroy", "tpc_last_error",
            "tpc2d_setup", "tpc2d_solve", "tpc2d_apply", "tpc2d_apply_f32", "tpc2d_vcycle",
            "tpc2d_level_size", "tpc2d_finest_level", "tpc2d_coarsest_level",
            "tpc2d_last_solve_cycles", "tpc2d_kernel_launches", "tpc2d_last_error",
            "tpc2d_destroy",
            "tpc_server_default_config", "tpc_server_create", "tpc_server_submit",
            "tpc_server_poll", "tpc_server_outstanding", "tpc_server_get_stats",
            "tpc_server_destroy"]


class TpcParams(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("kernel", ctypes.c_int),
                ("kernel_a", ctypes.c_double), ("gamma0", ctypes.c_double),
                ("shift", ctypes.c_double), ("m1", ctypes.c_int), ("m2", ctypes.c_int),
                ("omega_pre", ctypes.c_double), ("omega_post", ctypes.c_double),
                ("coarsest_level", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("inner_cycles", ctypes.c_int),
                ("autotune", ctypes.c_int), ("poison", ctypes.c_int),
                ("transfer", ctypes.c_int), ("box_residual", ctypes.c_int),
                ("outer", ctypes.c_int)]


class TpcServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_handles_per_key", ctypes.c_int)]


class TpcRequest(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("delta", ctypes.c_double), ("h", ctypes.c_double),
                ("n", ctypes.c_longlong), ("b_host", ctypes.c_void_p), ("x_host", ctypes.c_void_p),
                ("tol", ctypes.c_double), ("kernel", ctypes.c_int), ("kernel_a", ctypes.c_double),
                ("dim", ctypes.c_int), ("transfer", ctypes.c_int), ("outer", ctypes.c_int)]


class TpcServerStats(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_longlong), ("setups", ctypes.c_longlong),
                ("evictions", ctypes.c_longlong), ("elapsed_s", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("inflight_s", ctypes.c_double),
                ("max_inflight_seen", ctypes.c_int), ("resident_bytes", ctypes.c_size_t)]


class TpcServerResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_longlong), ("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("relres", ctypes.c_double), ("latency_s", ctypes.c_double),
                ("queue_s", ctypes.c_double)]


class TpcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tpcamg error {code}: {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load the in-tree library (built by ``__graft_entry__.build()``); raise if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2202_11288_gb300._build")
    L = ctypes.CDLL(LIB_PATH)
    P, D, I, LL, SZ = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_longlong, ctypes.c_size_t
    pp = ctypes.POINTER(TpcParams)
    L.tpc_default_params.argtypes = [pp]
    L.tpc_default_params.restype = None
    L.tpc_setup.argtypes = [pp, D, D, I, P, ctypes.POINTER(P)]
    L.tpc_setup.restype = I
    L.tpc_solve.argtypes = [P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    L.tpc_solve.restype = I
    L.tpc_solve_batch.argtypes = [P, I, P, P, D, P, P, P]
    L.tpc_solve_batch.restype = I
    L.tpc_tune_get.argtypes = [I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]
    L.tpc_tune_get.restype = I
    L.tpc_tune_set.argtypes = [I, I, I, I, I]
    L.tpc_tune_set.restype = I
    L.tpc_tune_reset.argtypes = []
    L.tpc_tune_reset.restype = None
    L.tpc_batch_create.argtypes = [P, I, ctypes.POINTER(P)]
    L.tpc_batch_create.restype = I
    L.tpc_batch_create_2d.argtypes = [P, I, P, I, ctypes.POINTER(P)]
    L.tpc_batch_create_2d.restype = I
    L.tpc_batch_solve.argtypes = [P, P, P, D, P, P, P]
    L.tpc_batch_solve.restype = I
    L.tpc_batch_set_product_mode.argtypes = [P, I]
    L.tpc_batch_set_product_mode.restype = I
    L.tpc_batch_groups.argtypes = [P]
    L.tpc_batch_groups.restype = I
    L.tpc_batch_grouped_instances.argtypes = [P]
    L.tpc_batch_grouped_instances.restype = I
    L.tpc_batch_destroy.argtypes = [P]
    L.tpc_batch_destroy.restype = None
    L.tpc_grid_wait_selftest.argtypes = [ctypes.c_uint, ctypes.POINTER(I), ctypes.POINTER(I)]
    L.tpc_grid_wait_selftest.restype = I
    L.tpc_solve_host.argtypes = [P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    L.tpc_solve_host.restype = I
    L.tpc_apply.argtypes = [P, I, P, P]
    L.tpc_apply.restype = I
    L.tpc_apply_f32.argtypes = [P, I, P, P]
    L.tpc_apply_f32.restype = I
    L.tpc_vcycle.argtypes = [P, P, P]
    L.tpc_vcycle.restype = I
    L.tpc_level_size.argtypes = [P, I]
    L.tpc_level_size.restype = LL
    L.tpc_finest_level.argtypes = [P]
    L.tpc_finest_level.restype = I
    L.tpc_coarsest_level.argtypes = [P]
    L.tpc_coarsest_level.restype = I
    L.tpc_export_level.argtypes = [P, I, P, SZ, ctypes.POINTER(SZ)]
    L.tpc_export_level.restype = I
    L.tpc_host_hierarchy.argtypes = [pp, D, D, I, P, SZ, ctypes.POINTER(SZ)]
    L.tpc_host_hierarchy.restype = I
    L.tpc_host_dense_level.argtypes = [pp, D, D, I, I, P, SZ, ctypes.POINTER(SZ)]
    L.tpc_host_dense_level.restype = I
    L.tpc_bdf4_coefficients.argtypes = [pp, D, D, D, ctypes.POINTER(D), ctypes.POINTER(D)]
    L.tpc_bdf4_coefficients.restype = I
    L.tpc_collocation_rhs.argtypes = [pp, D, D, P, P, P, P]
    L.tpc_collocation_rhs.restype = I
    L.tpc_bdf4_step.argtypes = [P, P, P, P, P, D, P, D, D, P, ctypes.POINTER(I), ctypes.POINTER(D)]
    L.tpc_bdf4_step.restype = I
    L.tpc_time_level_kernels.argtypes = [P, I, I, P, P, P, ctypes.POINTER(D)]
    L.tpc_time_level_kernels.restype = I
    L.tpc_time_level_kernels_f32.argtypes = [P, I, I, P, P, P, ctypes.POINTER(D)]
    L.tpc_time_level_kernels_f32.restype = I
    L.tpc_kernel_launches.argtypes = [P]
    L.tpc_kernel_launches.restype = LL
    L.tpc_last_solve_cycles.argtypes = [P]
    L.tpc_last_solve_cycles.restype = I
    L.tpc_residual.argtypes = [P, P, P, P]
    L.tpc_residual.restype = I
    L.tpc_uses_box_residual.argtypes = [P]
    L.tpc_uses_box_residual.restype = I
    L.tpc_apply_noalloc.argtypes = [LL, P, P, P, P, P, P, P, P, D, P, P, P]
    L.tpc_apply_noalloc.restype = I
    L.tpc_server_default_config.argtypes = [ctypes.POINTER(TpcServerConfig)]
    L.tpc_server_default_config.restype = None
    L.tpc_server_create.argtypes = [ctypes.POINTER(TpcServerConfig), pp, ctypes.POINTER(P)]
    L.tpc_server_create.restype = I
    L.tpc_server_submit.argtypes = [P, ctypes.POINTER(TpcRequest), ctypes.POINTER(LL)]
    L.tpc_server_submit.restype = I
    L.tpc_server_poll.argtypes = [P, ctypes.POINTER(TpcServerResult), I, I]
    L.tpc_server_poll.restype = I
    L.tpc_server_outstanding.argtypes = [P]
    L.tpc_server_outstanding.restype = LL
    L.tpc_server_get_stats.argtypes = [P, ctypes.POINTER(TpcServerStats), I]
    L.tpc_server_get_stats.restype = I
    L.tpc_server_destroy.argtypes = [P]
    L.tpc_server_destroy.restype = None
    L.tpc_destroy.argtypes = [P]
    L.tpc_destroy.restype = None
    L.tpc2d_setup.argtypes = [pp, D, D, P, ctypes.POINTER(P)]
    L.tpc2d_setup.restype = I
    L.tpc2d_solve.argtypes = [P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    L.tpc2d_solve.restype = I
    for nm in ("tpc2d_apply", "tpc2d_apply_f32"):
        getattr(L, nm).argtypes = [P, I, P, P]
        getattr(L, nm).restype = I
    L.tpc2d_vcycle.argtypes = [P, P, P]
    L.tpc2d_vcycle.restype = I
    L.tpc2d_level_size.argtypes = [P, I]
    L.tpc2d_level_size.restype = LL
    for nm in ("tpc2d_finest_level", "tpc2d_coarsest_level", "tpc2d_last_solve_cycles"):
        getattr(L, nm).argtypes = [P]
        getattr(L, nm).restype = I
    L.tpc2d_kernel_launches.argtypes = [P]
    L.tpc2d_kernel_launches.restype = LL
    L.tpc2d_last_error.argtypes = [P]
    L.tpc2d_last_error.restype = ctypes.c_char_p
    L.tpc2d_destroy.argtypes = [P]
    L.tpc2d_destroy.restype = None
    L.tpc_last_error.argtypes = [P]
    L.tpc_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def tpc_default_params(**overrides) -> TpcParams:
    p = TpcParams()
    lib().tpc_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def tpc_last_error(handle=None) -> str:
    msg = lib().tpc_last_error(handle)
    return msg.decode() if msg else ""


def _check(rc: int, handle=None, allow=(TPC_OK,)) -> int:
    if rc not in allow:
        raise TpcError(rc, tpc_last_error(handle))
    return rc


def _split_levels(buf: np.ndarray) -> list:
    levels, o = [], 0
    while o < buf.size:
        N = int(buf[o])
        G = 2 * N - 1
        d = {"N": N, "o": float(buf[o + 1])}
        o += 2
        for key in ("A", "B", "C", "D"):
            d[key] = buf[o:o + G].copy()
            o += G
        for key in ("p", "q", "xi", "zeta"):
            d[key] = buf[o:o + N].copy()
            o += N
        levels.append(d)
    return levels


def tpc_host_hierarchy(delta: float, h: float, levels: int = 0, params: TpcParams | None = None):
    """Host-only hierarchy (no GPU): list of levels, finest first, in the export layout."""
    p = params if params is not None else tpc_default_params()
    need = ctypes.c_size_t(0)
    _check(lib().tpc_host_hierarchy(ctypes.byref(p), delta, h, levels, None, 0, ctypes.byref(need)))
    buf = np.empty(need.value, dtype=np.float64)
    _check(lib().tpc_host_hierarchy(ctypes.byref(p), delta, h, levels,
                                    buf.ctypes.data_as(ctypes.c_void_p), need.value,
                                    ctypes.byref(need)))
    return _split_levels(buf)


def _ptr(t):
    if t is None:
        return None  # NULL
    return t.data_ptr() if hasattr(t, "data_ptr") else int(t)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def tpc_setup(delta: float, h: float, levels: int = 0, params: TpcParams | None = None,
              stream=None) -> ctypes.c_void_p:
    p = params if params is not None else tpc_default_params()
    H = ctypes.c_void_p()
    _check(lib().tpc_setup(ctypes.byref(p), delta, h, levels, _stream_handle(stream),
                           ctypes.byref(H)))
    return H


def tpc_solve(H, b, x, tol: float = 1e-10, use_x0: bool = False):
    it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
    rc = _check(lib().tpc_solve(H, _ptr(b), _ptr(x), tol, int(use_x0), ctypes.byref(it),
                                ctypes.byref(rel)), H, allow=(TPC_OK, TPC_ENOTCONV))
    return rc, it.value, rel.value


def tpc_host_dense_level(delta: float, h: float, level: int, levels: int = 0,
                         params: TpcParams | None = None) -> np.ndarray:
    """Dense matrix of one level of the host hierarchy (small levels only; no GPU)."""
    p = params if params is not None else tpc_default_params()
    need = ctypes.c_size_t(0)
    _check(lib().tpc_host_dense_level(ctypes.byref(p), delta, h, levels, level, None, 0,
                                      ctypes.byref(need)))
    out = np.empty(need.value, dtype=np.float64)
    _check(lib().tpc_host_dense_level(ctypes.byref(p), delta, h, levels, level,
                                      out.ctypes.data_as(ctypes.c_void_p), need.value,
                                      ctypes.byref(need)))
    n = int(round(need.value ** 0.5))
    return out.reshape(n, n)


def tpc_bdf4_coefficients(delta: float, h: float, tau: float, params: TpcParams | None = None):
    """(sigma, eta_h / tau) of one BDF4 step of size tau (host only)."""
    p = params if params is not None else tpc_default_params()
    sh, hs = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().tpc_bdf4_coefficients(ctypes.byref(p), delta, h, tau, ctypes.byref(sh),
                                       ctypes.byref(hs)))
    return sh.value, hs.value


def tpc_collocation_rhs(delta: float, h: float, f_colloc=None, g_left=None, g_right=None,
                        params: TpcParams | None = None) -> np.ndarray:
    """eta_h f - (exterior couplings of g) at the collocation points (host arrays; None = 0)."""
    p = params if params is not None else tpc_default_params()
    n = int(round(2.0 / h)) - 1
    fa, gl, gr = (None if a is None else np.ascontiguousarray(a, dtype=np.float64)
                  for a in (f_colloc, g_left, g_right))
    out = np.empty(n, dtype=np.float64)

    def ptr(a):
        return None if a is None else a.ctypes.data_as(ctypes.c_void_p)

    _check(lib().tpc_collocation_rhs(ctypes.byref(p), delta, h, ptr(fa), ptr(gl), ptr(gr),
                                     ptr(out)))
    return out


def tpc_bdf4_step(H, u1, u2, u3, u4, hist_scale: float, g, g_scale: float, tol: float, out):
    it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
    rc = _check(lib().tpc_bdf4_step(H, _ptr(u1), _ptr(u2), _ptr(u3), _ptr(u4), hist_scale,
                                    _ptr(g) if g is not None else None, g_scale, tol, _ptr(out),
                                    ctypes.byref(it), ctypes.byref(rel)), H,
                allow=(TPC_OK, TPC_ENOTCONV))
    return rc, it.value, rel.value


def tpc_solve_batch(handles, bs, xs, tol: float = 1e-10):
    """Solve len(handles) independent systems concurrently; returns (rc, iters, relres, status)
    lists. handles: tpc handles (distinct); bs, xs: device tensors (or pointers)."""
    n = len(handles)
    HA = (ctypes.c_void_p * n)(*[h.value if hasattr(h, "value") else h for h in handles])
    BA = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
    XA = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    it = (ctypes.c_int * n)()
    rel = (ctypes.c_double * n)()
    stt = (ctypes.c_int * n)()
    rc = lib().tpc_solve_batch(HA, n, BA, XA, tol, it, rel, stt)
    if rc < 0 and rc not in (TPC_EDIVERGED,):
        raise TpcError(rc, tpc_last_error(None))
    return rc, list(it), list(rel), list(stt)


class Batch:
    """Stage-batched solves over a fixed list of handles (tpc_batch_*): ``Batch(handles)`` then
    ``solve(bs, xs)``; groups instances of identical level structure into one launch per stage.
    ``handles2d`` (2-D handles) are further instances, solved beside the groups; their vectors
    follow the 1-D ones in ``bs`` and ``xs``."""

    def __init__(self, handles, handles2d=()):
        n, n2 = len(handles), len(handles2d)
        self._n = n + n2
        val = lambda h: h.value if hasattr(h, "value") else h
        HA = (ctypes.c_void_p * max(n, 1))(*[val(h) for h in handles])
        HB = (ctypes.c_void_p * max(n2, 1))(*[val(h) for h in handles2d])
        self.handle = ctypes.c_void_p()
        _check(lib().tpc_batch_create_2d(HA, n, HB, n2, ctypes.byref(self.handle)))

    def solve(self, bs, xs, tol: float = 1e-10):
        n = self._n
        BA = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
        XA = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
        it = (ctypes.c_int * n)()
        rel = (ctypes.c_double * n)()
        stt = (ctypes.c_int * n)()
        rc = lib().tpc_batch_solve(self.handle, BA, XA, tol, it, rel, stt)
        if rc < 0 and rc not in (TPC_EDIVERGED,):
            raise TpcError(rc, tpc_last_error(None))
        return rc, list(it), list(rel), list(stt)

    def set_product_mode(self, mode: int) -> None:
        _check(lib().tpc_batch_set_product_mode(self.handle, int(mode)))

    def groups(self) -> int:
        return int(lib().tpc_batch_groups(self.handle))

    def grouped_instances(self) -> int:
        return int(lib().tpc_batch_grouped_instances(self.handle))

    def close(self) -> None:
        if self.handle:
            lib().tpc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def tpc_tune_get(word: int, logm: int):
    """(logL, logC, reg) of the process-wide FFT plan table for levels of size 2^logm in FP32
    (word 4) or FP64 (word 8), or None when there is no entry."""
    a, c, r = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    rc = lib().tpc_tune_get(word, logm, ctypes.byref(a), ctypes.byref(c), ctypes.byref(r))
    if rc < 0:
        raise TpcError(rc, tpc_last_error(None))
    return (a.value, c.value, r.value) if rc == 1 else None


def tpc_tune_set(word: int, logm: int, logL: int, logC: int, reg: int = 0) -> None:
    _check(lib().tpc_tune_set(word, logm, logL, logC, reg))


def tpc_tune_reset() -> None:
    lib().tpc_tune_reset()


def tpc_grid_wait_selftest(max_polls: int):
    """(gave_up, passed) of a grid barrier nothing can reach, waited with max_polls polls."""
    g, p = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().tpc_grid_wait_selftest(int(max_polls), ctypes.byref(g), ctypes.byref(p)))
    return g.value, p.value


def tpc_solve_host(H, b: np.ndarray, x: np.ndarray, tol: float = 1e-10, use_x0: bool = False):
    assert b.dtype == np.float64 and x.dtype == np.float64
    assert b.flags.c_contiguous and x.flags.c_contiguous
    it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
    rc = _check(lib().tpc_solve_host(H, b.ctypes.data_as(ctypes.c_void_p),
                                     x.ctypes.data_as(ctypes.c_void_p), tol, int(use_x0),
                                     ctypes.byref(it), ctypes.byref(rel)), H,
                allow=(TPC_OK, TPC_ENOTCONV))
    return rc, it.value, rel.value


def tpc_apply(H, level: int, x, y) -> None:
    _check(lib().tpc_apply(H, level, _ptr(x), _ptr(y)), H)


def tpc_apply_f32(H, level: int, x, y) -> None:
    _check(lib().tpc_apply_f32(H, level, _ptr(x), _ptr(y)), H)


def tpc_vcycle(H, r, e) -> None:
    _check(lib().tpc_vcycle(H, _ptr(r), _ptr(e)), H)


def tpc_level_size(H, level: int) -> int:
    return int(lib().tpc_level_size(H, level))


def tpc_finest_level(H) -> int:
    return int(lib().tpc_finest_level(H))


def tpc_coarsest_level(H) -> int:
    return int(lib().tpc_coarsest_level(H))


def tpc_export_level(H, level: int) -> dict:
    need = ctypes.c_size_t(0)
    _check(lib().tpc_export_level(H, level, None, 0, ctypes.byref(need)), H)
    buf = np.empty(need.value, dtype=np.float64)
    _check(lib().tpc_export_level(H, level, buf.ctypes.data_as(ctypes.c_void_p), need.value,
                                  ctypes.byref(need)), H)
    return _split_levels(buf)[0]


def tpc_time_level_kernels(H, level: int, reps: int, x, f, y):
    """Average ms per launch of [forward strided, contiguous-block, inverse strided] kernels."""
    out = (ctypes.c_double * 3)()
    _check(lib().tpc_time_level_kernels(H, level, reps, _ptr(x), _ptr(f), _ptr(y), out), H)
    return [out[0], out[1], out[2]]


def tpc_time_level_kernels_f32(H, level: int, reps: int, x, f, y):
    """The same for the FP32 level copy of a mixed handle (float32 device tensors)."""
    out = (ctypes.c_double * 3)()
    _check(lib().tpc_time_level_kernels_f32(H, level, reps, _ptr(x), _ptr(f), _ptr(y), out), H)
    return [out[0], out[1], out[2]]


def tpc_kernel_launches(H) -> int:
    return int(lib().tpc_kernel_launches(H))


def tpc_residual(H, x, b, r) -> None:
    _check(lib().tpc_residual(H, _ptr(x), _ptr(b), _ptr(r)), H)


def tpc_uses_box_residual(H) -> int:
    return int(lib().tpc_uses_box_residual(H))


def tpc_last_solve_cycles(H) -> int:
    return int(lib().tpc_last_solve_cycles(H))


def tpc_apply_noalloc(N: int, tA, tB, tC, tD, p, q, xi, zeta, o: float, x, y,
                      stream=None) -> None:
    """y = A x for one level from device generators and Cross vectors, with no device
    allocation (for callers that cannot allocate; see include/tpcamg.h for the limits)."""
    _check(lib().tpc_apply_noalloc(N, _ptr(tA), _ptr(tB), _ptr(tC), _ptr(tD), _ptr(p), _ptr(q),
                                   _ptr(xi), _ptr(zeta), float(o), _ptr(x), _ptr(y),
                                   _stream_handle(stream)))


def tpc_destroy(H) -> None:
    if H:
        lib().tpc_destroy(H)


class Solver:
    """Owns one handle: ``Solver(delta, h, variant=TPC_SPD, ...)`` then ``solve(b, x)``."""

    def __init__(self, delta: float, h: float, levels: int = 0, stream=None, **params):
        self.params = tpc_default_params(**params)
        self.handle = tpc_setup(delta, h, levels, self.params, stream)
        self.K = tpc_finest_level(self.handle)
        self.kc = tpc_coarsest_level(self.handle)
        self.n = tpc_level_size(self.handle, self.K)

    def solve(self, b, x, tol: float = 1e-10, use_x0: bool = False):
        return tpc_solve(self.handle, b, x, tol, use_x0)

    def solve_host(self, b: np.ndarray, x: np.ndarray, tol: float = 1e-10, use_x0: bool = False):
        return tpc_solve_host(self.handle, b, x, tol, use_x0)

    def bdf4_step(self, u1, u2, u3, u4, hist_scale: float, g, g_scale: float, out,
                  tol: float = 1e-12):
        """One step of eq. (5.1) (the handle's shift must be sigma, tpc_bdf4_coefficients)."""
        return tpc_bdf4_step(self.handle, u1, u2, u3, u4, hist_scale, g, g_scale, tol, out)

    def apply(self, level: int, x, y) -> None:
        tpc_apply(self.handle, level, x, y)

    def apply_f32(self, level: int, x, y) -> None:
        tpc_apply_f32(self.handle, level, x, y)

    def vcycle(self, r, e) -> None:
        tpc_vcycle(self.handle, r, e)

    def residual(self, x, b, r) -> None:
        tpc_residual(self.handle, x, b, r)

    def level_size(self, level: int) -> int:
        return tpc_level_size(self.handle, level)

    def export_level(self, level: int) -> dict:
        return tpc_export_level(self.handle, level)

    def close(self) -> None:
        if self.handle:
            tpc_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Solver2D:
    """Owns one 2-D handle (tpc2d_*): ``Solver2D(delta, h, variant=TPC_SPD, ...)`` then
    ``solve(b, x)`` with b, x device tensors of n^2 doubles (row-major U[i][j])."""

    def __init__(self, delta: float, h: float, stream=None, **params):
        self.params = tpc_default_params(**params)
        H = ctypes.c_void_p()
        _check(lib().tpc2d_setup(ctypes.byref(self.params), delta, h, _stream_handle(stream),
                                 ctypes.byref(H)))
        self.handle = H
        self.K = int(lib().tpc2d_finest_level(H))
        self.kc = int(lib().tpc2d_coarsest_level(H))
        self.nn = int(lib().tpc2d_level_size(H, self.K))
        self.n = int(round(self.nn ** 0.5))

    def _check(self, rc, allow=(TPC_OK,)):
        if rc not in allow:
            msg = lib().tpc2d_last_error(self.handle)
            raise TpcError(rc, msg.decode() if msg else "")
        return rc

    def solve(self, b, x, tol: float = 1e-10, use_x0: bool = False):
        it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
        rc = self._check(lib().tpc2d_solve(self.handle, _ptr(b), _ptr(x), tol, int(use_x0),
                                           ctypes.byref(it), ctypes.byref(rel)),
                         allow=(TPC_OK, TPC_ENOTCONV))
        return rc, it.value, rel.value

    def apply(self, level: int, x, y) -> None:
        self._check(lib().tpc2d_apply(self.handle, level, _ptr(x), _ptr(y)))

    def apply_f32(self, level: int, x, y) -> None:
        self._check(lib().tpc2d_apply_f32(self.handle, level, _ptr(x), _ptr(y)))

    def vcycle(self, r, e) -> None:
        self._check(lib().tpc2d_vcycle(self.handle, _ptr(r), _ptr(e)))

    def level_size(self, level: int) -> int:
        return int(lib().tpc2d_level_size(self.handle, level))

    def last_cycles(self) -> int:
        return int(lib().tpc2d_last_solve_cycles(self.handle))

    def close(self) -> None:
        if self.handle:
            lib().tpc2d_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request server (continuous batching): ``submit`` queues a solve on host buffers,
    ``poll`` returns finished results. Buffers must stay alive until their result is polled."""

    def __init__(self, hbm_budget_bytes: int | None = None, max_inflight: int | None = None,
                 precision: int = TPC_MIXED, max_handles_per_key: int | None = None, **params):
        cfg = TpcServerConfig()
        lib().tpc_server_default_config(ctypes.byref(cfg))
        if hbm_budget_bytes is not None:
            cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        if max_inflight is not None:
            cfg.max_inflight = int(max_inflight)
        if max_handles_per_key is not None:
            cfg.max_handles_per_key = int(max_handles_per_key)
        cfg.precision = precision
        p = tpc_default_params(**params)
        self.handle = ctypes.c_void_p()
        _check(lib().tpc_server_create(ctypes.byref(cfg), ctypes.byref(p), ctypes.byref(self.handle)))
        self._keep = {}

    def submit(self, variant: int, delta: float, h: float, b, x, tol: float = 1e-10,
               kernel: int = 0, kernel_a: float = 0.0, dim: int = 1,
               transfer: int | None = None, outer: int | None = None) -> int:
        """b, x: contiguous float64 host arrays (numpy, or pinned torch CPU tensors); dim 2 for
        the 2-D system ((2/h - 1)^2 unknowns); transfer: TPC_TRANSFER_PAPER or
        TPC_TRANSFER_GEOMETRIC, outer: TPC_OUTER_VCYCLE or TPC_OUTER_FGMRES, None for the
        server's parameters' choice."""
        n = b.numel() if hasattr(b, "numel") else b.size
        bp = b.data_ptr() if hasattr(b, "data_ptr") else b.ctypes.data
        xp = x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
        rt = 0 if transfer is None else 1 + int(transfer)   # TPC_REQUEST_TRANSFER_*
        ro = 0 if outer is None else 1 + int(outer)         # TPC_REQUEST_OUTER_*
        r = TpcRequest(variant, delta, h, n, bp, xp, tol, kernel, kernel_a, dim, rt, ro)
        t = ctypes.c_longlong(0)
        _check(lib().tpc_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = (b, x)
        return t.value

    def poll(self, cap: int = 256, wait_ms: int = 0) -> list:
        out = (TpcServerResult * cap)()
        k = lib().tpc_server_poll(self.handle, out, cap, wait_ms)
        res = []
        for i in range(max(k, 0)):
            r = out[i]
            self._keep.pop(r.ticket, None)
            res.append({"ticket": r.ticket, "status": r.status, "iters": r.iters,
                        "relres": r.relres, "latency_s": r.latency_s, "queue_s": r.queue_s})
        return res

    def outstanding(self) -> int:
        return int(lib().tpc_server_outstanding(self.handle))

    def stats(self, reset: bool = False) -> dict:
        st = TpcServerStats()
        _check(lib().tpc_server_get_stats(self.handle, ctypes.byref(st), int(reset)))
        return {f: getattr(st, f) for f, _ in TpcServerStats._fields_}

    def close(self) -> None:
        if self.handle:
            lib().tpc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
