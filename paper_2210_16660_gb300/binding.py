"""Python binding of libpcgamg: argument marshalling only.

Every step of setup and solve runs in the CUDA library through its C ABI
(``include/pcgamg.h``); this module converts numpy arrays / torch tensors to
pointers, passes torch's current CUDA stream, and can route the library's
device allocations through torch's caching allocator. If the library cannot
be loaded the import of this module raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_OOM, ERR_BREAKDOWN, ERR_NOCONV, ERR_NAN, ERR_CUDA, ERR_TIMEOUT, ERR_COARSE, ERR_BUSY, ERR_MATCH = range(11)
MODE_PCG64, MODE_FCG32 = 0, 1
_MODES = {"pcg64": MODE_PCG64, "fcg32": MODE_FCG32}
COARSE_AUTO, COARSE_DENSE, COARSE_ITER = 0, 1, 2
_COARSE = {"auto": COARSE_AUTO, "dense": COARSE_DENSE, "iter": COARSE_ITER}

# Every symbol the header declares (checked by the CPU tests).
EXPORTS = ("amg_default_params", "amg_set_allocator", "amg_setup", "amg_set_mode", "pcg_solve",
           "amg_last_true_residual", "amg_info", "amg_level_agg", "amg_level_csr", "amg_setup_times",
           "amg_destroy", "amg_last_error", "amg_profile", "amg_profile_read", "amg_launch_count",
           "amg_level_layout", "amg_level_pattern", "amg_residual_noalloc", "pcg_solve_multi", "amg_multi_info",
           "amg_batch_create", "pcg_solve_batch", "amg_batch_destroy", "amg_server_default_params",
           "amg_serve_plan", "amg_server_create", "amg_server_mesh_info", "amg_server_info", "amg_server_submit",
           "amg_server_progress", "amg_server_result", "amg_server_destroy", "amg_autotune", "amg_level_shape",
           "amg_set_level_shape", "amg_profile_levels", "amg_refresh", "amg_refresh_time", "amg_set_smoother",
           "amg_coarse_info", "amg_coarse_factors", "amg_coarse_solve", "amg_level_prolongator")


class AmgCsr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int)]


class AmgParams(C.Structure):
    _fields_ = [("coarse_max", C.c_int), ("n_pass", C.c_int), ("max_levels", C.c_int), ("mode", C.c_int),
                ("hbm_budget", C.c_size_t), ("coarse_solver", C.c_int), ("coarse_maxit", C.c_int),
                ("coarse_tol", C.c_double), ("smoothed", C.c_int)]


class ServerParams(C.Structure):
    _fields_ = [("mode", C.c_int), ("slots", C.c_int), ("max_engines", C.c_int), ("chunk", C.c_int),
                ("queue_cap", C.c_int), ("maxit", C.c_int), ("rtol", C.c_double), ("hbm_budget", C.c_size_t),
                ("solo", C.c_int), ("batch_min", C.c_int), ("lane_priority", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

_lib = None


def load(build_if_missing: bool = True):
    """Load libpcgamg.so (building it with nvcc when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libpcgamg not built: {path}")
    lib = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    lib.amg_default_params.argtypes = [C.POINTER(AmgParams)]
    lib.amg_default_params.restype = None
    lib.amg_set_allocator.argtypes = [P, P, P]
    lib.amg_set_allocator.restype = I
    lib.amg_setup.argtypes = [C.POINTER(AmgCsr), C.POINTER(AmgParams), P, C.POINTER(P)]
    lib.amg_setup.restype = I
    lib.amg_set_mode.argtypes = [P, I]
    lib.amg_set_mode.restype = I
    lib.pcg_solve.argtypes = [P, P, P, D, I, C.POINTER(I), P, P]
    lib.pcg_solve.restype = I
    lib.amg_last_true_residual.argtypes = [P]
    lib.amg_last_true_residual.restype = D
    lib.amg_info.argtypes = [P, C.POINTER(I), P, P]
    lib.amg_info.restype = I
    lib.amg_level_agg.argtypes = [P, I, I, P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.amg_level_agg.restype = I
    lib.amg_level_layout.argtypes = [P, I, C.POINTER(I), C.POINTER(C.c_int64), C.POINTER(I)]
    lib.amg_level_layout.restype = I
    lib.amg_level_pattern.argtypes = [P, I, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.amg_level_pattern.restype = I
    lib.amg_level_csr.argtypes = [P, I, P, P, P]
    lib.amg_level_csr.restype = I
    lib.amg_setup_times.argtypes = [P, P]
    lib.amg_setup_times.restype = I
    lib.amg_refresh.argtypes = [P, C.POINTER(AmgCsr), P]
    lib.amg_refresh.restype = I
    lib.amg_refresh_time.argtypes = [P, C.POINTER(C.c_double)]
    lib.amg_refresh_time.restype = I
    lib.amg_set_smoother.argtypes = [P, I, I, P]
    lib.amg_set_smoother.restype = I
    lib.amg_level_prolongator.argtypes = [P, I, C.POINTER(C.c_int64), P, P, P]
    lib.amg_level_prolongator.restype = I
    lib.amg_coarse_info.argtypes = [P, C.POINTER(I), C.POINTER(I), C.POINTER(I)]
    lib.amg_coarse_info.restype = I
    lib.amg_coarse_factors.argtypes = [P, P]
    lib.amg_coarse_factors.restype = I
    lib.amg_coarse_solve.argtypes = [P, P, P, C.POINTER(I), P]
    lib.amg_coarse_solve.restype = I
    lib.amg_profile.argtypes = [P, I]
    lib.amg_profile.restype = I
    lib.amg_profile_read.argtypes = [P, P, P, I]
    lib.amg_profile_read.restype = I
    lib.amg_launch_count.argtypes = [P]
    lib.amg_launch_count.restype = C.c_int64
    lib.amg_residual_noalloc.argtypes = [P, P, P, P, P, P]
    lib.amg_residual_noalloc.restype = I
    lib.pcg_solve_multi.argtypes = [P, I, P, P, D, I, P, P, P]
    lib.pcg_solve_multi.restype = I
    lib.amg_multi_info.argtypes = [P, C.POINTER(I), P, P]
    lib.amg_multi_info.restype = I
    lib.amg_batch_create.argtypes = [I, P, C.POINTER(P)]
    lib.amg_batch_create.restype = I
    lib.pcg_solve_batch.argtypes = [P, P, P, D, I, P, P, P]
    lib.pcg_solve_batch.restype = I
    lib.amg_batch_destroy.argtypes = [P]
    lib.amg_batch_destroy.restype = None
    SZ, I64 = C.c_size_t, C.c_int64
    lib.amg_server_default_params.argtypes = [C.POINTER(ServerParams)]
    lib.amg_server_default_params.restype = None
    lib.amg_serve_plan.argtypes = [I, P, P, P, SZ, I, P, C.POINTER(SZ)]
    lib.amg_serve_plan.restype = I
    lib.amg_server_create.argtypes = [C.POINTER(ServerParams), I, P, P, C.POINTER(P)]
    lib.amg_server_create.restype = I
    lib.amg_server_mesh_info.argtypes = [P, I, C.POINTER(I), C.POINTER(I), C.POINTER(SZ), C.POINTER(SZ)]
    lib.amg_server_mesh_info.restype = I
    lib.amg_server_info.argtypes = [P, C.POINTER(SZ), C.POINTER(SZ), C.POINTER(I), C.POINTER(I), C.POINTER(I64)]
    lib.amg_server_info.restype = I
    lib.amg_server_submit.argtypes = [P, I, P, P, P, C.POINTER(I64)]
    lib.amg_server_submit.restype = I
    lib.amg_server_progress.argtypes = [P, I, C.POINTER(I)]
    lib.amg_server_progress.restype = I
    lib.amg_server_result.argtypes = [P, I64, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(D), C.POINTER(I),
                                      P]
    lib.amg_server_result.restype = I
    lib.amg_server_destroy.argtypes = [P]
    lib.amg_server_destroy.restype = None
    lib.amg_autotune.argtypes = [P, I, C.POINTER(I), P]
    lib.amg_autotune.restype = I
    lib.amg_level_shape.argtypes = [P, I, P]
    lib.amg_level_shape.restype = I
    lib.amg_set_level_shape.argtypes = [P, I, P]
    lib.amg_set_level_shape.restype = I
    lib.amg_profile_levels.argtypes = [P, I, P, P]
    lib.amg_profile_levels.restype = I
    lib.amg_destroy.argtypes = [P]
    lib.amg_destroy.restype = None
    lib.amg_last_error.argtypes = []
    lib.amg_last_error.restype = C.c_char_p
    _lib = lib
    return lib


class AmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def last_error() -> str:
    return load().amg_last_error().decode()


# ------------------------------------------------------------ torch glue
_torch_alloc_refs = None


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_alloc_refs
    lib = load()
    if not enable:
        lib.amg_set_allocator(None, None, None)
        _torch_alloc_refs = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    refs = (ALLOC_FN(_alloc), FREE_FN(_free))
    st = lib.amg_set_allocator(C.cast(refs[0], C.c_void_p), C.cast(refs[1], C.c_void_p), None)
    if st:
        raise AmgError(st, last_error())
    _torch_alloc_refs = refs


def _current_device() -> int | None:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_device()
    except Exception:
        return None
    return None


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream or None
        except Exception:
            return None
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _ptr(a, dtype):
    """Pointer of a numpy array or torch tensor (contiguous, given dtype)."""
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected contiguous {dtype} array")
        return a.ctypes.data, False
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise TypeError("expected a contiguous tensor")
        return a.data_ptr(), a.is_cuda
    raise TypeError(f"unsupported array type {type(a)}")


@dataclasses.dataclass
class SolveResult:
    status: int
    iters: int
    hist: np.ndarray
    true_rel: float
    message: str


class AMG:
    """A resident AMG hierarchy (``amg_setup``) and its solves (``pcg_solve``)."""

    def __init__(self, row_ptr, col, val, n: int | None = None, coarse_max: int = 200, n_pass: int = 2,
                 max_levels: int = 30, mode: str = "pcg64", hbm_budget: int = 0, stream=None,
                 coarse: str = "auto", coarse_maxit: int = 30, coarse_tol: float = 1e-3, smoothed: bool = False):
        lib = load()
        rp, rp_dev = _ptr(row_ptr, np.int32)
        ci, ci_dev = _ptr(col, np.int32)
        v, v_dev = _ptr(val, np.float64)
        if not (rp_dev == ci_dev == v_dev):
            raise TypeError("CSR arrays must all be host or all device")
        nrows = (len(row_ptr) - 1) if n is None else n
        nnz = len(col)
        csr = AmgCsr(nrows, nnz, rp, ci, v, int(rp_dev))
        prm = AmgParams()
        lib.amg_default_params(C.byref(prm))
        prm.coarse_max, prm.n_pass, prm.max_levels = coarse_max, n_pass, max_levels
        prm.mode, prm.hbm_budget = _MODES[mode], hbm_budget
        prm.coarse_solver, prm.coarse_maxit, prm.coarse_tol = _COARSE[coarse], coarse_maxit, coarse_tol
        prm.smoothed = int(bool(smoothed))
        h = C.c_void_p()
        st = lib.amg_setup(C.byref(csr), C.byref(prm), _stream_ptr(stream), C.byref(h))
        if st:
            raise AmgError(st, last_error())
        self._h = h
        self.n = nrows
        self.mode = mode
        self.device = _current_device()

    @classmethod
    def from_csr(cls, A, **kw):
        return cls(A.row_ptr, A.col, A.val, n=A.n, **kw)

    def close(self):
        if getattr(self, "_h", None):
            load().amg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mode(self, mode: str):
        st = load().amg_set_mode(self._h, _MODES[mode])
        if st:
            raise AmgError(st, last_error())
        self.mode = mode

    def solve(self, b, x, rtol: float = 1e-8, maxit: int = 1000, stream=None, hist: bool = True,
              check: bool = False) -> SolveResult:
        """``pcg_solve``: x (in: initial guess, out: solution) is updated in place."""
        lib = load()
        bp, _ = _ptr(b, np.float64)
        xp, _ = _ptr(x, np.float64)
        h = np.zeros(maxit + 1) if hist else None
        it = C.c_int(0)
        st = lib.pcg_solve(self._h, bp, xp, rtol, maxit, C.byref(it),
                           h.ctypes.data if hist else None, _stream_ptr(stream))
        msg = last_error() if st else ""
        if check and st:
            raise AmgError(st, msg)
        return SolveResult(st, it.value, h[: it.value + 1] if hist else None,
                           lib.amg_last_true_residual(self._h), msg)

    def solve_multi(self, B, X, rtol: float = 1e-8, maxit: int = 1000, stream=None, hist: bool = True):
        """``pcg_solve_multi``: B, X are (n, k) row-major; X is updated in place.

        Returns (status, iters[k], hist[k, maxit+1] or None, statuses[k], true_rel[k]).
        """
        lib = load()
        k = int(B.shape[1])
        bp, _ = _ptr(B, np.float64)
        xp, _ = _ptr(X, np.float64)
        it = np.zeros(k, np.int32)
        h = np.zeros((k, maxit + 1)) if hist else None
        st = lib.pcg_solve_multi(self._h, k, bp, xp, rtol, maxit, it.ctypes.data,
                                 h.ctypes.data if hist else None, _stream_ptr(stream))
        kk = C.c_int(0)
        sts = np.zeros(32, np.int32)
        tr = np.zeros(32)
        lib.amg_multi_info(self._h, C.byref(kk), sts.ctypes.data, tr.ctypes.data)
        return st, it, h, sts[:k].copy(), tr[:k].copy()

    def info(self):
        lib = load()
        L = C.c_int(0)
        lib.amg_info(self._h, C.byref(L), None, None)
        n = np.zeros(L.value, np.int64)
        z = np.zeros(L.value, np.int64)
        lib.amg_info(self._h, C.byref(L), n.ctypes.data, z.ctypes.data)
        return list(zip(n.tolist(), z.tolist()))

    def level_agg(self, level: int, ps: int = -1):
        lib = load()
        n, nc = C.c_int64(), C.c_int64()
        st = lib.amg_level_agg(self._h, level, ps, None, C.byref(n), C.byref(nc))
        if st:
            raise AmgError(st, last_error())
        a = np.empty(n.value, np.int32)
        st = lib.amg_level_agg(self._h, level, ps, a.ctypes.data, C.byref(n), C.byref(nc))
        if st:
            raise AmgError(st, last_error())
        return a, nc.value

    def level_layout(self, level: int) -> dict:
        sl, st, ib = C.c_int(), C.c_int64(), C.c_int()
        r = load().amg_level_layout(self._h, level, C.byref(sl), C.byref(st), C.byref(ib))
        if r:
            raise AmgError(r, last_error())
        return {"slice": sl.value, "stored": st.value, "index_bytes": ib.value}

    def level_pattern(self, level: int) -> dict:
        """Slices (and their stored entries) of a level kept with a shared
        offset pattern (level 0 of a structured mesh: nearly all)."""
        sl, en = C.c_int64(), C.c_int64()
        r = load().amg_level_pattern(self._h, level, C.byref(sl), C.byref(en))
        if r:
            raise AmgError(r, last_error())
        return {"slices": sl.value, "entries": en.value}

    def level_csr(self, level: int):
        n, z = self.info()[level]
        rp = np.empty(n + 1, np.int32)
        ci = np.empty(z, np.int32)
        v = np.empty(z)
        st = load().amg_level_csr(self._h, level, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
        if st:
            raise AmgError(st, last_error())
        return rp, ci, v

    KINDS = ("down0", "post0", "spmv", "update", "residual", "coarse_levels", "axpy", "prolong0")

    def profile(self, enable: bool = True):
        st = load().amg_profile(self._h, int(enable))
        if st:
            raise AmgError(st, last_error())

    def profile_read(self) -> dict:
        ms = np.zeros(8)
        cnt = np.zeros(8, np.int64)
        load().amg_profile_read(self._h, ms.ctypes.data, cnt.ctypes.data, 8)
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.KINDS)}

    def autotune(self, reps: int = 5, stream=None) -> int:
        """``amg_autotune``: pick each level's fastest sweep launch shape; returns how many changed."""
        c = C.c_int(0)
        st = load().amg_autotune(self._h, reps, C.byref(c), _stream_ptr(stream))
        if st:
            raise AmgError(st, last_error())
        return c.value

    def level_shape(self, level: int) -> list[int]:
        """``amg_level_shape``: [float down, float post, float64 down, float64 post]."""
        out = np.zeros(4, np.int32)
        st = load().amg_level_shape(self._h, level, out.ctypes.data)
        if st:
            raise AmgError(st, last_error())
        return [int(v) for v in out]

    def profile_levels(self):
        """``amg_profile_levels``: (ms[L+1, 3], counts[L+1, 3]) per level: down, up, coarsest."""
        nl = len(self.info())
        ms = np.zeros(3 * nl)
        cnt = np.zeros(3 * nl, np.int64)
        st = load().amg_profile_levels(self._h, nl, ms.ctypes.data, cnt.ctypes.data)
        if st:
            raise AmgError(st, last_error())
        return ms.reshape(nl, 3), cnt.reshape(nl, 3)

    def set_level_shape(self, level: int, shape) -> None:
        """``amg_set_level_shape`` (levels 1..L)."""
        arr = np.ascontiguousarray(shape, dtype=np.int32)
        st = load().amg_set_level_shape(self._h, level, arr.ctypes.data)
        if st:
            raise AmgError(st, last_error())

    def launch_count(self) -> int:
        return int(load().amg_launch_count(self._h))

    def residual_noalloc(self, b, x, r, stream=None):
        """``amg_residual_noalloc``: r = b - A x (device tensors); returns (||r||, ||b||)."""
        for name, t in (("b", b), ("x", x), ("r", r)):
            n = t.size if isinstance(t, np.ndarray) else t.numel()
            if n != self.n:
                raise ValueError(f"{name} holds {n} values, the hierarchy has {self.n} rows")
            if hasattr(t, "device") and getattr(t, "is_cuda", False) and t.device.index != self.device:
                raise ValueError(f"{name} is on cuda:{t.device.index}, the hierarchy on cuda:{self.device}")
        norms = np.zeros(2)
        bp, _ = _ptr(b, np.float64)
        xp, _ = _ptr(x, np.float64)
        rp, _ = _ptr(r, np.float64)
        st = load().amg_residual_noalloc(self._h, bp, xp, rp, norms.ctypes.data, _stream_ptr(stream))
        if st:
            raise AmgError(st, last_error())
        return float(norms[0]), float(norms[1])

    def prolongator(self, level: int):
        """``amg_level_prolongator``: the smoothed P of a level as CSR parts."""
        lib = load()
        nz = C.c_int64()
        st = lib.amg_level_prolongator(self._h, level, C.byref(nz), None, None, None)
        if st:
            raise AmgError(st, last_error())
        n = self.info()[level][0]
        rp = np.empty(n + 1, np.int32)
        ci = np.empty(max(nz.value, 1), np.int32)
        v = np.empty(max(nz.value, 1))
        st = lib.amg_level_prolongator(self._h, level, C.byref(nz), rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
        if st:
            raise AmgError(st, last_error())
        return rp, ci[: nz.value], v[: nz.value]

    def coarse_info(self) -> dict:
        """``amg_coarse_info``: the coarsest solver in use ("dense"/"iter"),
        its rows and its ILU(1) blocks."""
        k, r, b = C.c_int(), C.c_int(), C.c_int()
        st = load().amg_coarse_info(self._h, C.byref(k), C.byref(r), C.byref(b))
        if st:
            raise AmgError(st, last_error())
        return {"kind": "iter" if k.value == COARSE_ITER else "dense", "rows": r.value, "blocks": b.value}

    def coarse_factors(self) -> np.ndarray:
        """``amg_coarse_factors``: (blocks, 32, 32) ILU(1) factors, L below
        the diagonal (unit diagonal implied), U on and above."""
        nb = self.coarse_info()["blocks"]
        F = np.empty((nb, 32, 32))
        st = load().amg_coarse_factors(self._h, F.ctypes.data)
        if st:
            raise AmgError(st, last_error())
        return F

    def coarse_solve(self, b, x, stream=None) -> int:
        """``amg_coarse_solve``: the iterative coarsest solve alone; returns
        the iterations run (x written in place)."""
        bp, _ = _ptr(b, np.float64)
        xp, _ = _ptr(x, np.float64)
        it = C.c_int(0)
        st = load().amg_coarse_solve(self._h, bp, xp, C.byref(it), _stream_ptr(stream))
        if st:
            raise AmgError(st, last_error())
        return it.value

    def setup_times(self):
        ms = np.zeros(4)
        load().amg_setup_times(self._h, ms.ctypes.data)
        return {"total_ms": ms[0], "matching_ms": ms[1], "galerkin_ms": ms[2], "other_ms": ms[3]}

    def refresh(self, A, stream=None, check: bool = True) -> int:
        """``amg_refresh``: new values of the finest matrix on the same pattern
        (same aggregates and prolongator weights; coarse operators, smoothers
        and the coarsest inverse formed again). Returns the status (raises
        with ``check``)."""
        lib = load()
        rp, rp_dev = _ptr(A.row_ptr, np.int32)
        ci, ci_dev = _ptr(A.col, np.int32)
        v, v_dev = _ptr(A.val, np.float64)
        if not (rp_dev == ci_dev == v_dev):
            raise TypeError("CSR arrays must all be host or all device")
        csr = AmgCsr(int(A.n), len(A.col), rp, ci, v, int(rp_dev))
        st = lib.amg_refresh(self._h, C.byref(csr), _stream_ptr(stream))
        if check and st:
            raise AmgError(st, last_error())
        return st

    def set_smoother(self, nu: int, nblocks: int = 0, stream=None):
        """``amg_set_smoother``: nu = 0 the one-sweep l1-Jacobi default; nu >= 1
        sweeps of l1 hybrid Gauss-Seidel over ``nblocks`` row blocks per level."""
        st = load().amg_set_smoother(self._h, nu, nblocks, _stream_ptr(stream))
        if st:
            raise AmgError(st, last_error())

    def refresh_ms(self) -> float:
        ms = C.c_double(0.0)
        load().amg_refresh_time(self._h, C.byref(ms))
        return ms.value


class Batch:
    """``amg_batch_create`` / ``pcg_solve_batch``: independent systems in one launch."""

    def __init__(self, amgs):
        lib = load()
        self.amgs = list(amgs)           # keeps the handles alive
        arr = (C.c_void_p * len(self.amgs))(*[a._h.value for a in self.amgs])
        b = C.c_void_p()
        st = lib.amg_batch_create(len(self.amgs), arr, C.byref(b))
        if st:
            raise AmgError(st, last_error())
        self._b = b

    def close(self):
        if getattr(self, "_b", None):
            load().amg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, bs, xs, rtol: float = 1e-8, maxit: int = 1000, stream=None):
        """Solve every system; xs updated in place. Returns (status, iters[m], statuses[m])."""
        m = len(self.amgs)
        bp = (C.c_void_p * m)(*[_ptr(b, np.float64)[0] for b in bs])
        xp = (C.c_void_p * m)(*[_ptr(x, np.float64)[0] for x in xs])
        it = np.zeros(m, np.int32)
        sts = np.zeros(m, np.int32)
        st = load().pcg_solve_batch(self._b, bp, xp, rtol, maxit, it.ctypes.data, sts.ctypes.data,
                                    _stream_ptr(stream))
        return st, it, sts


def serve_plan(resident, engine_bytes, budget: int, max_engines: int, loads=None):
    """``amg_serve_plan`` (host only): engines per mesh under a byte budget.

    Returns (status, engines[m], planned bytes)."""
    m = len(resident)
    res = np.ascontiguousarray(resident, dtype=np.uint64)
    eb = np.ascontiguousarray(engine_bytes, dtype=np.uint64)
    ld = None if loads is None else np.ascontiguousarray(loads, dtype=np.float64)
    eng = np.zeros(m, np.int32)
    tot = C.c_size_t(0)
    st = load().amg_serve_plan(m, res.ctypes.data, eb.ctypes.data, None if ld is None else ld.ctypes.data,
                               int(budget), int(max_engines), eng.ctypes.data, C.byref(tot))
    return st, eng, int(tot.value)


@dataclasses.dataclass
class ServeResult:
    status: int
    iters: int
    true_rel: float
    lane: int          # 0: whole-solve lane, 1: engine slot
    queue_ms: float
    run_ms: float
    total_ms: float


class Server:
    """``amg_server_*``: continuous-batching request loop over resident hierarchies.

    ``submit`` queues (mesh, b, x0, x) and returns a ticket; ``progress`` visits
    the engines; ``result`` returns a ServeResult once the request finished
    (None before). Buffers passed to ``submit`` are kept referenced here until
    the request's result has been read."""

    def __init__(self, amgs, mode: str = "fcg32", slots: int = 4, max_engines: int = 2, chunk: int = 4,
                 queue_cap: int = 4096, rtol: float = 1e-8, maxit: int = 1000, hbm_budget: int = 0, loads=None,
                 solo: bool = True, batch_min: int = 3, lane_priority: bool = False):
        lib = load()
        self.amgs = list(amgs)
        p = ServerParams()
        lib.amg_server_default_params(C.byref(p))
        p.mode = _MODES[mode] if isinstance(mode, str) else int(mode)
        p.slots, p.max_engines, p.chunk, p.queue_cap = slots, max_engines, chunk, queue_cap
        p.rtol, p.maxit, p.hbm_budget, p.solo = rtol, maxit, int(hbm_budget), int(bool(solo))
        p.batch_min, p.lane_priority = batch_min, int(bool(lane_priority))
        arr = (C.c_void_p * len(self.amgs))(*[a._h.value for a in self.amgs])
        ld = None if loads is None else np.ascontiguousarray(loads, dtype=np.float64)
        srv = C.c_void_p()
        st = lib.amg_server_create(C.byref(p), len(self.amgs), arr, None if ld is None else ld.ctypes.data,
                                   C.byref(srv))
        if st:
            raise AmgError(st, last_error())
        self._s = srv
        self._keep = {}

    def close(self):
        if getattr(self, "_s", None):
            load().amg_server_destroy(self._s)
            self._s = None
            self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def mesh_info(self, mesh: int):
        """(engines, slots, engine bytes, resident bytes) of one mesh."""
        e, k = C.c_int(), C.c_int()
        eb, rb = C.c_size_t(), C.c_size_t()
        st = load().amg_server_mesh_info(self._s, mesh, C.byref(e), C.byref(k), C.byref(eb), C.byref(rb))
        if st:
            raise AmgError(st, last_error())
        return e.value, k.value, eb.value, rb.value

    def info(self):
        """dict: budget, used (planned bytes), queued, running, launches."""
        b, u = C.c_size_t(), C.c_size_t()
        q, r = C.c_int(), C.c_int()
        n = C.c_int64()
        st = load().amg_server_info(self._s, C.byref(b), C.byref(u), C.byref(q), C.byref(r), C.byref(n))
        if st:
            raise AmgError(st, last_error())
        return {"budget": b.value, "used": u.value, "queued": q.value, "running": r.value, "launches": n.value}

    def submit(self, mesh: int, b, x0, x):
        """Queue a request; returns (status, ticket)."""
        t = C.c_int64(0)
        st = load().amg_server_submit(self._s, mesh, _ptr(b, np.float64)[0], _ptr(x0, np.float64)[0],
                                          _ptr(x, np.float64)[0], C.byref(t))
        if st == OK:
            self._keep[t.value] = (b, x0, x)
        return st, t.value

    def progress(self, wait: bool = False) -> int:
        """One visit of every engine; returns the number of requests finished."""
        f = C.c_int(0)
        st = load().amg_server_progress(self._s, int(bool(wait)), C.byref(f))
        if st:
            raise AmgError(st, last_error())
        return f.value

    def result(self, ticket: int):
        done, sts, it, lane = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        tr = C.c_double()
        tm = np.zeros(3)
        st = load().amg_server_result(self._s, ticket, C.byref(done), C.byref(sts), C.byref(it), C.byref(tr),
                                      C.byref(lane), tm.ctypes.data)
        if st:
            raise AmgError(st, last_error())
        if not done.value:
            return None
        self._keep.pop(ticket, None)
        return ServeResult(sts.value, it.value, tr.value, lane.value, float(tm[0]), float(tm[1]), float(tm[2]))

    def drain(self, tickets):
        """Run until every ticket has finished; returns {ticket: ServeResult}."""
        out = {}
        pending = list(tickets)
        while pending:
            self.progress(wait=True)
            rest = []
            for t in pending:
                r = self.result(t)
                if r is None:
                    rest.append(t)
                else:
                    out[t] = r
            pending = rest
        return out
