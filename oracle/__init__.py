"""ctypes front end of the CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle checks the CUDA library and is used by
the test suite, the package smoke check and the CPU-baseline leg of the
benchmark, nothing else. It imports nothing from the CUDA package.

``build()`` compiles ``oracle.c`` with gcc (``-O2 -ffp-contract=off``) into
``oracle/_build/liboracle.so``; ``load()`` builds on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

OK, ERR_ARG, ERR_OOM, ERR_BREAKDOWN, ERR_NOCONV, ERR_NAN, ERR_COARSE = 0, 1, 2, 3, 4, 5, 8

_lib = None


class _Cfg(C.Structure):
    """or_cfg_t: hierarchy and coarsest-solver options."""
    _fields_ = [("coarse_max", C.c_int), ("n_pass", C.c_int), ("max_levels", C.c_int),
                ("smoothed", C.c_int), ("csolver", C.c_int), ("cb", C.c_int), ("cmaxit", C.c_int),
                ("ctol", C.c_double)]


COARSE = {"auto": 0, "dense": 1, "iter": 2}

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, no GPU)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(LIB)
    I, P, D = C.c_int, C.c_void_p, C.c_double
    lib.or_weight.restype = D
    lib.or_weight.argtypes = [D, D, D, D, D]
    lib.or_l1_diag.restype = None
    lib.or_l1_diag.argtypes = [I, _i32p, _i32p, _f64p, _f64p]
    lib.or_spmv.restype = None
    lib.or_spmv.argtypes = [I, _i32p, _i32p, _f64p, _f64p, _f64p]
    lib.or_match.restype = I
    lib.or_match.argtypes = [I, _i32p, _i32p, _f64p, _f64p, _i32p]
    lib.or_aggregate.restype = I
    lib.or_aggregate.argtypes = [I, _i32p, _i32p, _f64p, _i32p, _f64p, _i32p, _f64p, _f64p]
    lib.or_rap.restype = I
    lib.or_rap.argtypes = [I, _i32p, _i32p, _f64p, _i32p, _f64p, I, C.POINTER(C.c_int64),
                           P, P, P]
    lib.or_chol.restype = I
    lib.or_chol.argtypes = [I, _f64p, _f64p]
    lib.or_chol_solve.restype = None
    lib.or_chol_solve.argtypes = [I, _f64p, _f64p, _f64p]
    lib.or_setup.restype = I
    lib.or_setup.argtypes = [I, _i32p, _i32p, _f64p, I, I, I, C.POINTER(P)]
    lib.or_setup_ex.restype = I
    lib.or_setup_ex.argtypes = [I, _i32p, _i32p, _f64p, I, I, I, I, C.POINTER(P)]
    lib.or_setup_cfg.restype = I
    lib.or_setup_cfg.argtypes = [I, _i32p, _i32p, _f64p, C.POINTER(_Cfg), C.POINTER(P)]
    lib.or_coarse_kind.restype = I
    lib.or_coarse_kind.argtypes = [P]
    lib.or_coarse_ilu_nnz.restype = C.c_int64
    lib.or_coarse_ilu_nnz.argtypes = [P]
    lib.or_coarse_ilu.restype = None
    lib.or_coarse_ilu.argtypes = [P, _i32p, _i32p, _f64p, _i32p]
    lib.or_coarse_solve.restype = I
    lib.or_coarse_solve.argtypes = [P, _f64p, _f64p]
    lib.or_coarse_prec.restype = None
    lib.or_coarse_prec.argtypes = [P, _f64p, _f64p]
    lib.or_coarse_stats.restype = None
    lib.or_coarse_stats.argtypes = [P, C.POINTER(C.c_int64)]
    lib.or_level_P_nnz.restype = C.c_int64
    lib.or_level_P_nnz.argtypes = [P, I]
    lib.or_level_P.restype = None
    lib.or_level_P.argtypes = [P, I, _i32p, _i32p, _f64p]
    lib.or_set_smoother.restype = I
    lib.or_set_smoother.argtypes = [P, I, I]
    lib.or_refresh.restype = I
    lib.or_refresh.argtypes = [P, I, _i32p, _i32p, _f64p]
    lib.or_free.restype = None
    lib.or_free.argtypes = [P]
    lib.or_nlevels.restype = I
    lib.or_nlevels.argtypes = [P]
    lib.or_level_size.restype = None
    lib.or_level_size.argtypes = [P, I, C.POINTER(I), C.POINTER(C.c_int64), C.POINTER(I)]
    lib.or_level_copy.restype = None
    lib.or_level_copy.argtypes = [P, I, _i32p, _i32p, _f64p, _f64p, _f64p]
    lib.or_level_agg.restype = None
    lib.or_level_agg.argtypes = [P, I, _i32p, _f64p]
    lib.or_pass_agg.restype = I
    lib.or_pass_agg.argtypes = [P, I, I, _i32p]
    lib.or_pass_n.restype = I
    lib.or_pass_n.argtypes = [P, I, I]
    lib.or_coarse_factor.restype = None
    lib.or_coarse_factor.argtypes = [P, _f64p]
    lib.or_vcycle.restype = I
    lib.or_vcycle.argtypes = [P, _f64p, _f64p, I]
    lib.or_solve.restype = I
    lib.or_solve.argtypes = [P, _f64p, _f64p, D, I, I, C.POINTER(I), P, C.POINTER(D)]
    _lib = lib
    return lib


def _csr_args(A):
    return (int(A.n), np.ascontiguousarray(A.row_ptr, np.int32),
            np.ascontiguousarray(A.col, np.int32), np.ascontiguousarray(A.val, np.float64))


# ------------------------------------------------------------ primitives
def weight(aij, aii, ajj, wi, wj) -> float:
    """Eq. (weights) for one edge."""
    return load().or_weight(aij, aii, ajj, wi, wj)


def l1_diag(A) -> np.ndarray:
    n, rp, ci, v = _csr_args(A)
    d = np.empty(n)
    load().or_l1_diag(n, rp, ci, v, d)
    return d


def spmv(A, x) -> np.ndarray:
    n, rp, ci, v = _csr_args(A)
    y = np.empty(n)
    load().or_spmv(n, rp, ci, v, np.ascontiguousarray(x, np.float64), y)
    return y


def match(A, w) -> np.ndarray:
    """Greedy matching (mate array, -1 = unmatched)."""
    n, rp, ci, v = _csr_args(A)
    mate = np.empty(n, np.int32)
    st = load().or_match(n, rp, ci, v, np.ascontiguousarray(w, np.float64), mate)
    if st < 0:
        raise MemoryError("oracle matching")
    return mate


def aggregate(A, mate, w):
    """Aggregates of one pass: (agg, p, w_c)."""
    n, rp, ci, v = _csr_args(A)
    agg = np.empty(n, np.int32)
    p = np.empty(n)
    wc = np.empty(n)
    nc = load().or_aggregate(n, rp, ci, v, np.ascontiguousarray(mate, np.int32),
                             np.ascontiguousarray(w, np.float64), agg, p, wc)
    return agg, p, wc[:nc].copy()


def rap(A, agg, p, nc):
    """Galerkin product P^T A P with the tentative prolongator; returns CSR parts."""
    n, rp, ci, v = _csr_args(A)
    agg = np.ascontiguousarray(agg, np.int32)
    p = np.ascontiguousarray(p, np.float64)
    nz = C.c_int64(0)
    lib = load()
    st = lib.or_rap(n, rp, ci, v, agg, p, nc, C.byref(nz), None, None, None)
    if st:
        raise RuntimeError(f"oracle rap status {st}")
    rpc = np.empty(nc + 1, np.int32)
    cic = np.empty(nz.value, np.int32)
    vc = np.empty(nz.value)
    st = lib.or_rap(n, rp, ci, v, agg, p, nc, C.byref(nz), rpc.ctypes.data, cic.ctypes.data,
                    vc.ctypes.data)
    if st:
        raise RuntimeError(f"oracle rap status {st}")
    return rpc, cic, vc


def chol(Adense):
    n = Adense.shape[0]
    L = np.empty((n, n))
    st = load().or_chol(n, np.ascontiguousarray(Adense, np.float64), L)
    return st, L


def chol_solve(L, b):
    n = L.shape[0]
    x = np.empty(n)
    load().or_chol_solve(n, np.ascontiguousarray(L), np.ascontiguousarray(b, np.float64), x)
    return x


# ------------------------------------------------------------ hierarchy
class Hierarchy:
    """Oracle AMG hierarchy (aggregation by matching, tentative prolongator)."""

    def __init__(self, A, coarse_max: int = 200, n_pass: int = 3, max_levels: int = 30, smoothed: bool = False,
                 coarse: str = "dense", coarse_block: int = 32, coarse_tol: float = 1e-3,
                 coarse_maxit: int = 30):
        """``smoothed``: prolongators P = (I - omega D^-1 A) P_hat (smoothed
        aggregation, Sec. 3.1) instead of the tentative P_hat.

        ``coarse``: the coarsest solver (Sec. 3.1). "dense": Cholesky (the
        setup fails above 4096 rows); "iter": flexible CG preconditioned by
        block-Jacobi with ILU(1) blocks of ``coarse_block`` rows, stopped at
        ``||r|| <= coarse_tol ||b||`` or after ``coarse_maxit`` iterations;
        "auto": dense up to 4096 rows, else iterative."""
        lib = load()
        n, rp, ci, v = _csr_args(A)
        h = C.c_void_p()
        cfg = _Cfg(coarse_max, n_pass, max_levels, int(smoothed), COARSE[coarse], coarse_block, coarse_maxit,
                   coarse_tol)
        st = lib.or_setup_cfg(n, rp, ci, v, C.byref(cfg), C.byref(h))
        self.status = st
        if st:
            raise RuntimeError(f"oracle setup status {st}")
        self._h = h
        self.n = n

    def set_smoother(self, nu: int, nblocks: int = 0) -> int:
        """nu = 0: the setup's one-sweep l1-Jacobi; nu >= 1: nu sweeps of l1
        hybrid Gauss-Seidel (forward before, backward after the coarse
        correction) over ``nblocks`` row blocks per level (0: one row each)."""
        return load().or_set_smoother(self._h, nu, nblocks)

    def refresh(self, A) -> int:
        """Partial reuse (Sec. 4): new values of the finest matrix on the same
        pattern; the aggregates and prolongator weights are kept, the Galerkin
        products, smoothers and coarsest factor are formed again. Returns the
        status (ERR_ARG for another pattern; the hierarchy is then unchanged
        unless a later level failed)."""
        n, rp, ci, v = _csr_args(A)
        return load().or_refresh(self._h, n, rp, ci, v)

    def close(self):
        if getattr(self, "_h", None):
            load().or_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nlevels(self) -> int:
        return load().or_nlevels(self._h)

    def level_size(self, l: int):
        n, z, np_ = C.c_int(), C.c_int64(), C.c_int()
        load().or_level_size(self._h, l, C.byref(n), C.byref(z), C.byref(np_))
        return n.value, z.value, np_.value

    def level(self, l: int) -> dict:
        n, z, _ = self.level_size(l)
        rp = np.empty(n + 1, np.int32)
        ci = np.empty(z, np.int32)
        v = np.empty(z)
        dinv = np.empty(n)
        w = np.empty(n)
        load().or_level_copy(self._h, l, rp, ci, v, dinv, w)
        return {"n": n, "row_ptr": rp, "col": ci, "val": v, "dinv": dinv, "w": w}

    def level_agg(self, l: int):
        n, _, _ = self.level_size(l)
        agg = np.empty(n, np.int32)
        p = np.empty(n)
        load().or_level_agg(self._h, l, agg, p)
        return agg, p

    def pass_agg(self, l: int, ps: int):
        lib = load()
        m = lib.or_pass_n(self._h, l, ps)
        agg = np.empty(max(m, 1), np.int32)
        nc = lib.or_pass_agg(self._h, l, ps, agg)
        return agg[:m], nc

    def prolongator(self, l: int):
        """Explicit (smoothed) prolongator of level l as CSR parts, or None
        for the tentative one (use level_agg)."""
        lib = load()
        nz = lib.or_level_P_nnz(self._h, l)
        if nz < 0:
            return None
        n, _, _ = self.level_size(l)
        rp = np.empty(n + 1, np.int32)
        ci = np.empty(max(nz, 1), np.int32)
        v = np.empty(max(nz, 1))
        lib.or_level_P(self._h, l, rp, ci, v)
        return rp, ci[:nz], v[:nz]

    def coarse_factor(self):
        n, _, _ = self.level_size(self.nlevels - 1)
        L = np.empty((n, n))
        load().or_coarse_factor(self._h, L)
        return L

    @property
    def coarse_kind(self) -> str:
        """The coarsest solver in use: "dense" or "iter"."""
        return ("dense", "iter")[load().or_coarse_kind(self._h)]

    def coarse_ilu(self):
        """ILU(1) factors of the coarsest level's blocks as CSR parts plus the
        position of each row's diagonal (L strictly below it, with a unit
        diagonal not stored; U from it on)."""
        lib = load()
        nz = lib.or_coarse_ilu_nnz(self._h)
        if nz < 0:
            return None
        n, _, _ = self.level_size(self.nlevels - 1)
        rp = np.empty(n + 1, np.int32)
        ci = np.empty(max(nz, 1), np.int32)
        v = np.empty(max(nz, 1))
        dg = np.empty(max(n, 1), np.int32)
        lib.or_coarse_ilu(self._h, rp, ci, v, dg)
        return rp, ci[:nz], v[:nz], dg[:n]

    def coarse_solve(self, b):
        """The coarsest solver alone: (x, inner iterations)."""
        n, _, _ = self.level_size(self.nlevels - 1)
        x = np.empty(n)
        its = load().or_coarse_solve(self._h, np.ascontiguousarray(b, np.float64), x)
        if its < 0:
            raise MemoryError("oracle coarse solve")
        return x, its

    def coarse_prec(self, r):
        """The block-Jacobi ILU(1) preconditioner of the coarsest level."""
        n, _, _ = self.level_size(self.nlevels - 1)
        z = np.empty(n)
        load().or_coarse_prec(self._h, np.ascontiguousarray(r, np.float64), z)
        return z

    def coarse_stats(self):
        """(calls, inner iterations in total, inner iterations of the last call)"""
        out = (C.c_int64 * 3)()
        load().or_coarse_stats(self._h, out)
        return tuple(int(v) for v in out)

    def vcycle(self, r, fp32: bool = False) -> np.ndarray:
        z = np.empty(self.n)
        st = load().or_vcycle(self._h, np.ascontiguousarray(r, np.float64), z, int(fp32))
        if st:
            raise RuntimeError(f"oracle vcycle status {st}")
        return z

    def solve(self, b, x0=None, rtol: float = 1e-8, maxit: int = 1000, mode: str = "pcg64"):
        """PCG ("pcg64": float64 V-cycle) or FCG(1) ("fcg32": float32 V-cycle).

        Returns dict(status, x, iters, hist, true_rel).
        """
        m = {"pcg64": 0, "fcg32": 1}[mode]
        x = np.zeros(self.n) if x0 is None else np.array(x0, np.float64, copy=True)
        hist = np.zeros(maxit + 1)
        it = C.c_int(0)
        tr = C.c_double(0.0)
        st = load().or_solve(self._h, np.ascontiguousarray(b, np.float64), x, rtol, maxit, m,
                             C.byref(it), hist.ctypes.data, C.byref(tr))
        return {"status": st, "x": x, "iters": it.value, "hist": hist[: it.value + 1],
                "true_rel": tr.value}
