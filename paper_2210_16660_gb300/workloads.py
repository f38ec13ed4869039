"""Seeded synthetic inputs: graded-hex Q1 Laplacian systems.

This module only builds inputs. It holds none of the solver's arithmetic
(no smoothing, coarsening, Krylov or coarse-solve step), so both the CUDA
path and the CPU oracle may consume what it produces.

Stand-in for the paper's Bolund LES pressure systems (Sec. 5, Sec. 6.1.1:
unstructured tetrahedral meshes with a wall-modelled boundary layer): the
trilinear (Q1) hexahedral stiffness matrix of the Laplacian on a tensor grid
with the z-spacing graded geometrically away from a Dirichlet wall at z = 0.

Matrix recipe
-------------
* Nodes ``N^3``; node index ``i = ix + N*(iy + N*iz)`` (x fastest).
* 1D assembled stiffness ``K`` (element ``(1/h)[[1,-1],[-1,1]]``) and mass
  ``M`` (element ``(h/6)[[2,1],[1,2]]``) along each axis.
* ``A = Kx(x)My(x)Mz + Mx(x)Ky(x)Mz + Mx(x)My(x)Kz``, each entry evaluated as
  exactly that three-term sum, each term left to right, so every entry is
  deterministic and ``a_ij == a_ji`` bitwise.
* Homogeneous Neumann on every face but ``z = 0``; on ``z = 0`` the Dirichlet
  condition ``u = 0`` is imposed by dropping the off-diagonal entries of those
  rows and columns while keeping the diagonal (so the dof count stays ``N^3``).
* The full 27-point pattern is stored, exact zeros included; columns sorted.

Right-hand side: ``b = A x*`` with ``x* ~ N(0,1)`` on non-Dirichlet nodes and
``x* = 0`` on the wall, drawn from a counter-based SplitMix64 stream mapped to
normals by Box-Muller, both in float64.
"""
from __future__ import annotations

import dataclasses

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 stream of ``seed``.

    Counter form of Steele, Lea & Flood's SplitMix64: output ``k`` mixes
    ``seed + (k+1)*gamma`` (all arithmetic mod 2^64).
    """
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def normals(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` standard normals (float64) by Box-Muller on SplitMix64 words.

    Normal ``2m`` and ``2m+1`` come from words ``2m`` and ``2m+1``;
    ``u = (word >> 11 + 1) * 2^-53`` lies in ``(0, 1]``.
    """
    pairs = (count + 1) // 2
    first = offset // 2
    w = splitmix64(seed, 2 * pairs + 2, 2 * first)
    u = ((w >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u1, u2 = u[0::2][: pairs + 1], u[1::2][: pairs + 1]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * (pairs + 1))
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    s = offset - 2 * first
    return z[s: s + count]


def graded_spacing(npts: int, ratio: float, length: float = 1.0) -> np.ndarray:
    """Cell sizes ``h_k = h0 * ratio^k`` (k = 0..npts-2) summing to ``length``.

    Powers are formed by repeated multiplication (plain IEEE operations, no
    libm ``pow``) so the sizes are bit-identical on every platform.
    """
    m = npts - 1
    if ratio == 1.0:
        return np.full(m, length / m)
    pw = [1.0]
    for _ in range(m):
        pw.append(pw[-1] * ratio)
    h0 = length * (ratio - 1.0) / (pw[m] - 1.0)
    return h0 * np.array(pw[:m])


def _tridiag_1d(h: np.ndarray):
    """1D assembled stiffness and mass: (K_diag, K_off, M_diag, M_off).

    ``*_off[k]`` couples nodes ``k`` and ``k+1``.
    """
    npts = h.size + 1
    kd = np.zeros(npts)
    md = np.zeros(npts)
    kd[:-1] += 1.0 / h
    kd[1:] += 1.0 / h
    md[:-1] += h / 3.0
    md[1:] += h / 3.0
    return kd, -1.0 / h, md, h / 6.0


def _band(diag: np.ndarray, off: np.ndarray, d: int) -> np.ndarray:
    """Values ``T[k, k+d]`` for every node k (0 where k+d is outside)."""
    out = np.zeros_like(diag)
    if d == 0:
        out[:] = diag
    elif d == 1:
        out[:-1] = off
    else:
        out[1:] = off
    return out


@dataclasses.dataclass
class CSR:
    """Square sparse matrix, CSR with int32 indices and float64 values."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        a[rows, self.col] = self.val
        return a


@dataclasses.dataclass
class Problem:
    """One synthetic pressure system ``A x = b`` with its manufactured solution."""

    name: str
    N: int
    A: CSR
    b: np.ndarray
    x_star: np.ndarray
    wall: np.ndarray  # bool, True on the Dirichlet nodes (iz == 0)
    spacing: tuple  # (hx, hy, hz) cell sizes


def q1_laplacian(N: int, ratio: float = 1.0, lx: float = 1.0, ly: float = 1.0,
                 lz: float = 1.0) -> tuple[CSR, np.ndarray, tuple]:
    """Q1 hex Laplacian on ``N^3`` nodes, z graded by ``ratio`` from z = 0."""
    if N < 2:
        raise ValueError("need at least 2 nodes per side")
    hx = graded_spacing(N, 1.0, lx)
    hy = graded_spacing(N, 1.0, ly)
    hz = graded_spacing(N, ratio, lz)
    kx, kxo, mx, mxo = _tridiag_1d(hx)
    ky, kyo, my, myo = _tridiag_1d(hy)
    kz, kzo, mz, mzo = _tridiag_1d(hz)
    n = N ** 3
    ix = np.arange(N)
    vals = np.zeros((n, 27))
    mask = np.zeros((n, 27), dtype=bool)
    cols = np.zeros((n, 27), dtype=np.int64)
    node = np.arange(n, dtype=np.int64)
    iz_of = node // (N * N)
    wall = iz_of == 0
    k = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                vx = ((ix + dx) >= 0) & ((ix + dx) < N)
                Kx, Mx = _band(kx, kxo, dx), _band(mx, mxo, dx)
                Ky, My = _band(ky, kyo, dy), _band(my, myo, dy)
                Kz, Mz = _band(kz, kzo, dz), _band(mz, mzo, dz)
                vy = ((ix + dy) >= 0) & ((ix + dy) < N)
                vz = ((ix + dz) >= 0) & ((ix + dz) < N)
                # broadcast over [iz, iy, ix]
                t1 = (Kx[None, None, :] * My[None, :, None]) * Mz[:, None, None]
                t2 = (Mx[None, None, :] * Ky[None, :, None]) * Mz[:, None, None]
                t3 = (Mx[None, None, :] * My[None, :, None]) * Kz[:, None, None]
                v = (t1 + t2) + t3
                ok = vz[:, None, None] & vy[None, :, None] & vx[None, None, :]
                vals[:, k] = v.reshape(-1)
                m = ok.reshape(-1)
                jz = iz_of + dz
                if k != 13:
                    m = m & ~wall & (jz != 0)
                mask[:, k] = m
                cols[:, k] = node + dx + N * (dy + N * dz)
                k += 1
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2 ** 31:
        raise ValueError("nnz does not fit int32 row pointers")
    A = CSR(n, row_ptr.astype(np.int32), cols[mask].astype(np.int32),
            np.ascontiguousarray(vals[mask]))
    return A, wall, (hx, hy, hz)


def spmv(A: CSR, x: np.ndarray) -> np.ndarray:
    """``A @ x`` for input generation (segment sums over each row's entries)."""
    prod = A.val * x[A.col]
    out = np.zeros(A.n)
    nonempty = np.diff(A.row_ptr) > 0
    if prod.size:
        sums = np.add.reduceat(prod, A.row_ptr[:-1][nonempty])
        out[nonempty] = sums
    return out


def make_problem(N: int, ratio: float = 1.0, seed: int = 1, lx: float = 1.0,
                 name: str | None = None) -> Problem:
    """System of one pressure solve: ``b = A x*``, ``x*`` seeded normals."""
    A, wall, sp = q1_laplacian(N, ratio, lx=lx)
    xs = normals(seed, A.n)
    xs[wall] = 0.0
    b = spmv(A, xs)
    return Problem(name or f"q1_{N}^3_r{ratio}", N, A, b, xs, wall, sp)


def rescaled(A: CSR, seed: int, spread: float = 0.5) -> CSR:
    """New coefficients on the same pattern: ``a'_ij = (d_i d_j) a_ij`` with
    ``d = 1 + spread * u``, ``u`` uniform on [0, 1) from SplitMix64 words.

    ``D A D`` stays SPD, and ``d_i d_j == d_j d_i`` exactly, so a bitwise
    symmetric ``A`` gives a bitwise symmetric ``A'``.
    """
    u = (splitmix64(seed, A.n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    d = 1.0 + spread * u
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    return CSR(A.n, A.row_ptr.copy(), A.col.copy(), (d[rows] * d[A.col]) * A.val)


def make_rhs(problem: Problem, k: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """``k`` further right-hand sides: columns of ``X*`` and ``B = A X*``.

    Returned row-major ``(n, k)`` (the k values of one row are contiguous).
    """
    n = problem.A.n
    xs = normals(seed, n * k).reshape(k, n)
    xs[:, problem.wall] = 0.0
    bs = np.stack([spmv(problem.A, xs[c]) for c in range(k)])
    return np.ascontiguousarray(bs.T), np.ascontiguousarray(xs.T)


def perturb_step(problem: Problem, x_prev: np.ndarray, seed: int, step: int,
                 scale: float = 0.01) -> tuple[np.ndarray, np.ndarray]:
    """Time-step-like request: ``x*_t = x_prev + scale*rms(x_prev)*xi``.

    Returns ``(b_t, x*_t)`` with ``b_t = A x*_t``; the warm start is ``x_prev``.
    """
    n = problem.A.n
    xi = normals(seed, n, offset=step * n)
    rms = float(np.sqrt(np.mean(x_prev * x_prev)))
    xs = x_prev + scale * rms * xi
    xs[problem.wall] = 0.0
    return spmv(problem.A, xs), xs


def batch_sizes(count: int = 48, lo: int = 24, hi: int = 112, seed: int = 3) -> list[int]:
    """Node counts per side for a batch of independent systems, uniform on [lo, hi]."""
    w = splitmix64(seed, count)
    return [int(lo + int(v % np.uint64(hi - lo + 1))) for v in w]


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream of ``count`` requests at ``rate``
    per second, starting at 0: exponential gaps ``-ln(u) / rate`` with ``u``
    in ``(0, 1]`` from SplitMix64 words; rate = inf puts every arrival at 0."""
    if not np.isfinite(rate):
        return np.zeros(count)
    w = splitmix64(seed, count)
    u = ((w >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    gaps = -np.log(u) / rate
    gaps[0] = 0.0
    return np.cumsum(gaps)


def uniform_choices(count: int, m: int, seed: int) -> np.ndarray:
    """``count`` indices uniform on ``0..m-1`` (which mesh each request is for)."""
    w = splitmix64(seed, count, offset=1 << 20)
    return (w % np.uint64(m)).astype(np.int64)


def time_steps(problem: Problem, x_start: np.ndarray, steps: int, seed: int,
               scale: float = 0.01) -> list[tuple[np.ndarray, np.ndarray, np.ndarray]]:
    """A chain of time-step-like requests on one mesh: step t has exact
    solution ``x*_t`` (``perturb_step`` of ``x*_{t-1}``), right-hand side
    ``b_t = A x*_t`` and warm start ``x0_t = x*_{t-1}``. Returns
    ``[(b_t, x0_t, x*_t)]`` for t = 1..steps."""
    out = []
    x_prev = x_start
    for t in range(1, steps + 1):
        b, xs = perturb_step(problem, x_prev, seed, t, scale)
        out.append((b, x_prev, xs))
        x_prev = xs
    return out
