"""Pins of the oracle's iterative coarsest solver (Sec. 3.1, coarsest solver:
flexible CG preconditioned by block-Jacobi whose blocks are solved by ILU(1),
stopped after a residual reduction of three orders of magnitude or 30
iterations).

Checked against facts other than the oracle itself:
  * the kept pattern equals the level-1 fill set of graph theory (an entry
    (i, j) of a block has fill level <= 1 iff it is stored or some k <
    min(i, j) of the block has both (i, k) and (k, j) stored), computed here
    with numpy;
  * the defining property of an incomplete LU on a pattern P: L unit lower,
    U upper, both supported on P, and (L U)_ij = a_ij on P;
  * without fill (tridiagonal blocks) ILU(1) is the exact LU, so the
    preconditioner is the exact block inverse and a block-aligned
    block-diagonal system is solved in one iteration;
  * the preconditioner equals two triangular solves with scipy;
  * the inner iteration equals textbook PCG (numpy) with the same
    preconditioner, stops at the first iterate meeting the tolerance, never
    runs more than its cap, and with a tight tolerance gives the dense
    solution;
  * scale covariance: the factors of 2A are L and 2U bit for bit;
  * the outer solve with the iterative coarsest solver reaches the dense
    solution of the whole system.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle as O
from paper_2210_16660_gb300 import workloads as W


def _csr_from_dense(a):
    n = a.shape[0]
    rp, ci, v = [0], [], []
    for i in range(n):
        nz = np.nonzero(a[i])[0]
        ci.extend(nz.tolist())
        v.extend(a[i, nz].tolist())
        rp.append(len(ci))
    return W.CSR(n, np.array(rp, np.int32), np.array(ci, np.int32), np.array(v))


def _laplace2d(m, shift=0.0):
    """5-point Laplacian on an m x m grid (+ shift I): has level-1 fill."""
    n = m * m
    a = np.zeros((n, n))
    for y in range(m):
        for x in range(m):
            i = x + m * y
            a[i, i] = 4.0 + shift
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                xx, yy = x + dx, y + dy
                if 0 <= xx < m and 0 <= yy < m:
                    a[i, xx + m * yy] = -1.0
    return a


def _q1_dense(N, ratio, lx=1.0):
    A, _, _ = W.q1_laplacian(N, ratio, lx=lx)
    return A, A.to_dense()


def _one_level(A, cb=32, **kw):
    """A hierarchy whose only (coarsest) level is A itself."""
    return O.Hierarchy(A, coarse_max=A.n, n_pass=2, coarse="iter", coarse_block=cb, **kw)


def _factors(h, n):
    rp, ci, v, dg = h.coarse_ilu()
    F = np.zeros((n, n))
    kept = np.zeros((n, n), bool)
    rows = np.repeat(np.arange(n), np.diff(rp))
    F[rows, ci] = v
    kept[rows, ci] = True
    for i in range(n):
        assert ci[dg[i]] == i
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)
    L = np.tril(F, -1) + np.eye(n)
    U = np.triu(F)
    return L, U, kept


def _level1_pattern(a, cb):
    """Stored entries of each block plus their level-1 fill, by the path rule."""
    n = a.shape[0]
    P = np.zeros((n, n), bool)
    for s in range(0, n, cb):
        e = min(n, s + cb)
        B = a[s:e, s:e] != 0
        m = e - s
        idx = np.arange(m)
        fill = np.zeros((m, m), bool)
        for k in range(m):
            col = B[:, k] & (idx > k)
            row = B[k, :] & (idx > k)
            fill |= np.outer(col, row)
        P[s:e, s:e] = B | fill
    return P


@pytest.mark.parametrize("m,cb", [(12, 32), (12, 50), (12, 144), (9, 20)])
def test_ilu1_pattern_and_product(m, cb):
    a = _laplace2d(m)
    n = a.shape[0]
    h = _one_level(_csr_from_dense(a), cb=cb)
    assert h.nlevels == 1 and h.coarse_kind == "iter"
    L, U, kept = _factors(h, n)
    P = _level1_pattern(a, cb)
    assert np.array_equal(kept, P)
    # the test is discriminating: there is fill of level 1 beyond A's pattern
    assert (P & (a == 0)).any()
    # incomplete LU on P: (LU)_ij = a_ij on P; L, U supported on P
    LU = L @ U
    assert np.abs(LU[P] - a[P]).max() <= 1e-13 * np.abs(a).max()
    assert not (L[~P] != 0).any() and not (U[~P] != 0).any()
    # and it is not the complete LU (fill of level 2 and more is dropped)
    blk = sl.block_diag(*[a[s:min(n, s + cb), s:min(n, s + cb)] for s in range(0, n, cb)])
    assert np.abs(LU - blk).max() > 1e-3


def test_ilu1_on_a_coarse_q1_level():
    A, a = _q1_dense(9, 1.04)
    h = O.Hierarchy(A, coarse_max=90, n_pass=2, coarse="iter")
    lv = h.level(h.nlevels - 1)
    ac = W.CSR(lv["n"], lv["row_ptr"], lv["col"], lv["val"]).to_dense()
    n = ac.shape[0]
    L, U, kept = _factors(h, n)
    # stored zeros count as stored entries (level 0)
    stored = np.zeros((n, n), bool)
    stored[np.repeat(np.arange(n), np.diff(lv["row_ptr"])), lv["col"]] = True
    marker = np.where(stored, 1.0, 0.0)
    assert np.array_equal(kept, _level1_pattern(marker, 32))
    LU = L @ U
    assert np.abs(LU[kept] - ac[kept]).max() <= 1e-13 * np.abs(ac).max()


def test_without_fill_ilu1_is_the_exact_block_inverse():
    # tridiagonal blocks have no fill: ILU(1) = LU, M = blockdiag(A_b)
    n, cb = 96, 32
    a = np.zeros((n, n))
    rng = np.random.default_rng(5)
    for i in range(n):
        a[i, i] = 2.5 + rng.random()
        if i + 1 < n and (i + 1) % cb:
            a[i, i + 1] = a[i + 1, i] = -1.0
    h = _one_level(_csr_from_dense(a), cb=cb)
    r = rng.standard_normal(n)
    z = h.coarse_prec(r)
    assert np.abs(z - np.linalg.solve(a, r)).max() <= 1e-13 * np.abs(z).max()
    x, its = h.coarse_solve(r)
    assert its == 1
    assert np.abs(x - np.linalg.solve(a, r)).max() <= 1e-12 * np.abs(x).max()


def test_preconditioner_is_two_triangular_solves():
    a = _laplace2d(11, shift=0.3)
    n, cb = a.shape[0], 32
    h = _one_level(_csr_from_dense(a), cb=cb)
    L, U, _ = _factors(h, n)
    r = np.random.default_rng(1).standard_normal(n)
    z = h.coarse_prec(r)
    for s in range(0, n, cb):
        e = min(n, s + cb)
        y = sl.solve_triangular(L[s:e, s:e], r[s:e], lower=True, unit_diagonal=True)
        want = sl.solve_triangular(U[s:e, s:e], y, lower=False)
        assert np.abs(z[s:e] - want).max() <= 1e-12 * np.abs(want).max()


def _textbook_pcg(a, b, minv, tol, maxit):
    x = np.zeros_like(b)
    r = b.copy()
    z = minv(r)
    p = z.copy()
    rho = r @ z
    bn = np.linalg.norm(b)
    for k in range(1, maxit + 1):
        q = a @ p
        alpha = rho / (p @ q)
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= tol * bn:
            return x, k
        z = minv(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, maxit


def _stalled_coarse_level():
    """Coarsest level of a stretched, strongly graded mesh whose coarsening
    stalls (the level keeps more than 0.9 of its rows)."""
    A, _, _ = W.q1_laplacian(40, 1.2, lx=4.0)
    h = O.Hierarchy(A, coarse_max=200, n_pass=2, coarse="iter")
    lv = h.level(h.nlevels - 1)
    ac = W.CSR(lv["n"], lv["row_ptr"], lv["col"], lv["val"])
    return h, ac


def test_inner_iteration_follows_its_rule():
    h, ac = _stalled_coarse_level()
    n = ac.n
    assert n > 200  # stalled above the coarse target
    a = ac.to_dense()
    L, U, _ = _factors(h, n)

    def minv(r):
        z = np.empty_like(r)
        for s in range(0, n, 32):
            e = min(n, s + 32)
            y = sl.solve_triangular(L[s:e, s:e], r[s:e], lower=True, unit_diagonal=True)
            z[s:e] = sl.solve_triangular(U[s:e, s:e], y, lower=False)
        return z

    rng = np.random.default_rng(7)
    for trial in range(3):
        b = rng.standard_normal(n)
        x, its = h.coarse_solve(b)
        assert 1 <= its <= 30
        res = np.linalg.norm(b - a @ x) / np.linalg.norm(b)
        if its < 30:
            assert res <= 1e-3 * (1 + 1e-9)
        # first iterate meeting the tolerance: the one before does not
        xr, kr = _textbook_pcg(a, b, minv, 1e-3, 30)
        assert kr == its
        assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)


def test_inner_iteration_cap_and_tight_tolerance():
    A, _, _ = W.q1_laplacian(40, 1.2, lx=4.0)
    b0 = None
    for tol, cap in ((1e-3, 2), (1e-13, 3000)):
        h = O.Hierarchy(A, coarse_max=200, n_pass=2, coarse="iter", coarse_tol=tol, coarse_maxit=cap)
        lv = h.level(h.nlevels - 1)
        a = W.CSR(lv["n"], lv["row_ptr"], lv["col"], lv["val"]).to_dense()
        if b0 is None:
            b0 = np.random.default_rng(3).standard_normal(a.shape[0])
        x, its = h.coarse_solve(b0)
        if cap == 2:
            assert its == 2
            assert np.linalg.norm(b0 - a @ x) > 1e-3 * np.linalg.norm(b0)
        else:
            assert its < cap
            xd = np.linalg.solve(a, b0)
            assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_factors_scale_with_the_matrix():
    A, _, _ = W.q1_laplacian(12, 1.04)
    h1 = O.Hierarchy(A, coarse_max=90, n_pass=2, coarse="iter")
    A2 = W.CSR(A.n, A.row_ptr, A.col, 2.0 * A.val)
    h2 = O.Hierarchy(A2, coarse_max=90, n_pass=2, coarse="iter")
    rp1, ci1, v1, dg1 = h1.coarse_ilu()
    rp2, ci2, v2, dg2 = h2.coarse_ilu()
    assert np.array_equal(rp1, rp2) and np.array_equal(ci1, ci2)
    n = rp1.size - 1
    upper = np.zeros(v1.size, bool)
    for i in range(n):
        upper[dg1[i]:rp1[i + 1]] = True
    assert np.array_equal(v2[upper], 2.0 * v1[upper])
    assert np.array_equal(v2[~upper], v1[~upper])
    # a refresh with the same values keeps them bit for bit, one with 2A
    # gives the factors of a fresh setup of 2A
    assert h1.refresh(A) == 0
    assert np.array_equal(h1.coarse_ilu()[2], v1)
    assert h1.refresh(A2) == 0
    assert np.array_equal(h1.coarse_ilu()[2], v2)


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_outer_solve_with_iterative_coarse_reaches_dense_solution(mode):
    prob = W.make_problem(14, 1.1, seed=3, lx=2.0)
    a = prob.A.to_dense()
    xd = np.linalg.solve(a, prob.b)
    hd = O.Hierarchy(prob.A, coarse_max=300, n_pass=2, coarse="dense")
    hi = O.Hierarchy(prob.A, coarse_max=300, n_pass=2, coarse="iter")
    assert hi.nlevels == hd.nlevels >= 2
    rd = hd.solve(prob.b, rtol=1e-8, mode=mode)
    ri = hi.solve(prob.b, rtol=1e-8, mode=mode)
    assert ri["status"] == 0 and ri["true_rel"] <= 1e-8
    assert np.linalg.norm(ri["x"] - xd) <= 1e-5 * np.linalg.norm(xd)
    # an approximate coarsest solve costs a few outer iterations at most
    assert rd["iters"] <= ri["iters"] <= rd["iters"] + 6
    calls, total, _ = hi.coarse_stats()
    assert calls == ri["iters"] and total <= 30 * calls


def test_vcycle_with_tight_inner_solve_equals_dense():
    A, _, _ = W.q1_laplacian(12, 1.04)
    hd = O.Hierarchy(A, coarse_max=90, n_pass=2, coarse="dense")
    hi = O.Hierarchy(A, coarse_max=90, n_pass=2, coarse="iter", coarse_tol=1e-14, coarse_maxit=5000)
    r = np.random.default_rng(2).standard_normal(A.n)
    zd, zi = hd.vcycle(r), hi.vcycle(r)
    assert np.linalg.norm(zi - zd) <= 1e-10 * np.linalg.norm(zd)


def test_auto_choice_and_dense_limit():
    A, _, _ = W.q1_laplacian(12, 1.04)
    assert O.Hierarchy(A, coarse_max=90, n_pass=2, coarse="auto").coarse_kind == "dense"
    # a stretched, strongly graded mesh whose coarsening stalls at 4162 rows,
    # above the dense limit of 4096
    B, _, _ = W.q1_laplacian(64, 1.1, lx=4.0)
    with pytest.raises(RuntimeError, match="status 8"):
        O.Hierarchy(B, coarse_max=200, n_pass=2, coarse="dense")
    h = O.Hierarchy(B, coarse_max=200, n_pass=2, coarse="auto")
    assert h.coarse_kind == "iter" and h.level_size(h.nlevels - 1)[0] == 4162
