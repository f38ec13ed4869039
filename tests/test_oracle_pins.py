"""Pins of the CPU oracle against facts other than itself.

Each check comes from the mathematics of the method (Sec. 3.1 of the paper)
or from an independent computation: closed forms, invariants of the
tentative prolongator, brute force on tiny graphs, a different matching
algorithm with a provably equal result, dense linear algebra (numpy/scipy),
and the explicit product of error-propagation matrices of the V-cycle
(Eq. multiplicative composition).
"""
import itertools
import math

import numpy as np
import pytest

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


def _random_spd_graph(rng, n, density=0.5):
    """Random SPD matrix with mixed-sign couplings (diagonally dominant)."""
    a = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < density:
                a[i, j] = a[j, i] = rng.uniform(-1.0, 0.4)
    a[np.diag_indices(n)] = np.abs(a).sum(1) + rng.uniform(0.1, 1.0, n)
    return a


def _prolongator(agg, p, nc):
    n = agg.size
    P = np.zeros((n, nc))
    for i in range(n):
        if agg[i] >= 0:
            P[i, agg[i]] = p[i]
    return P


# ------------------------------------------------------------------ weights
def test_weight_closed_form():
    # a_ij = -1, a_ii = a_jj = 2, w = 1: c = 1 - (-2)/4 = 1.5
    assert O.weight(-1.0, 2.0, 2.0, 1.0, 1.0) == 1.5
    # positive coupling lowers the weight below 1
    assert O.weight(0.5, 2.0, 2.0, 1.0, 1.0) == 0.75
    # w scaling: a_ij=-1, a_ii=1, a_jj=4, w=(2,1): 1 + 4/(4+4) = 1.5
    assert O.weight(-1.0, 1.0, 4.0, 2.0, 1.0) == 1.5
    # zero coupling is neutral
    assert O.weight(0.0, 3.0, 5.0, 0.7, 1.3) == 1.0


# ----------------------------------------------------------------- matching
def _candidates(a, w):
    n = a.shape[0]
    out = {}
    for i in range(n):
        for j in range(i + 1, n):
            if a[i, j] != 0:
                c = O.weight(a[i, j], a[i, i], a[j, j], w[i], w[j])
                if c > 1:
                    out[(i, j)] = c
    return out


def _locally_dominant(n, cand):
    """Matching by repeatedly taking edges heaviest at both ends (Preis-style).

    Under a strict total order this equals the greedy matching; it is a
    different algorithm, so agreement pins the oracle's sort-and-scan.
    """
    key = lambda e: (-cand[e], e[0], e[1])
    mate = [-1] * n
    live = dict(cand)
    while live:
        best = {}
        for e in live:
            for v in e:
                if v not in best or key(e) < key(best[v]):
                    best[v] = e
        taken = [e for e in live if best[e[0]] == e and best[e[1]] == e]
        assert taken
        for (i, j) in taken:
            mate[i], mate[j] = j, i
        live = {e: c for e, c in live.items() if mate[e[0]] < 0 and mate[e[1]] < 0}
    return np.array(mate)


def _all_matchings(edges, n):
    """Every matching of a small graph (list of edge subsets)."""
    out = [[]]

    def rec(k, used, cur):
        if k == len(edges):
            return
        for t in range(k, len(edges)):
            i, j = edges[t]
            if i in used or j in used:
                continue
            nxt = cur + [edges[t]]
            out.append(nxt)
            rec(t + 1, used | {i, j}, nxt)
    rec(0, frozenset(), [])
    return out


@pytest.mark.parametrize("seed", range(12))
def test_matching_pins(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(4, 12))
    a = _random_spd_graph(rng, n, 0.55)
    w = rng.uniform(0.5, 2.0, n) if seed % 2 else np.ones(n)
    A = _csr_from_dense(a)
    mate = O.match(A, w)
    cand = _candidates(a, w)
    # a matching
    for i in range(n):
        if mate[i] >= 0:
            assert mate[mate[i]] == i and mate[i] != i
            assert (min(i, mate[i]), max(i, mate[i])) in cand
    # maximal over the candidate edges
    for (i, j) in cand:
        assert mate[i] >= 0 or mate[j] >= 0
    # equal to the locally-dominant matching
    assert np.array_equal(mate, _locally_dominant(n, cand))
    # half-approximation of the maximum product (max log-weight) matching
    edges = sorted(cand)
    best = max(sum(math.log(cand[e]) for e in m) for m in _all_matchings(edges, n))
    got = sum(math.log(cand[(i, mate[i])]) for i in range(n) if mate[i] > i)
    assert got >= 0.5 * best - 1e-12


def test_matching_ties_break_by_index():
    # a path 0-1-2-3 with equal weights: greedy by (i, j) takes (0,1), (2,3)
    a = np.diag([2.0] * 4)
    for i in range(3):
        a[i, i + 1] = a[i + 1, i] = -1.0
    a[1, 1] = a[2, 2] = 2.0
    mate = O.match(_csr_from_dense(a), np.ones(4))
    assert list(mate) == [1, 0, 3, 2]


# --------------------------------------------------------------- aggregates
@pytest.mark.parametrize("seed", range(6))
def test_tentative_prolongator_invariants(seed):
    rng = np.random.default_rng(100 + seed)
    n = 40
    a = _random_spd_graph(rng, n, 0.12)
    # two decoupled rows
    for i in (3, 17):
        a[i, :] = 0
        a[:, i] = 0
        a[i, i] = 2.0
    w = rng.uniform(0.3, 3.0, n)
    A = _csr_from_dense(a)
    mate = O.match(A, w)
    agg, p, wc = O.aggregate(A, mate, w)
    nc = wc.size
    P = _prolongator(agg, p, nc)
    # decoupled rows leave the coarse space, every other row is in one aggregate
    off = a - np.diag(np.diag(a))
    decoupled = ~np.any(off != 0, axis=1)
    assert decoupled[3] and decoupled[17]
    assert np.all(agg[decoupled] == -1) and np.all(agg[~decoupled] >= 0)
    sizes = np.bincount(agg[agg >= 0], minlength=nc)
    assert np.all((sizes == 1) | (sizes == 2))
    # pairs are exactly the matched edges
    for i in range(n):
        if mate[i] >= 0:
            assert agg[i] == agg[mate[i]]
    # numbering increases with the first member
    first = [np.nonzero(agg == I)[0][0] for I in range(nc)]
    assert first == sorted(first)
    # orthonormal columns: P^T P = I
    assert np.allclose(P.T @ P, np.eye(nc), atol=1e-15)
    # range contains w on the coupled rows: P w_c = w (Eq. prolongator)
    keep = agg >= 0
    assert np.allclose((P @ wc)[keep], w[keep], rtol=1e-15)


# ---------------------------------------------------------------------- RAP
@pytest.mark.parametrize("N,ratio", [(4, 1.0), (6, 1.04), (8, 1.04)])
def test_rap_equals_dense_product(N, ratio):
    A, _, _ = W.q1_laplacian(N, ratio)
    w = np.ones(A.n)
    mate = O.match(A, w)
    agg, p, wc = O.aggregate(A, mate, w)
    nc = wc.size
    rp, ci, v = O.rap(A, agg, p, nc)
    Ac = W.CSR(nc, rp, ci, v).to_dense()
    P = _prolongator(agg, p, nc)
    ref = P.T @ A.to_dense() @ P
    assert np.allclose(Ac, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    # bitwise symmetric, SPD
    assert np.array_equal(Ac, Ac.T)
    assert np.linalg.eigvalsh(Ac).min() > 0
    # A_c w_c = P^T A w (w in the range of P)
    assert np.allclose(Ac @ wc, P.T @ (A.to_dense() @ w), atol=1e-12 * np.abs(ref).max())
    # pattern: every coupled aggregate pair is stored, columns sorted
    for I in range(nc):
        c = ci[rp[I]:rp[I + 1]]
        assert np.all(np.diff(c) > 0)


def test_l1_diagonal_dominates():
    A, _, _ = W.q1_laplacian(6, 1.04)
    a = A.to_dense()
    d = O.l1_diag(A)
    assert np.allclose(d, np.abs(a).sum(1), rtol=1e-15)
    assert np.all(d >= np.diag(a))
    # 2 D_l1 - A is SPD, so the smoother is A-convergent
    assert np.linalg.eigvalsh(2 * np.diag(d) - a).min() > 0


# ------------------------------------------------------------------ Cholesky
def test_cholesky():
    rng = np.random.default_rng(5)
    a = _random_spd_graph(rng, 30, 0.4)
    st, L = O.chol(a)
    assert st == 0
    assert np.allclose(L @ L.T, a, rtol=1e-13, atol=1e-13)
    b = rng.standard_normal(30)
    assert np.allclose(O.chol_solve(L, b), np.linalg.solve(a, b), rtol=1e-11)
    a[4, 4] = -1.0
    assert O.chol(a)[0] == O.ERR_BREAKDOWN


# ------------------------------------------------------------------ V-cycle
def _dense_vcycle_operator(h):
    """B from Eq. (multiplicative composition) with nu = 1, M = D_l1."""
    L = h.nlevels - 1
    levels = [h.level(l) for l in range(L + 1)]
    dense = [W.CSR(lv["n"], lv["row_ptr"], lv["col"], lv["val"]).to_dense() for lv in levels]
    B = np.linalg.inv(dense[L])
    for l in range(L - 1, -1, -1):
        Al = dense[l]
        n = Al.shape[0]
        Minv = np.diag(levels[l]["dinv"])
        agg, p = h.level_agg(l)
        P = _prolongator(agg, p, dense[l + 1].shape[0])
        I = np.eye(n)
        S = I - Minv @ Al
        E = S @ (I - P @ B @ P.T @ Al) @ S
        B = (I - E) @ np.linalg.inv(Al)
    return B


@pytest.mark.parametrize("N,ratio,cmax", [(6, 1.0, 8), (8, 1.04, 8), (8, 1.04, 40)])
def test_vcycle_is_the_multiplicative_composition(N, ratio, cmax):
    A, _, _ = W.q1_laplacian(N, ratio)
    h = O.Hierarchy(A, coarse_max=cmax, n_pass=2)
    assert h.nlevels >= 3
    B = _dense_vcycle_operator(h)
    Bo = np.stack([h.vcycle(e) for e in np.eye(A.n)], axis=1)
    assert np.allclose(Bo, B, rtol=1e-9, atol=1e-11 * np.abs(B).max())
    # symmetric and positive definite; spectrum of B A in (0, 1]
    rel = np.abs(Bo - Bo.T).max() / np.abs(Bo).max()
    assert rel < 1e-13
    assert np.linalg.eigvalsh((Bo + Bo.T) / 2).min() > 0
    ev = np.linalg.eigvals(Bo @ A.to_dense()).real
    assert ev.min() > 0 and ev.max() <= 1 + 1e-10


def test_vcycle_symmetry_large():
    A, _, _ = W.q1_laplacian(12, 1.04)
    h = O.Hierarchy(A, coarse_max=20, n_pass=3)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(A.n), rng.standard_normal(A.n)
    bx, by = h.vcycle(x), h.vcycle(y)
    assert abs(y @ bx - x @ by) <= 1e-13 * abs(y @ bx) + 1e-13 * np.linalg.norm(bx) * np.linalg.norm(y)
    # linear
    assert np.allclose(h.vcycle(2 * x - 3 * y), 2 * bx - 3 * by, rtol=1e-12, atol=1e-12 * np.abs(bx).max())


def test_vcycle32_close_to_vcycle64():
    A, _, _ = W.q1_laplacian(10, 1.04)
    h = O.Hierarchy(A, coarse_max=20)
    r = np.random.default_rng(2).standard_normal(A.n)
    z64, z32 = h.vcycle(r), h.vcycle(r, fp32=True)
    assert np.linalg.norm(z32 - z64) <= 1e-5 * np.linalg.norm(z64)
    assert not np.array_equal(z32, z64)


def test_single_level_is_exact():
    A, _, _ = W.q1_laplacian(5, 1.04)
    h = O.Hierarchy(A, coarse_max=200)
    assert h.nlevels == 1
    b = np.random.default_rng(3).standard_normal(A.n)
    assert np.allclose(h.vcycle(b), np.linalg.solve(A.to_dense(), b), rtol=1e-10)
    res = h.solve(b, rtol=1e-10)
    assert res["status"] == 0 and res["iters"] == 1


# --------------------------------------------------------------------- PCG
@pytest.mark.parametrize("N,ratio,mode", [(4, 1.0, "pcg64"), (6, 1.04, "pcg64"), (8, 1.04, "pcg64"),
                                          (8, 1.04, "fcg32")])
def test_pcg_matches_dense_solution(N, ratio, mode):
    p = W.make_problem(N, ratio, seed=11)
    a = p.A.to_dense()
    h = O.Hierarchy(p.A, coarse_max=16, n_pass=2)
    rtol = 1e-10
    res = h.solve(p.b, rtol=rtol, mode=mode)
    assert res["status"] == 0
    x_ref = np.linalg.solve(a, p.b)
    kappa = np.linalg.cond(a)
    assert np.linalg.norm(res["x"] - x_ref) <= kappa * rtol * np.linalg.norm(x_ref)
    assert np.linalg.norm(res["x"] - p.x_star) <= kappa * rtol * np.linalg.norm(p.x_star)
    # true residual within rtol; history starts at 1 (x0 = 0) and ends below rtol
    assert np.linalg.norm(p.b - a @ res["x"]) <= rtol * np.linalg.norm(p.b)
    assert res["hist"][0] == pytest.approx(1.0)
    assert res["hist"][-1] <= rtol
    # iteration count within the CG bound for kappa(BA)
    B = np.stack([h.vcycle(e) for e in np.eye(p.A.n)], axis=1)
    ev = np.linalg.eigvals(B @ a).real
    kb = ev.max() / ev.min()
    q = (math.sqrt(kb) - 1) / (math.sqrt(kb) + 1)
    bound = math.ceil(math.log(rtol / (2 * math.sqrt(kappa))) / math.log(q))
    assert res["iters"] <= bound


def test_pcg_error_monotone_in_a_norm():
    p = W.make_problem(8, 1.04, seed=4)
    a = p.A.to_dense()
    h = O.Hierarchy(p.A, coarse_max=16, n_pass=2)
    errs = []
    for k in range(1, 12):
        res = h.solve(p.b, rtol=1e-30, maxit=k)
        e = res["x"] - p.x_star
        errs.append(e @ a @ e)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))


def test_pcg_special_cases():
    p = W.make_problem(6, 1.04, seed=5)
    h = O.Hierarchy(p.A, coarse_max=16)
    # b = 0: x = 0 and no iteration
    res = h.solve(np.zeros(p.A.n), x0=np.ones(p.A.n))
    assert res["status"] == 0 and res["iters"] == 0 and not res["x"].any()
    # initial guess already converged
    res = h.solve(p.b, x0=np.linalg.solve(p.A.to_dense(), p.b), rtol=1e-8)
    assert res["status"] == 0 and res["iters"] == 0
    # maxit exhausted
    res = h.solve(p.b, rtol=1e-14, maxit=2)
    assert res["status"] == O.ERR_NOCONV and res["iters"] == 2
    # NaN in b
    b = p.b.copy()
    b[7] = np.nan
    assert h.solve(b)["status"] == O.ERR_NAN


def test_setup_rejects_bad_input():
    A, _, _ = W.q1_laplacian(4, 1.0)
    bad = W.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    bad.col[[1, 2]] = bad.col[[2, 1]]  # unsorted row
    with pytest.raises(RuntimeError):
        O.Hierarchy(bad)
    neg = W.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    neg.val[neg.col == 0] *= -1  # non-positive diagonal in row 0
    with pytest.raises(RuntimeError):
        O.Hierarchy(neg)


def test_indefinite_rejected():
    # symmetric, positive diagonal, but indefinite: the dense coarsest factor
    # (here the only level) reports breakdown instead of returning garbage
    a = np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.5], [0.0, 0.5, 1.0]])
    with pytest.raises(RuntimeError, match="status 3"):
        O.Hierarchy(_csr_from_dense(a), coarse_max=8, n_pass=1)


def test_hand_worked_pairwise_aggregation():
    """The oracle against a small example worked by hand from the equations
    of Sec. 3.1 (tests/golden/path5_pairwise_aggregation.json): edge weights,
    tie-break, numbering, normalised tentative prolongator, w_c and both
    Galerkin products of two passes."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "path5_pairwise_aggregation.json")))
    Ad = np.array(g["matrix_dense"], float)
    n = Ad.shape[0]
    rows, cols = np.nonzero(Ad)
    rp = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    A = W.CSR(n, rp, cols.astype(np.int32), Ad[rows, cols])
    w = np.ones(n)
    for i, j in zip(rows, cols):
        if i < j:
            assert O.weight(Ad[i, j], Ad[i, i], Ad[j, j], w[i], w[j]) == pytest.approx(g["edge_weight"], rel=1e-15)
    mate = O.match(A, w)
    assert list(mate) == g["pass0"]["mate"]
    agg, p, wc = O.aggregate(A, mate, w)
    assert list(agg) == g["pass0"]["agg"]
    np.testing.assert_allclose(p, g["pass0"]["p"], rtol=1e-15)
    np.testing.assert_allclose(wc, g["pass0"]["w_c"], rtol=1e-15)
    rpc, cic, vc = O.rap(A, agg, p, len(wc))
    Ac = np.zeros((len(wc), len(wc)))
    for i in range(len(wc)):
        Ac[i, cic[rpc[i]:rpc[i + 1]]] = vc[rpc[i]:rpc[i + 1]]
    np.testing.assert_allclose(Ac, g["pass0"]["A_c"], rtol=1e-15, atol=1e-15)
    h = O.Hierarchy(A, coarse_max=1, n_pass=2)
    assert h.nlevels == g["levels"]
    a1, nc1 = h.pass_agg(0, 1)
    assert list(a1) == g["pass1"]["agg"] and nc1 == g["pass1"]["n_c"]
    L1 = h.level(1)
    A1 = np.zeros((L1["n"], L1["n"]))
    for i in range(L1["n"]):
        A1[i, L1["col"][L1["row_ptr"][i]:L1["row_ptr"][i + 1]]] = L1["val"][L1["row_ptr"][i]:L1["row_ptr"][i + 1]]
    np.testing.assert_allclose(A1, g["level1"]["A"], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(L1["w"], g["level1"]["w"], rtol=1e-15)
    cagg, cp = h.level_agg(0)
    assert list(cagg) == g["level0_composed"]["agg"]
    np.testing.assert_allclose(cp, g["level0_composed"]["p"], rtol=1e-15)
