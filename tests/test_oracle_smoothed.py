"""Pins of the oracle's smoothed-aggregation prolongator (Sec. 3.1:
P = (I - omega D^-1 A) P_hat, D = diag(A), omega = 1 / ||D^-1 A||_inf).

Checked against: the dense product built here from the definition with
numpy's omega, the dense Galerkin product P^T A P and its exact symmetry, the
dense Eq. (multiplicative composition) with the explicit P, dense solves, and
the scale invariance of the whole construction (a refresh to 2A equals a fresh
setup of 2A bit for bit).
"""
import numpy as np
import pytest

import oracle as O
from paper_2210_16660_gb300 import workloads as W


def _dense(parts, n, m):
    rp, ci, v = parts
    M = np.zeros((n, m))
    rows = np.repeat(np.arange(n), np.diff(rp))
    M[rows, ci] = v
    return M


def _level_dense(h, l):
    lv = h.level(l)
    return W.CSR(lv["n"], lv["row_ptr"], lv["col"], lv["val"]).to_dense()


def _tentative(h, l, nc):
    agg, p = h.level_agg(l)
    P = np.zeros((agg.size, nc))
    keep = agg >= 0
    P[np.nonzero(keep)[0], agg[keep]] = p[keep]
    return P


@pytest.mark.parametrize("N,ratio", [(8, 1.0), (10, 1.04)])
def test_prolongator_is_the_smoothed_tentative_one(N, ratio):
    A, _, _ = W.q1_laplacian(N, ratio)
    h = O.Hierarchy(A, coarse_max=8, n_pass=2, smoothed=True)
    assert h.nlevels >= 3
    for l in range(h.nlevels - 1):
        a = _level_dense(h, l)
        n, nc = a.shape[0], h.level_size(l + 1)[0]
        d = np.diag(a)
        omega = 1.0 / (np.abs(a) / d[:, None]).sum(1).max()
        ref = (np.eye(n) - omega * (a / d[:, None])) @ _tentative(h, l, nc)
        P = _dense(h.prolongator(l), n, nc)
        assert np.abs(P - ref).max() <= 1e-14 * np.abs(ref).max()
        # pattern: the tentative column and the columns of the row's couplings
        agg, _ = h.level_agg(l)
        rp, ci, _ = h.prolongator(l)
        lv = h.level(l)
        for i in range(0, n, max(1, n // 50)):
            want = {int(agg[j]) for j in lv["col"][lv["row_ptr"][i]:lv["row_ptr"][i + 1]] if agg[j] >= 0}
            if agg[i] >= 0:
                want.add(int(agg[i]))
            assert list(ci[rp[i]:rp[i + 1]]) == sorted(want)
    assert h.prolongator(h.nlevels - 1) is None or h.nlevels == 1


@pytest.mark.parametrize("N,ratio", [(8, 1.0), (10, 1.04)])
def test_coarse_matrices_are_the_galerkin_products(N, ratio):
    A, _, _ = W.q1_laplacian(N, ratio)
    h = O.Hierarchy(A, coarse_max=8, n_pass=2, smoothed=True)
    for l in range(h.nlevels - 1):
        a = _level_dense(h, l)
        n, nc = a.shape[0], h.level_size(l + 1)[0]
        P = _dense(h.prolongator(l), n, nc)
        ac = _level_dense(h, l + 1)
        ref = P.T @ a @ P
        assert np.abs(ac - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.array_equal(ac, ac.T)               # bitwise symmetric by construction


def test_vcycle_is_the_multiplicative_composition_with_smoothed_P():
    A, _, _ = W.q1_laplacian(8, 1.04)
    h = O.Hierarchy(A, coarse_max=8, n_pass=2, smoothed=True)
    L = h.nlevels - 1
    dense = [_level_dense(h, l) for l in range(L + 1)]
    B = np.linalg.inv(dense[L])
    for l in range(L - 1, -1, -1):
        a = dense[l]
        n = a.shape[0]
        P = _dense(h.prolongator(l), n, dense[l + 1].shape[0])
        S = np.eye(n) - np.diag(h.level(l)["dinv"]) @ a
        E = S @ (np.eye(n) - P @ B @ P.T @ a) @ S
        B = (np.eye(n) - E) @ np.linalg.inv(a)
    Bo = np.stack([h.vcycle(e) for e in np.eye(A.n)], axis=1)
    assert np.allclose(Bo, B, rtol=1e-9, atol=1e-11 * np.abs(B).max())
    assert np.abs(Bo - Bo.T).max() <= 1e-12 * np.abs(Bo).max()
    ev = np.linalg.eigvals(Bo @ A.to_dense()).real
    assert ev.min() > 0 and ev.max() <= 1 + 1e-10


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_smoothed_aggregation_solves(mode):
    prob = W.make_problem(14, 1.04, seed=5)
    tent = O.Hierarchy(prob.A, coarse_max=30, n_pass=2).solve(prob.b, rtol=1e-8, mode=mode)
    h = O.Hierarchy(prob.A, coarse_max=30, n_pass=2, smoothed=True)
    res = h.solve(prob.b, rtol=1e-8, mode=mode)
    assert res["status"] == O.OK
    x_dense = np.linalg.solve(prob.A.to_dense(), prob.b)
    assert np.linalg.norm(res["x"] - x_dense) <= 1e-6 * np.linalg.norm(x_dense)
    assert res["iters"] < tent["iters"]


def test_refresh_of_2A_equals_a_fresh_smoothed_setup_of_2A():
    A = W.make_problem(9, 1.04, seed=4).A
    A2 = W.CSR(A.n, A.row_ptr.copy(), A.col.copy(), 2.0 * A.val)
    h = O.Hierarchy(A, coarse_max=8, n_pass=2, smoothed=True)
    old = [h.level(l)["val"].copy() for l in range(h.nlevels)]
    assert h.refresh(A) == O.OK
    assert all(np.array_equal(h.level(l)["val"], old[l]) for l in range(h.nlevels))
    assert h.refresh(A2) == O.OK
    fresh = O.Hierarchy(A2, coarse_max=8, n_pass=2, smoothed=True)
    assert fresh.nlevels == h.nlevels
    for l in range(h.nlevels):
        assert np.array_equal(h.level(l)["val"], fresh.level(l)["val"])
        assert np.array_equal(h.level(l)["val"], 2.0 * old[l])
        if l + 1 < h.nlevels:
            for x, y in zip(h.prolongator(l), fresh.prolongator(l)):
                assert np.array_equal(x, y)


def test_smoothed_prolongator_with_hybrid_gauss_seidel():
    """Both of the paper's choices at once (smoothed P, nu = 4 hybrid GS): the
    V-cycle is the dense composition with the explicit P and M = blockdiag(L + D_l1)."""
    A, _, _ = W.q1_laplacian(7, 1.04)
    h = O.Hierarchy(A, coarse_max=8, n_pass=2, smoothed=True)
    nu, nblocks = 4, 5
    assert h.set_smoother(nu, nblocks) == O.OK
    L = h.nlevels - 1
    dense = [_level_dense(h, l) for l in range(L + 1)]
    B = np.linalg.inv(dense[L])
    for l in range(L - 1, -1, -1):
        a = dense[l]
        n = a.shape[0]
        nb = max(1, -(-n // nblocks))
        M = np.zeros_like(a)
        for lo in range(0, n, nb):
            hi = min(n, lo + nb)
            M[lo:hi, lo:hi] = np.tril(a[lo:hi, lo:hi], -1)
            for i in range(lo, hi):
                M[i, i] = a[i, i] + np.abs(a[i]).sum() - np.abs(a[i, lo:hi]).sum()
        P = _dense(h.prolongator(l), n, dense[l + 1].shape[0])
        I = np.eye(n)
        pre = np.linalg.matrix_power(I - np.linalg.solve(M, a), nu)
        post = np.linalg.matrix_power(I - np.linalg.solve(M.T, a), nu)
        E = post @ (I - P @ B @ P.T @ a) @ pre
        B = (I - E) @ np.linalg.inv(a)
    Bo = np.stack([h.vcycle(e) for e in np.eye(A.n)], axis=1)
    assert np.allclose(Bo, B, rtol=1e-9, atol=1e-11 * np.abs(B).max())
    prob_b = W.spmv(A, W.normals(3, A.n))
    res = h.solve(prob_b, rtol=1e-10, mode="pcg64")
    assert res["status"] == O.OK
    assert np.linalg.norm(res["x"] - np.linalg.solve(A.to_dense(), prob_b)) <= 1e-8 * np.linalg.norm(res["x"])
