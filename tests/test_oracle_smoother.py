"""Pins of the oracle's hybrid Gauss-Seidel smoother (Sec. 3.1: nu sweeps of
block Jacobi over the row blocks of the distribution, each block solved by a
forward (pre) or backward (post) Gauss-Seidel pass; l1 form, see the oracle).

Checked against: the one-sweep l1-Jacobi V-cycle it must reduce to with one
row per block, the dense Eq. (multiplicative composition) with
M = blockdiag(L_pp + D_l1) built here from the definition, symmetry and the
spectrum of B A, and dense solves.
"""
import numpy as np
import pytest

import oracle as O
from paper_2210_16660_gb300 import workloads as W


def _prolongator(agg, p, nc):
    P = np.zeros((agg.size, nc))
    keep = agg >= 0
    P[np.nonzero(keep)[0], agg[keep]] = p[keep]
    return P


def _rows_per_block(n, nblocks):
    return 1 if nblocks == 0 else max(1, -(-n // nblocks))


def _hybrid_M(a, nb):
    """blockdiag(L_pp + D_l1): lower triangle of each diagonal block, with
    d_i = a_ii + sum over j outside i's block of |a_ij|."""
    n = a.shape[0]
    M = np.zeros_like(a)
    for lo in range(0, n, nb):
        hi = min(n, lo + nb)
        M[lo:hi, lo:hi] = np.tril(a[lo:hi, lo:hi], -1)
        for i in range(lo, hi):
            off = np.abs(a[i]).sum() - np.abs(a[i, lo:hi]).sum()
            M[i, i] = a[i, i] + off
    return M


def _dense_B(h, nu, nblocks):
    L = h.nlevels - 1
    levels = [h.level(l) for l in range(L + 1)]
    dense = [W.CSR(lv["n"], lv["row_ptr"], lv["col"], lv["val"]).to_dense() for lv in levels]
    B = np.linalg.inv(dense[L])
    for l in range(L - 1, -1, -1):
        a = dense[l]
        n = a.shape[0]
        M = _hybrid_M(a, _rows_per_block(n, nblocks))
        np.testing.assert_allclose(levels[l]["dinv"], 1.0 / np.diag(M), rtol=1e-15)
        agg, p = h.level_agg(l)
        P = _prolongator(agg, p, dense[l + 1].shape[0])
        I = np.eye(n)
        pre = np.linalg.matrix_power(I - np.linalg.solve(M, a), nu)
        post = np.linalg.matrix_power(I - np.linalg.solve(M.T, a), nu)
        E = post @ (I - P @ B @ P.T @ a) @ pre
        B = (I - E) @ np.linalg.inv(a)
    return B


@pytest.mark.parametrize("fp32", [False, True])
def test_one_row_per_block_and_one_sweep_is_l1_jacobi(fp32):
    A = W.make_problem(9, 1.04, seed=3).A
    h = O.Hierarchy(A, coarse_max=20, n_pass=2)
    r = W.normals(31, A.n)
    z_jacobi = h.vcycle(r, fp32=fp32)
    assert h.set_smoother(1, 0) == O.OK
    z_sweep = h.vcycle(r, fp32=fp32)
    assert np.array_equal(z_sweep, z_jacobi)
    assert h.set_smoother(0, 0) == O.OK
    assert np.array_equal(h.vcycle(r, fp32=fp32), z_jacobi)


@pytest.mark.parametrize("nu,nblocks", [(1, 7), (2, 7), (4, 7), (4, 3), (2, 0)])
def test_hybrid_vcycle_is_the_multiplicative_composition(nu, nblocks):
    A, _, _ = W.q1_laplacian(8, 1.04)
    h = O.Hierarchy(A, coarse_max=8, n_pass=2)
    assert h.nlevels >= 3
    assert h.set_smoother(nu, nblocks) == O.OK
    B = _dense_B(h, nu, nblocks)
    Bo = np.stack([h.vcycle(e) for e in np.eye(A.n)], axis=1)
    assert np.allclose(Bo, B, rtol=1e-9, atol=1e-11 * np.abs(B).max())
    rel = np.abs(Bo - Bo.T).max() / np.abs(Bo).max()
    assert rel < 1e-12
    assert np.linalg.eigvalsh((Bo + Bo.T) / 2).min() > 0
    ev = np.linalg.eigvals(Bo @ A.to_dense()).real
    assert ev.min() > 0 and ev.max() <= 1 + 1e-10


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_hybrid_gs_solves_and_takes_fewer_iterations(mode):
    prob = W.make_problem(14, 1.04, seed=5)
    h = O.Hierarchy(prob.A, coarse_max=30, n_pass=2)
    base = h.solve(prob.b, rtol=1e-8, mode=mode)
    assert h.set_smoother(4, 64) == O.OK
    res = h.solve(prob.b, rtol=1e-8, mode=mode)
    assert res["status"] == O.OK
    x_dense = np.linalg.solve(prob.A.to_dense(), prob.b)
    assert np.linalg.norm(res["x"] - x_dense) <= 1e-6 * np.linalg.norm(x_dense)
    assert res["iters"] < base["iters"]


def test_set_smoother_rejects_bad_arguments():
    A = W.make_problem(6, 1.0, seed=2).A
    h = O.Hierarchy(A, coarse_max=8, n_pass=2)
    assert h.set_smoother(-1, 0) == O.ERR_ARG
    assert h.set_smoother(1, -2) == O.ERR_ARG
    assert h.set_smoother(65, 0) == O.ERR_ARG


def test_refresh_keeps_the_hybrid_diagonal():
    A = W.make_problem(8, 1.04, seed=6).A
    h = O.Hierarchy(A, coarse_max=8, n_pass=2)
    assert h.set_smoother(2, 5) == O.OK
    r = W.normals(7, A.n)
    z = h.vcycle(r)
    assert h.refresh(A) == O.OK
    assert np.array_equal(h.vcycle(r), z)
