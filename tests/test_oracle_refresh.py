"""Pins of the oracle's partial hierarchy reuse (Sec. 4: with the topology
fixed and new coefficients, the same prolongators/restrictors rebuild the
hierarchy and its smoothers).

Checked against facts outside the refresh code: a fresh setup (same values,
and 2A, whose matching weights are scale-free so its aggregates are the same),
exact power-of-two scaling of every Galerkin product, the dense triple product
with the kept prolongator, numpy's l1 row sums, and dense solves.
"""
import numpy as np
import pytest

import oracle as O
from paper_2210_16660_gb300 import workloads as W


def _snapshot(h):
    levels = [h.level(l) for l in range(h.nlevels)]
    aggs = [h.level_agg(l) for l in range(h.nlevels - 1)]
    passes = [[h.pass_agg(l, ps)[0].copy() for ps in range(h.level_size(l)[2])] for l in range(h.nlevels - 1)]
    return levels, aggs, passes, h.coarse_factor()


def _scaled(A, s):
    return W.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val * s)


def _same(a, b):
    la, ga, pa, fa = a
    lb, gb, pb, fb = b
    assert len(la) == len(lb)
    for x, y in zip(la, lb):
        for key in ("row_ptr", "col", "val", "dinv", "w"):
            assert np.array_equal(x[key], y[key]), key
    for (m1, p1), (m2, p2) in zip(ga, gb):
        assert np.array_equal(m1, m2) and np.array_equal(p1, p2)
    for q1, q2 in zip(pa, pb):
        assert all(np.array_equal(u, v) for u, v in zip(q1, q2))
    assert np.array_equal(fa, fb)


@pytest.mark.parametrize("N,ratio", [(6, 1.0), (9, 1.04)])
def test_refresh_with_the_same_values_is_the_identity(N, ratio):
    A = W.make_problem(N, ratio, seed=3).A
    h = O.Hierarchy(A, coarse_max=8, n_pass=2)
    before = _snapshot(h)
    assert h.refresh(A) == O.OK
    _same(before, _snapshot(h))


@pytest.mark.parametrize("N,ratio", [(6, 1.0), (9, 1.04)])
def test_refresh_of_2A_equals_a_fresh_setup_of_2A(N, ratio):
    """Eq. (weights) is invariant under A -> 2A, so setup(2A) keeps the
    aggregates of setup(A); a refresh to 2A must then give setup(2A) bit for
    bit, and every coarse matrix is exactly twice the old one."""
    A = W.make_problem(N, ratio, seed=4).A
    h = O.Hierarchy(A, coarse_max=8, n_pass=2)
    old = _snapshot(h)
    assert h.refresh(_scaled(A, 2.0)) == O.OK
    new = _snapshot(h)
    fresh = O.Hierarchy(_scaled(A, 2.0), coarse_max=8, n_pass=2)
    _same(new, _snapshot(fresh))
    for x, y in zip(old[0], new[0]):
        assert np.array_equal(y["val"], 2.0 * x["val"])
        assert np.array_equal(y["dinv"], 0.5 * x["dinv"])
    np.testing.assert_allclose(new[3], np.sqrt(2.0) * old[3], rtol=1e-14, atol=1e-14)


def test_refresh_equals_the_dense_galerkin_product():
    """New coefficients D A D: the maps stay, every level is P^T A' P with the
    kept composed prolongator, and D^-1 is the inverse l1 row sum."""
    A = W.make_problem(10, 1.04, seed=5).A
    A2 = W.rescaled(A, seed=11)
    h = O.Hierarchy(A, coarse_max=8, n_pass=2)
    old = _snapshot(h)
    assert h.refresh(A2) == O.OK
    new = _snapshot(h)
    for (m1, p1), (m2, p2) in zip(old[1], new[1]):
        assert np.array_equal(m1, m2) and np.array_equal(p1, p2)
    for q1, q2 in zip(old[2], new[2]):
        assert all(np.array_equal(u, v) for u, v in zip(q1, q2))
    levels = new[0]
    assert np.array_equal(levels[0]["val"], A2.val)
    for l in range(len(levels) - 1):
        a = W.CSR(levels[l]["n"], levels[l]["row_ptr"], levels[l]["col"], levels[l]["val"]).to_dense()
        agg, p = new[1][l]
        nc = levels[l + 1]["n"]
        P = np.zeros((a.shape[0], nc))
        keep = agg >= 0
        P[np.nonzero(keep)[0], agg[keep]] = p[keep]
        ref = P.T @ a @ P
        got = W.CSR(nc, levels[l + 1]["row_ptr"], levels[l + 1]["col"], levels[l + 1]["val"]).to_dense()
        assert np.array_equal(levels[l + 1]["row_ptr"], old[0][l + 1]["row_ptr"])
        assert np.array_equal(levels[l + 1]["col"], old[0][l + 1]["col"])
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    for lv in levels:
        a = W.CSR(lv["n"], lv["row_ptr"], lv["col"], lv["val"]).to_dense()
        np.testing.assert_allclose(lv["dinv"], 1.0 / np.abs(a).sum(1), rtol=1e-15)
    # the factor is the Cholesky factor of the new coarsest matrix
    last = levels[-1]
    aL = W.CSR(last["n"], last["row_ptr"], last["col"], last["val"]).to_dense()
    L = new[3]
    np.testing.assert_allclose(np.tril(L) @ np.tril(L).T, aL, rtol=0, atol=1e-12 * np.abs(aL).max())


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_refreshed_hierarchy_solves_the_new_system(mode):
    """A new grading of the same mesh (same pattern, other coefficients)."""
    old = W.make_problem(12, 1.04, seed=6)
    new = W.make_problem(12, 1.08, seed=7)
    assert np.array_equal(old.A.col, new.A.col)
    h = O.Hierarchy(old.A, coarse_max=20, n_pass=2)
    assert h.refresh(new.A) == O.OK
    res = h.solve(new.b, rtol=1e-8, mode=mode)
    assert res["status"] == O.OK
    x_dense = np.linalg.solve(new.A.to_dense(), new.b)
    assert np.linalg.norm(res["x"] - x_dense) <= 1e-6 * np.linalg.norm(x_dense)
    fresh = O.Hierarchy(new.A, coarse_max=20, n_pass=2).solve(new.b, rtol=1e-8, mode=mode)
    # the kept aggregates stay a good coarse space for the new coefficients
    assert res["iters"] <= 2 * fresh["iters"] + 5


def test_refresh_rejects_another_pattern_and_keeps_the_hierarchy():
    A = W.make_problem(8, 1.04, seed=8).A
    h = O.Hierarchy(A, coarse_max=8, n_pass=2)
    before = _snapshot(h)
    other = W.make_problem(9, 1.04, seed=8).A
    assert h.refresh(other) == O.ERR_ARG
    moved = W.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    row = A.n // 2                                  # an interior row (27 entries)
    s, e = moved.row_ptr[row], moved.row_ptr[row + 1]
    assert e - s > 1
    moved.col[s:e] = moved.col[s:e][::-1].copy()   # unsorted columns, other pattern
    assert h.refresh(moved) == O.ERR_ARG
    _same(before, _snapshot(h))
