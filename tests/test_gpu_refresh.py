"""amg_refresh (partial reuse of the hierarchy, Sec. 4) on the GPU.

Bar: after refreshing to new coefficients on the same pattern, the device
hierarchy equals the oracle's refreshed hierarchy bit for bit (coarse
matrices; kept aggregates), and solves meet the oracle's bar (iterations
+-1, true residual <= rtol, ||x - x_oracle|| / ||x_oracle|| <= 1e-6). Arrays
are updated in place, so graphs captured before the refresh (whole-solve,
batch) must give the same bits as a handle refreshed before its first solve.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2210_16660_gb300 import binding as B  # noqa: E402
from paper_2210_16660_gb300 import workloads as W  # noqa: E402

RTOL = 1e-8
X_TOL = 1e-6


def _levels_equal(h_or, amg):
    info = amg.info()
    assert len(info) == h_or.nlevels
    for l in range(h_or.nlevels):
        lv = h_or.level(l)
        rp, ci, v = amg.level_csr(l)
        assert np.array_equal(rp, lv["row_ptr"]) and np.array_equal(ci, lv["col"])
        assert np.array_equal(v.view(np.int64), lv["val"].view(np.int64)), f"level {l} values differ"
        if l + 1 < h_or.nlevels:
            agg_or, _ = h_or.level_agg(l)
            agg_gpu, _ = amg.level_agg(l, -1)
            assert np.array_equal(agg_gpu, agg_or)


def _rhs(A, seed):
    xs = W.normals(seed, A.n)
    return W.spmv(A, xs)


@pytest.mark.parametrize("N,ratio", [(13, 1.04), (33, 1.04)])
def test_refreshed_hierarchy_bit_exact_vs_oracle(N, ratio):
    A = W.make_problem(N, ratio, seed=3).A
    A2 = W.rescaled(A, seed=12)
    h_or = O.Hierarchy(A, coarse_max=200, n_pass=2)
    amg = B.AMG.from_csr(A)
    aggs = [amg.level_agg(l, -1)[0].copy() for l in range(len(amg.info()) - 1)]
    assert h_or.refresh(A2) == O.OK
    amg.refresh(A2)
    _levels_equal(h_or, amg)
    for l, a in enumerate(aggs):
        assert np.array_equal(amg.level_agg(l, -1)[0], a)      # the aggregates were kept
    assert amg.refresh_ms() > 0.0


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_refreshed_solve_parity(mode):
    """New grading of the same mesh: other coefficients, same pattern."""
    old = W.make_problem(40, 1.04, seed=6)
    new = W.make_problem(40, 1.08, seed=7)
    h_or = O.Hierarchy(old.A, coarse_max=200, n_pass=2)
    assert h_or.refresh(new.A) == O.OK
    ref = h_or.solve(new.b, rtol=RTOL, maxit=1000, mode=mode)
    amg = B.AMG.from_csr(old.A, mode=mode)
    amg.refresh(new.A)
    b = torch.from_numpy(new.b).cuda()
    x = torch.zeros_like(b)
    res = amg.solve(b, x, rtol=RTOL, maxit=1000)
    assert res.status == 0, res.message
    assert abs(res.iters - ref["iters"]) <= 1, (res.iters, ref["iters"])
    xs = x.cpu().numpy()
    assert np.linalg.norm(new.b - W.spmv(new.A, xs)) <= RTOL * np.linalg.norm(new.b)
    assert np.linalg.norm(xs - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_graphs_captured_before_a_refresh_stay_valid(mode):
    prob = W.make_problem(32, 1.04, seed=8)
    A2 = W.rescaled(prob.A, seed=13)
    b_old = torch.from_numpy(prob.b).cuda()
    b = torch.from_numpy(_rhs(A2, 14)).cuda()
    a1 = B.AMG.from_csr(prob.A, mode=mode)
    assert a1.solve(b_old, torch.zeros_like(b_old)).status == 0      # captures the solve graph
    batch = B.Batch([a1])
    xb = [torch.zeros_like(b_old)]
    assert batch.solve([b_old], xb, rtol=RTOL)[0] == 0                 # and a batch graph
    a1.refresh(A2)
    x1 = torch.zeros_like(b)
    r1 = a1.solve(b, x1)
    a2 = B.AMG.from_csr(prob.A, mode=mode)
    a2.refresh(A2)                                                     # no graph before the refresh
    x2 = torch.zeros_like(b)
    r2 = a2.solve(b, x2)
    assert r1.status == r2.status == 0 and r1.iters == r2.iters
    assert torch.equal(x1, x2)
    xb = [torch.zeros_like(b)]
    st, it, _ = batch.solve([b], xb, rtol=RTOL)
    assert st == 0 and it[0] == r1.iters and torch.equal(xb[0], x1)
    batch.close()
    # many right-hand sides on the refreshed hierarchy
    Bm = torch.stack([b, 2.0 * b], 1).contiguous()
    X = torch.zeros_like(Bm)
    st, its, _, sts, _ = a1.solve_multi(Bm, X, rtol=RTOL)
    assert st == 0 and list(sts) == [0, 0]
    assert (X[:, 0] - x1).norm().item() <= 1e-6 * x1.norm().item()


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_refresh_with_the_same_values_keeps_the_bits(mode):
    prob = W.make_problem(36, 1.04, seed=9)
    b = torch.from_numpy(prob.b).cuda()
    amg = B.AMG.from_csr(prob.A, mode=mode)
    x0, x1 = torch.zeros_like(b), torch.zeros_like(b)
    r0 = amg.solve(b, x0)
    amg.refresh(prob.A)
    r1 = amg.solve(b, x1)
    assert r0.status == r1.status == 0 and r0.iters == r1.iters
    assert torch.equal(x0, x1)


def test_cluster_tail_is_refreshed():
    """The tail's shared-memory copy of the small levels is rebuilt: the same
    bits with and without the tail after a refresh."""
    import os
    prob = W.make_problem(48, 1.04, seed=15)
    A2 = W.rescaled(prob.A, seed=16)
    b = torch.from_numpy(_rhs(A2, 17)).cuda()
    a1 = B.AMG.from_csr(prob.A, mode="fcg32")
    os.environ["PCGAMG_TAIL"] = "0"
    try:
        a2 = B.AMG.from_csr(prob.A, mode="fcg32")
    finally:
        del os.environ["PCGAMG_TAIL"]
    a1.refresh(A2)
    a2.refresh(A2)
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    r1, r2 = a1.solve(b, x1), a2.solve(b, x2)
    assert r1.status == r2.status == 0 and r1.iters == r2.iters
    assert torch.equal(x1, x2)


def test_refresh_rejections_leave_the_handle_unchanged():
    prob = W.make_problem(20, 1.04, seed=18)
    b = torch.from_numpy(prob.b).cuda()
    amg = B.AMG.from_csr(prob.A)
    x0 = torch.zeros_like(b)
    amg.solve(b, x0)
    other = W.make_problem(21, 1.04, seed=18).A
    with pytest.raises(B.AmgError) as e:
        amg.refresh(other)
    assert e.value.status == B.ERR_ARG
    moved = W.CSR(prob.A.n, prob.A.row_ptr.copy(), prob.A.col.copy(), prob.A.val.copy())
    row = prob.A.n // 2
    s, t = moved.row_ptr[row], moved.row_ptr[row + 1]
    moved.col[s:t] = moved.col[s:t][::-1].copy()
    assert amg.refresh(moved, check=False) == B.ERR_ARG
    lopsided = W.CSR(prob.A.n, prob.A.row_ptr.copy(), prob.A.col.copy(), prob.A.val.copy())
    k = next(q for q in range(s, t) if prob.A.col[q] != row and prob.A.val[q] != 0.0)
    lopsided.val[k] *= 1.5                                   # a_ij != a_ji
    assert amg.refresh(lopsided, check=False) == B.ERR_ARG
    assert "symmetric" in B.last_error()
    x1 = torch.zeros_like(b)
    amg.solve(b, x1)
    assert torch.equal(x0, x1)


def test_full_size_128_refresh():
    """The benchmarked 128^3 system refreshed to new coefficients (D A D):
    same levels and aggregates, a converged solve, and far less time than a
    setup (no matching)."""
    prob = W.make_problem(128, 1.04, seed=2)
    A2 = W.rescaled(prob.A, seed=21)
    amg = B.AMG.from_csr(prob.A, mode="fcg32")
    info = amg.info()
    agg1 = amg.level_agg(1, -1)[0].copy()
    amg.refresh(A2)
    assert amg.info() == info
    assert np.array_equal(amg.level_agg(1, -1)[0], agg1)
    b = torch.from_numpy(_rhs(A2, 22)).cuda()
    x = torch.zeros_like(b)
    r = amg.solve(b, x, rtol=RTOL, maxit=1000)
    assert r.status == 0 and r.true_rel <= RTOL
    xs = x.cpu().numpy()
    bh = b.cpu().numpy()
    assert np.linalg.norm(bh - W.spmv(A2, xs)) <= RTOL * np.linalg.norm(bh)
    fresh = B.AMG.from_csr(A2, mode="fcg32")
    xf = torch.zeros_like(b)
    rf = fresh.solve(b, xf, rtol=RTOL, maxit=1000)
    assert r.iters <= 2 * rf.iters + 5
    assert amg.refresh_ms() < fresh.setup_times()["total_ms"]
