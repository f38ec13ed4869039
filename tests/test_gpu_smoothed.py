"""Smoothed aggregation on the GPU (Sec. 3.1: P = (I - omega D^-1 A) P_hat,
omega = 1 / ||D^-1 A||_inf, coarse matrices P^T A P) against the CPU oracle,
through the C ABI.

Bar: every level's smoothed prolongator, coarse matrix and aggregate map
equal the oracle's bit for bit (the device forms each value with the oracle's
summation order, every operation rounded on its own); solves keep the
single-solve bar (iterations within +-1, true relative residual <= rtol,
||x - x_oracle|| <= 1e-6 ||x_oracle||) in both modes, with the Gauss-Seidel
smoother and with the iterative coarsest solve; a refresh reproduces the
oracle's refreshed hierarchy bit for bit; batched solves equal single solves.
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


def _bits(a):
    return np.ascontiguousarray(a).view(np.int64)


def _compare(h_or, amg):
    info = amg.info()
    assert len(info) == h_or.nlevels
    for l in range(h_or.nlevels):
        lv = h_or.level(l)
        rp, ci, v = amg.level_csr(l)
        assert np.array_equal(rp, lv["row_ptr"]) and np.array_equal(ci, lv["col"])
        assert np.array_equal(_bits(v), _bits(lv["val"])), f"level {l} values differ"
        if l + 1 < h_or.nlevels:
            agg_or, _ = h_or.level_agg(l)
            agg_gpu, _ = amg.level_agg(l, -1)
            assert np.array_equal(agg_gpu, agg_or)
            prp, pci, pv = h_or.prolongator(l)
            grp, gci, gv = amg.prolongator(l)
            assert np.array_equal(grp, prp) and np.array_equal(gci, pci)
            assert np.array_equal(_bits(gv), _bits(pv)), f"level {l} prolongator differs"


@pytest.mark.parametrize("N,ratio,lx,cmax", [(8, 1.0, 1.0, 8), (13, 1.04, 1.0, 30), (24, 1.04, 4.0, 200),
                                             (33, 1.04, 1.0, 200)])
def test_smoothed_hierarchy_bit_exact(N, ratio, lx, cmax):
    A, _, _ = W.q1_laplacian(N, ratio, lx=lx)
    h_or = O.Hierarchy(A, coarse_max=cmax, n_pass=2, smoothed=True)
    amg = B.AMG.from_csr(A, coarse_max=cmax, smoothed=True)
    assert h_or.nlevels >= 2
    _compare(h_or, amg)
    amg.close()


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
@pytest.mark.parametrize("N,ratio", [(13, 1.04), (24, 1.04), (32, 1.0)])
def test_smoothed_solve_parity(N, ratio, mode):
    prob = W.make_problem(N, ratio, seed=21)
    h_or = O.Hierarchy(prob.A, coarse_max=200, n_pass=2, smoothed=True)
    ref = h_or.solve(prob.b, rtol=RTOL, maxit=1000, mode=mode)
    amg = B.AMG.from_csr(prob.A, mode=mode, smoothed=True)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    res = amg.solve(b, x, rtol=RTOL, maxit=1000)
    xs = x.cpu().numpy()
    assert res.status == 0, res.message
    assert abs(res.iters - ref["iters"]) <= 1, (res.iters, ref["iters"])
    assert np.linalg.norm(prob.b - W.spmv(prob.A, xs)) <= RTOL * np.linalg.norm(prob.b)
    assert np.linalg.norm(xs - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])
    # fewer iterations than with the tentative prolongator (Sec. 3.1)
    plain = O.Hierarchy(prob.A, coarse_max=200, n_pass=2).solve(prob.b, rtol=RTOL, maxit=1000, mode=mode)
    assert res.iters < plain["iters"]
    amg.close()


def test_smoothed_graph_and_stream_paths_agree():
    import os
    prob = W.make_problem(20, 1.04, seed=4)
    b = torch.from_numpy(prob.b).cuda()
    out = []
    for g in ("1", "0"):
        old = os.environ.get("PCGAMG_GRAPH")
        os.environ["PCGAMG_GRAPH"] = g
        try:
            amg = B.AMG.from_csr(prob.A, smoothed=True, mode="fcg32")
        finally:
            if old is None:
                del os.environ["PCGAMG_GRAPH"]
            else:
                os.environ["PCGAMG_GRAPH"] = old
        x = torch.zeros_like(b)
        r = amg.solve(b, x)
        assert r.status == 0
        out.append((r.iters, x))
        amg.close()
    assert out[0][0] == out[1][0] and torch.equal(out[0][1], out[1][1])


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_smoothed_with_gauss_seidel(mode):
    prob = W.make_problem(16, 1.04, seed=22)
    h_or = O.Hierarchy(prob.A, coarse_max=60, n_pass=2, smoothed=True)
    assert h_or.set_smoother(2, 97) == 0
    ref = h_or.solve(prob.b, rtol=RTOL, maxit=1000, mode=mode)
    amg = B.AMG.from_csr(prob.A, mode=mode, coarse_max=60, smoothed=True)
    amg.set_smoother(2, 97)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    res = amg.solve(b, x, rtol=RTOL)
    assert res.status == 0 and abs(res.iters - ref["iters"]) <= 1
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])
    amg.close()


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_smoothed_with_iterative_coarse(mode):
    prob = W.make_problem(40, 1.2, seed=23, lx=4.0)
    h_or = O.Hierarchy(prob.A, coarse_max=200, n_pass=2, smoothed=True, coarse="iter")
    ref = h_or.solve(prob.b, rtol=RTOL, maxit=1000, mode=mode)
    amg = B.AMG.from_csr(prob.A, mode=mode, smoothed=True, coarse="iter")
    _compare(h_or, amg)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    res = amg.solve(b, x, rtol=RTOL)
    assert res.status == 0 and abs(res.iters - ref["iters"]) <= 1
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])
    amg.close()


def test_smoothed_refresh_bit_exact():
    A, _, _ = W.q1_laplacian(20, 1.04)
    A2 = W.rescaled(A, seed=31)
    h_or = O.Hierarchy(A, coarse_max=60, n_pass=2, smoothed=True)
    amg = B.AMG.from_csr(A, coarse_max=60, smoothed=True, mode="fcg32")
    b = torch.from_numpy(W.spmv(A2, W.normals(3, A.n))).cuda()
    x0 = torch.zeros_like(b)
    amg.solve(b, x0)   # a graph captured before the refresh stays valid
    assert h_or.refresh(A2) == 0
    amg.refresh(A2)
    _compare(h_or, amg)
    ref = h_or.solve(b.cpu().numpy(), rtol=RTOL, maxit=1000, mode="fcg32")
    x = torch.zeros_like(b)
    r = amg.solve(b, x, rtol=RTOL)
    assert r.status == 0 and abs(r.iters - ref["iters"]) <= 1
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])
    amg.close()


def test_smoothed_batch_equals_single_solves():
    probs = [W.make_problem(N, 1.04, seed=60 + N) for N in (12, 18, 25)]
    amgs = [B.AMG.from_csr(p.A, mode=m, smoothed=True) for p, m in zip(probs, ("fcg32", "pcg64", "fcg32"))]
    batch = B.Batch(amgs)
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    st, it, sts = batch.solve(bs, xs, rtol=RTOL)
    assert st == 0 and list(sts) == [0, 0, 0]
    for k, a in enumerate(amgs):
        x1 = torch.zeros_like(bs[k])
        r = a.solve(bs[k], x1, rtol=RTOL)
        assert r.iters == it[k] and torch.equal(x1, xs[k]), k
    batch.close()
    for a in amgs:
        a.close()


def test_smoothed_refusals():
    prob = W.make_problem(12, 1.04, seed=2)
    amg = B.AMG.from_csr(prob.A, coarse_max=60, smoothed=True)
    X = np.zeros((prob.A.n, 4))
    st, *_ = amg.solve_multi(np.ones((prob.A.n, 4)), X)
    assert st == B.ERR_ARG
    with pytest.raises(B.AmgError):
        amg.set_level_shape(1, [4, 0, 0, 0])
    assert amg.autotune(reps=1) == 0
    with pytest.raises(B.AmgError):
        B.Server([amg], mode="fcg32")
    plain = B.AMG.from_csr(prob.A, coarse_max=60)
    with pytest.raises(B.AmgError):
        plain.prolongator(0)
    plain.close()
    amg.close()
