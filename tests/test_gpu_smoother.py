"""Hybrid Gauss-Seidel smoothing (amg_set_smoother; Sec. 3.1, nu sweeps of
block Jacobi with forward/backward Gauss-Seidel inside each row block) on the
GPU, against the oracle's same smoother.

Bar: with one row per block and one sweep the solve equals the l1-Jacobi
default bit for bit; otherwise iterations within +-1 of the oracle, true
residual <= rtol and ||x - x_oracle|| / ||x_oracle|| <= 1e-6, in both modes,
on ragged block sizes; and at full size (128^3, nu = 4) a converged solve in
fewer iterations than the default.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2210_16660_gb300 import binding as B  # noqa: E402
from paper_2210_16660_gb300 import workloads as W  # noqa: E402

RTOL = 1e-8
X_TOL = 1e-6


def _solve(amg, b):
    x = torch.zeros_like(b)
    r = amg.solve(b, x, rtol=RTOL, maxit=1000)
    return r, x


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_one_row_one_sweep_equals_the_default(mode):
    prob = W.make_problem(30, 1.04, seed=3)
    b = torch.from_numpy(prob.b).cuda()
    a1 = B.AMG.from_csr(prob.A, mode=mode)
    a2 = B.AMG.from_csr(prob.A, mode=mode)
    a2.set_smoother(1, 0)
    r1, x1 = _solve(a1, b)
    r2, x2 = _solve(a2, b)
    assert r1.status == r2.status == 0 and r1.iters == r2.iters
    assert torch.equal(x1, x2)
    a2.set_smoother(0)                     # back to the default sweeps
    r3, x3 = _solve(a2, b)
    assert r3.iters == r1.iters and torch.equal(x3, x1)


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
@pytest.mark.parametrize("nu,nblocks", [(1, 97), (4, 97), (2, 1000)])
def test_hybrid_gs_parity(mode, nu, nblocks):
    prob = W.make_problem(26, 1.04, seed=4)
    h_or = O.Hierarchy(prob.A, coarse_max=200, n_pass=2)
    assert h_or.set_smoother(nu, nblocks) == O.OK
    ref = h_or.solve(prob.b, rtol=RTOL, maxit=1000, mode=mode)
    amg = B.AMG.from_csr(prob.A, mode=mode)
    amg.set_smoother(nu, nblocks)
    b = torch.from_numpy(prob.b).cuda()
    res, x = _solve(amg, b)
    assert res.status == 0, res.message
    assert abs(res.iters - ref["iters"]) <= 1, (res.iters, ref["iters"])
    xs = x.cpu().numpy()
    assert np.linalg.norm(prob.b - W.spmv(prob.A, xs)) <= RTOL * np.linalg.norm(prob.b)
    assert np.linalg.norm(xs - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
@pytest.mark.parametrize("nu,rows_per_block", [(1, 32), (4, 32), (2, 8), (4, 4)])
def test_one_launch_warp_sweeps(mode, nu, rows_per_block):
    """Blocks whose size divides the 32-row slice sweep in one launch per
    sweep (one warp per slice); the two-launch sweeps (PCGAMG_GS_FUSED=0) and
    the oracle agree with it within the solve bar."""
    prob = W.make_problem(24, 1.04, seed=8)
    nblocks = prob.A.n // rows_per_block
    h_or = O.Hierarchy(prob.A, coarse_max=200, n_pass=2)
    assert h_or.set_smoother(nu, nblocks) == O.OK
    ref = h_or.solve(prob.b, rtol=RTOL, maxit=1000, mode=mode)
    b = torch.from_numpy(prob.b).cuda()
    out = []
    for fused in ("1", "0"):
        old = os.environ.get("PCGAMG_GS_FUSED")
        os.environ["PCGAMG_GS_FUSED"] = fused
        try:
            amg = B.AMG.from_csr(prob.A, mode=mode)
        finally:
            if old is None:
                del os.environ["PCGAMG_GS_FUSED"]
            else:
                os.environ["PCGAMG_GS_FUSED"] = old
        amg.set_smoother(nu, nblocks)
        res, x = _solve(amg, b)
        assert res.status == 0, res.message
        assert abs(res.iters - ref["iters"]) <= 1, (fused, res.iters, ref["iters"])
        xs = x.cpu().numpy()
        assert np.linalg.norm(xs - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])
        out.append((res, x))
        amg.close()
    assert abs(out[0][0].iters - out[1][0].iters) <= 1
    assert (out[0][1] - out[1][1]).norm().item() <= X_TOL * out[1][1].norm().item()


def test_graph_and_stream_paths_agree_with_gauss_seidel():
    prob = W.make_problem(28, 1.04, seed=5)
    b = torch.from_numpy(prob.b).cuda()
    a1 = B.AMG.from_csr(prob.A, mode="fcg32")
    os.environ["PCGAMG_GRAPH"] = "0"
    try:
        a2 = B.AMG.from_csr(prob.A, mode="fcg32")
    finally:
        del os.environ["PCGAMG_GRAPH"]
    for a in (a1, a2):
        a.set_smoother(4, 500)
    r1, x1 = _solve(a1, b)
    r2, x2 = _solve(a2, b)
    assert r1.status == r2.status == 0 and r1.iters == r2.iters
    assert torch.equal(x1, x2)


def test_gauss_seidel_handles_are_refused_where_only_jacobi_kernels_exist():
    prob = W.make_problem(14, 1.04, seed=6)
    amg = B.AMG.from_csr(prob.A, mode="fcg32")
    amg.set_smoother(2, 50)
    Bm = torch.from_numpy(np.stack([prob.b, prob.b], 1)).cuda()
    st = amg.solve_multi(Bm, torch.zeros_like(Bm), rtol=RTOL)[0]
    assert st == B.ERR_ARG
    assert amg.autotune(reps=2) == 0
    with pytest.raises(B.AmgError):
        amg.set_smoother(-1, 0)


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_multi_column_gauss_seidel(mode):
    """pcg_solve_multi with nu = 4 over blocks that divide the 32-row slices:
    each column within the solve bar of the same single-column solve and of
    the oracle."""
    prob = W.make_problem(24, 1.04, seed=9)
    nblocks = prob.A.n // 32
    amg = B.AMG.from_csr(prob.A, mode=mode)
    amg.set_smoother(4, nblocks)
    Bm, _ = W.make_rhs(prob, 5, seed=91)
    Bm = np.ascontiguousarray(Bm)
    X = torch.zeros((prob.A.n, 5), dtype=torch.float64, device="cuda")
    st, it, _, sts, tr = amg.solve_multi(torch.from_numpy(Bm).cuda(), X, rtol=RTOL)
    assert st == 0 and np.all(sts == 0) and np.all(tr <= RTOL)
    h_or = O.Hierarchy(prob.A, coarse_max=200, n_pass=2)
    assert h_or.set_smoother(4, nblocks) == O.OK
    for c in (0, 4):
        b1 = torch.from_numpy(Bm[:, c].copy()).cuda()
        r1, x1 = _solve(amg, b1)
        assert abs(r1.iters - int(it[c])) <= 1
        assert (x1 - X[:, c]).norm().item() <= X_TOL * x1.norm().item()
        ref = h_or.solve(Bm[:, c].copy(), rtol=RTOL, maxit=1000, mode=mode)
        assert abs(int(it[c]) - ref["iters"]) <= 1
        assert np.linalg.norm(X[:, c].cpu().numpy() - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])
    amg.close()


def test_served_gauss_seidel():
    """A server whose meshes smooth by nu = 4 Gauss-Seidel: every request
    meets rtol and matches its mesh's own pcg_solve within the solve bar."""
    from paper_2210_16660_gb300 import serving as S
    meshes = S.prepare_meshes((16, 20), ratio=1.04, seed=41, pool=2)
    for m in meshes:
        m.amg.set_smoother(4, m.problem.A.n // 32)
    srv = S.make_server(meshes, "fcg32", slots=4, max_engines=1, chunk=3, solo=False)
    reqs = [(i % 2, (i // 2) % 2) for i in range(8)]
    xs, tickets = [], []
    for m, k in reqs:
        b, x0 = meshes[m].steps[k]
        x = torch.empty_like(b)
        st, t = srv.submit(m, b, x0, x)
        assert st == B.OK
        xs.append(x)
        tickets.append(t)
    res = srv.drain(tickets)
    for j, (m, k) in enumerate(reqs):
        r = res[tickets[j]]
        assert r.status == B.OK and r.true_rel <= RTOL and r.lane == 1
        b, x0 = meshes[m].steps[k]
        x1 = x0.clone()
        r1 = meshes[m].amg.solve(b, x1, rtol=RTOL, hist=False)
        assert abs(r1.iters - r.iters) <= 1
        assert (x1 - xs[j]).norm().item() <= X_TOL * x1.norm().item()
    srv.close()
    for mm in meshes:
        mm.amg.close()


def test_batch_with_gauss_seidel_equals_single_solves():
    """Batches capture each system's own V-cycle, Gauss-Seidel sweeps included;
    a smoother set after the batch was created is picked up."""
    probs = [W.make_problem(N, 1.04, seed=70 + N) for N in (12, 20, 17)]
    amgs = [B.AMG.from_csr(p.A, mode=m) for p, m in zip(probs, ("fcg32", "pcg64", "fcg32"))]
    batch = B.Batch(amgs)
    amgs[0].set_smoother(4, 0)
    amgs[1].set_smoother(2, probs[1].A.n // 32)
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


def test_refresh_with_gauss_seidel_matches_the_oracle():
    old = W.make_problem(24, 1.04, seed=7)
    A2 = W.rescaled(old.A, seed=8)
    b2 = W.spmv(A2, W.normals(9, A2.n))
    h_or = O.Hierarchy(old.A, coarse_max=200, n_pass=2)
    assert h_or.set_smoother(4, 64) == O.OK
    assert h_or.refresh(A2) == O.OK
    ref = h_or.solve(b2, rtol=RTOL, maxit=1000, mode="pcg64")
    amg = B.AMG.from_csr(old.A, mode="pcg64")
    amg.set_smoother(4, 64)
    amg.refresh(A2)
    res, x = _solve(amg, torch.from_numpy(b2).cuda())
    assert res.status == 0 and abs(res.iters - ref["iters"]) <= 1
    xs = x.cpu().numpy()
    assert np.linalg.norm(xs - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])


def test_back_to_jacobi_after_a_refresh_under_gauss_seidel():
    """A refresh while Gauss-Seidel is active re-forms the cluster tail's image
    with the Gauss-Seidel diagonals; returning to the default must re-form it
    with the l1-Jacobi ones (same bits as a handle refreshed under Jacobi)."""
    prob = W.make_problem(48, 1.04, seed=19)
    A2 = W.rescaled(prob.A, seed=20)
    b = torch.from_numpy(W.spmv(A2, W.normals(21, A2.n))).cuda()
    a1 = B.AMG.from_csr(prob.A, mode="fcg32")
    a1.set_smoother(2, 4096)
    a1.refresh(A2)
    a1.set_smoother(0)
    a2 = B.AMG.from_csr(prob.A, mode="fcg32")
    a2.refresh(A2)
    r1, x1 = _solve(a1, b)
    r2, x2 = _solve(a2, b)
    assert r1.status == r2.status == 0 and r1.iters == r2.iters
    assert torch.equal(x1, x2)


def test_full_size_128_nu4():
    """The paper's nu = 4 on the benchmarked system, 65,536 row blocks per
    level (32 rows per block on level 0)."""
    prob = W.make_problem(128, 1.04, seed=2)
    b = torch.from_numpy(prob.b).cuda()
    amg = B.AMG.from_csr(prob.A, mode="fcg32")
    r0, _ = _solve(amg, b)
    amg.set_smoother(4, 65536)
    r, x = _solve(amg, b)
    assert r.status == 0 and r.true_rel <= RTOL
    xs = x.cpu().numpy()
    assert np.linalg.norm(prob.b - W.spmv(prob.A, xs)) <= RTOL * np.linalg.norm(prob.b)
    assert r.iters < r0.iters
