"""Iterative coarsest solve on the GPU (Sec. 3.1: flexible CG preconditioned
by block-Jacobi with ILU(1) blocks, stopped at a 1e-3 residual reduction or
30 iterations) against the CPU oracle, through the C ABI.

Bar: the ILU(1) factors of every 32-row block equal the oracle's bit for bit
(the same operations, each rounded on its own); the coarsest solve alone
runs the same number of inner iterations as the oracle's and agrees to
1e-9; whole solves (both modes, which then both run the flexible outer
recurrence) keep the single-solve bar: iterations within +-1, true relative
residual <= rtol and ||x - x_oracle|| <= 1e-6 ||x_oracle||. The
multi-column, batched, served and refreshed paths give the same results as
single solves. The stall-prone meshes are stretched (L_x = 4) and strongly
graded, so their coarsening stops with far more than 200 rows.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2210_16660_gb300 import binding as B  # noqa: E402
from paper_2210_16660_gb300 import serving as S  # noqa: E402
from paper_2210_16660_gb300 import workloads as W  # noqa: E402

RTOL = 1e-8
X_TOL = 1e-6

# (N, ratio, lx, coarse_max, coarse): coarsening stalls at 879 rows (forced
# iterative), at 4162 rows (above the dense limit: AUTO picks the iterative
# solve), and a small uniform case with the iterative solve forced
CASES = [(40, 1.2, 4.0, 200, "iter"), (64, 1.1, 4.0, 200, "auto"), (13, 1.04, 1.0, 50, "iter")]


def _oracle_blocks(h_or, nL):
    rp, ci, v, _ = h_or.coarse_ilu()
    nb = (nL + 31) // 32
    F = np.zeros((nb, 32, 32))
    for i in range(nL):
        b, il = divmod(i, 32)
        q = slice(rp[i], rp[i + 1])
        F[b, il, ci[q] - 32 * b] = v[q]
    return F


def _pair(N, ratio, lx, cmax, coarse, mode="pcg64", seed=1):
    prob = W.make_problem(N, ratio, seed=seed, lx=lx)
    h_or = O.Hierarchy(prob.A, coarse_max=cmax, n_pass=2, coarse=coarse)
    amg = B.AMG.from_csr(prob.A, coarse_max=cmax, coarse=coarse, mode=mode)
    return prob, h_or, amg


@pytest.mark.parametrize("N,ratio,lx,cmax,coarse", CASES)
def test_factors_bit_exact_and_inner_solve(N, ratio, lx, cmax, coarse):
    prob, h_or, amg = _pair(N, ratio, lx, cmax, coarse)
    ci = amg.coarse_info()
    nL = h_or.level_size(h_or.nlevels - 1)[0]
    assert ci["kind"] == "iter" and h_or.coarse_kind == "iter"
    assert ci["rows"] == nL and ci["blocks"] == (nL + 31) // 32
    assert len(amg.info()) == h_or.nlevels
    F = amg.coarse_factors()
    assert np.array_equal(F.view(np.int64), _oracle_blocks(h_or, nL).view(np.int64))
    rng = np.random.default_rng(N)
    for trial in range(3):
        bL = rng.standard_normal(nL)
        if trial == 2:
            bL[:] = 0.0  # b = 0: x = 0 without iterating
        xo, itso = h_or.coarse_solve(bL)
        xg = torch.full((nL,), 7.0, dtype=torch.float64, device="cuda")
        itsg = amg.coarse_solve(torch.from_numpy(bL).cuda(), xg)
        xg = xg.cpu().numpy()
        assert itsg == itso
        if trial == 2:
            assert itsg == 0 and not xg.any()
        else:
            assert 1 <= itsg <= 30
            assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)
    # host vectors take the same route
    xh = np.zeros(nL)
    assert amg.coarse_solve(bL.copy(), xh) == itso
    amg.close()


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
@pytest.mark.parametrize("N,ratio,lx,cmax,coarse", CASES)
def test_solve_parity_with_iterative_coarse(N, ratio, lx, cmax, coarse, mode):
    prob, h_or, amg = _pair(N, ratio, lx, cmax, coarse, mode=mode)
    ref = h_or.solve(prob.b, rtol=RTOL, maxit=1000, mode=mode)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    res = amg.solve(b, x, rtol=RTOL, maxit=1000)
    xs = x.cpu().numpy()
    assert res.status == 0, res.message
    assert abs(res.iters - ref["iters"]) <= 1, (res.iters, ref["iters"])
    true_rel = np.linalg.norm(prob.b - W.spmv(prob.A, xs)) / np.linalg.norm(prob.b)
    assert true_rel <= RTOL
    assert np.linalg.norm(xs - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])
    # the same solve again gives the same bits (deterministic reductions)
    x2 = torch.zeros_like(b)
    res2 = amg.solve(b, x2, rtol=RTOL, maxit=1000)
    assert res2.iters == res.iters and torch.equal(x, x2)
    amg.close()


def test_graph_and_stream_paths_agree_with_iterative_coarse():
    import os
    prob = W.make_problem(40, 1.2, seed=2, lx=4.0)
    b = torch.from_numpy(prob.b).cuda()
    out = []
    for g in ("1", "0"):
        old = os.environ.get("PCGAMG_GRAPH")
        os.environ["PCGAMG_GRAPH"] = g
        try:
            amg = B.AMG.from_csr(prob.A, coarse="iter", mode="fcg32")
        finally:
            if old is None:
                del os.environ["PCGAMG_GRAPH"]
            else:
                os.environ["PCGAMG_GRAPH"] = old
        x = torch.zeros_like(b)
        r = amg.solve(b, x)
        assert r.status == 0
        out.append((r.iters, x, r.hist))
        amg.close()
    assert out[0][0] == out[1][0] and torch.equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_multi_columns_with_iterative_coarse(mode):
    prob, h_or, amg = _pair(40, 1.2, 4.0, 200, "iter", mode=mode, seed=3)
    Bm, _ = W.make_rhs(prob, 5, seed=77)
    Bm = np.ascontiguousarray(Bm)
    X = torch.zeros((prob.A.n, 5), dtype=torch.float64, device="cuda")
    st, it, _, sts, tr = amg.solve_multi(torch.from_numpy(Bm).cuda(), X, rtol=RTOL)
    assert st == 0 and np.all(sts == 0) and np.all(tr <= RTOL)
    Xh = X.cpu().numpy()
    for c in (0, 4):
        ref = h_or.solve(Bm[:, c].copy(), rtol=RTOL, maxit=1000, mode=mode)
        assert abs(int(it[c]) - ref["iters"]) <= 1
        assert np.linalg.norm(Xh[:, c] - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])
        b1 = torch.from_numpy(Bm[:, c].copy()).cuda()
        x1 = torch.zeros_like(b1)
        r1 = amg.solve(b1, x1, rtol=RTOL)
        assert abs(r1.iters - int(it[c])) <= 1
        assert (x1 - X[:, c]).norm().item() <= X_TOL * x1.norm().item()
    amg.close()


def test_batch_with_iterative_coarse_equals_single_solves():
    probs = [W.make_problem(N, r, seed=50 + N, lx=lx) for N, r, lx in ((40, 1.2, 4.0), (20, 1.04, 1.0), (36, 1.2, 4.0))]
    amgs = [B.AMG.from_csr(p.A, mode=m, coarse=c)
            for p, m, c in zip(probs, ("fcg32", "pcg64", "pcg64"), ("iter", "auto", "iter"))]
    assert [a.coarse_info()["kind"] for a in amgs] == ["iter", "dense", "iter"]
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


@pytest.mark.parametrize("solo", [False, True])
def test_serving_with_iterative_coarse(solo):
    """A served request gives the same bits alone and in a mix, on meshes
    whose hierarchies use the iterative coarsest solve."""
    meshes = S.prepare_meshes((20, 24), ratio=1.2, seed=61, pool=2, lx=4.0, coarse="iter", coarse_max=40)
    assert all(m.amg.coarse_info()["kind"] == "iter" for m in meshes)
    srv = S.make_server(meshes, "fcg32", slots=4, max_engines=1, chunk=3, solo=solo)
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
    assert all(res[t].status == B.OK and res[t].true_rel <= RTOL for t in tickets)
    # alone in the same kind of place: an engine slot of a server without
    # lanes, or pcg_solve for a request that ran in a whole-solve lane
    alone = S.make_server(meshes, "fcg32", slots=4, max_engines=1, chunk=3, solo=False)
    for j in range(len(reqs)):
        m, k = reqs[j]
        b, x0 = meshes[m].steps[k]
        r = res[tickets[j]]
        if r.lane == 1:
            xa = torch.empty_like(b)
            st, t = alone.submit(m, b, x0, xa)
            ra = alone.drain([t])[t]
        else:
            xa = x0.clone()
            ra = meshes[m].amg.solve(b, xa, rtol=RTOL, hist=False)
        assert torch.equal(xa, xs[j]) and ra.iters == r.iters, (j, r.lane)
        if j not in (0, 3):
            continue
        ref = O.Hierarchy(meshes[m].problem.A, coarse_max=40, n_pass=2, coarse="iter").solve(
            b.cpu().numpy(), x0=x0.cpu().numpy(), rtol=RTOL, maxit=1000, mode="fcg32")
        assert abs(ref["iters"] - ra.iters) <= 1
        assert np.linalg.norm(xa.cpu().numpy() - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])
    alone.close()
    srv.close()
    for mm in meshes:
        mm.amg.close()


def test_refresh_rebuilds_the_factors_bit_exact():
    A, _, _ = W.q1_laplacian(40, 1.2, lx=4.0)
    A2 = W.rescaled(A, seed=9)
    h_or = O.Hierarchy(A, coarse_max=200, n_pass=2, coarse="iter")
    amg = B.AMG.from_csr(A, coarse="iter", mode="fcg32")
    nL = h_or.level_size(h_or.nlevels - 1)[0]
    assert h_or.refresh(A2) == 0
    amg.refresh(A2)
    assert np.array_equal(amg.coarse_factors().view(np.int64), _oracle_blocks(h_or, nL).view(np.int64))
    b = W.spmv(A2, W.normals(5, A.n))
    ref = h_or.solve(b, rtol=RTOL, maxit=1000, mode="fcg32")
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = amg.solve(torch.from_numpy(b).cuda(), x, rtol=RTOL)
    assert r.status == 0 and abs(r.iters - ref["iters"]) <= 1
    assert np.linalg.norm(x.cpu().numpy() - ref["x"]) <= X_TOL * np.linalg.norm(ref["x"])
    amg.close()


def test_iterative_coarse_arguments():
    A, _, _ = W.q1_laplacian(12, 1.04)
    # a single level cannot use the iterative solve
    with pytest.raises(B.AmgError) as e:
        B.AMG.from_csr(A, coarse_max=5000, coarse="iter")
    assert e.value.status == B.ERR_ARG
    # the dense solve refuses a coarsest level above 4096 rows
    Bm, _, _ = W.q1_laplacian(64, 1.1, lx=4.0)
    with pytest.raises(B.AmgError) as e:
        B.AMG.from_csr(Bm, coarse="dense")
    assert e.value.status == B.ERR_COARSE
    amg = B.AMG.from_csr(A, coarse_max=60)
    assert amg.coarse_info()["kind"] == "dense"
    with pytest.raises(B.AmgError):
        amg.coarse_factors()
    amg.close()
    with pytest.raises(B.AmgError):
        B.AMG.from_csr(A, coarse_max=60, coarse="iter", coarse_maxit=1001)
