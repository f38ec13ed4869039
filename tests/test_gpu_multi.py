"""Multi right-hand-side solves (pcg_solve_multi) against the oracle, per column.

Each column must meet the same bar as a single solve: iterations within +-1
of the oracle's, true relative residual <= rtol, and
||x_c - x_oracle,c|| / ||x_oracle,c|| <= 1e-6; columns that start converged,
have b = 0 or run out of iterations behave as the single path does.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2210_16660_gb300 import binding as B  # noqa: E402
from paper_2210_16660_gb300 import workloads as W  # noqa: E402

RTOL = 1e-8


def _rhs(prob, k, seed):
    Bm, Xs = W.make_rhs(prob, k, seed)
    return np.ascontiguousarray(Bm), Xs


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
@pytest.mark.parametrize("N,k", [(20, 3), (24, 8)])
def test_multi_matches_oracle_per_column(mode, N, k):
    prob = W.make_problem(N, 1.04, seed=21)
    Bm, _ = _rhs(prob, k, 300 + N)
    h_or = O.Hierarchy(prob.A, n_pass=2)
    amg = B.AMG.from_csr(prob.A, mode=mode)
    X = torch.zeros((prob.A.n, k), dtype=torch.float64, device="cuda")
    st, it, hist, sts, tr = amg.solve_multi(torch.from_numpy(Bm).cuda(), X, rtol=RTOL)
    assert st == 0 and np.all(sts == 0)
    Xh = X.cpu().numpy()
    for c in range(k):
        ref = h_or.solve(Bm[:, c], rtol=RTOL, maxit=1000, mode=mode)
        assert abs(int(it[c]) - ref["iters"]) <= 1, (c, it[c], ref["iters"])
        xc = Xh[:, c]
        rel = np.linalg.norm(Bm[:, c] - W.spmv(prob.A, xc)) / np.linalg.norm(Bm[:, c])
        assert rel <= RTOL and tr[c] <= RTOL
        assert np.linalg.norm(xc - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])
        assert hist[c, 0] == pytest.approx(1.0) and hist[c, it[c]] <= RTOL


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_multi_agrees_with_single_solves(mode):
    prob = W.make_problem(26, 1.04, seed=22)
    k = 5
    Bm, _ = _rhs(prob, k, 401)
    amg = B.AMG.from_csr(prob.A, mode=mode)
    X = torch.zeros((prob.A.n, k), dtype=torch.float64, device="cuda")
    st, it, _, _, _ = amg.solve_multi(torch.from_numpy(Bm).cuda(), X, rtol=RTOL)
    assert st == 0
    for c in range(k):
        b = torch.from_numpy(Bm[:, c].copy()).cuda()
        x = torch.zeros_like(b)
        r = amg.solve(b, x, rtol=RTOL)
        assert abs(r.iters - int(it[c])) <= 1
        d = (x - X[:, c]).norm().item() / x.norm().item()
        assert d <= 1e-6, (c, d)


def test_multi_column_states():
    """b = 0, a converged start, and ordinary columns in one call."""
    prob = W.make_problem(16, 1.04, seed=23)
    k = 4
    Bm, _ = _rhs(prob, k, 501)
    Bm[:, 0] = 0.0
    x_exact = np.linalg.solve(prob.A.to_dense(), Bm[:, 1])
    X0 = np.zeros((prob.A.n, k))
    X0[:, 0] = 1.0                       # must come back as zeros
    X0[:, 1] = x_exact
    amg = B.AMG.from_csr(prob.A, mode="fcg32")
    X = np.ascontiguousarray(X0)         # host buffers this time
    st, it, hist, sts, tr = amg.solve_multi(np.ascontiguousarray(Bm), X, rtol=RTOL)
    assert st == 0 and list(sts) == [0] * k
    assert it[0] == 0 and not X[:, 0].any()
    assert it[1] == 0 and np.allclose(X[:, 1], x_exact)
    assert it[2] > 0 and it[3] > 0
    for c in (2, 3):
        rel = np.linalg.norm(Bm[:, c] - W.spmv(prob.A, X[:, c])) / np.linalg.norm(Bm[:, c])
        assert rel <= RTOL


def test_multi_maxit_and_padding():
    prob = W.make_problem(14, 1.04, seed=24)
    k = 6                                 # runs as 8 columns internally
    Bm, _ = _rhs(prob, k, 601)
    amg = B.AMG.from_csr(prob.A)
    X = torch.zeros((prob.A.n, k), dtype=torch.float64, device="cuda")
    st, it, _, sts, _ = amg.solve_multi(torch.from_numpy(Bm).cuda(), X, rtol=1e-15, maxit=3)
    assert st == B.ERR_NOCONV and list(sts) == [B.ERR_NOCONV] * k and list(it) == [3] * k


def test_multi_32_columns_deterministic():
    prob = W.make_problem(16, 1.04, seed=25)
    k = 32
    Bm, _ = _rhs(prob, k, 701)
    amg = B.AMG.from_csr(prob.A, mode="fcg32")
    outs = []
    for _ in range(2):
        X = torch.zeros((prob.A.n, k), dtype=torch.float64, device="cuda")
        st, it, _, sts, tr = amg.solve_multi(torch.from_numpy(Bm).cuda(), X, rtol=RTOL)
        assert st == 0 and np.all(tr <= RTOL)
        outs.append(X.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_multi_rejects_bad_k():
    prob = W.make_problem(10, 1.0, seed=1)
    amg = B.AMG.from_csr(prob.A)
    X = np.zeros((prob.A.n, 33))
    st, *_ = amg.solve_multi(np.ones((prob.A.n, 33)), X)
    assert st == B.ERR_ARG


def test_full_size_320_eight_rhs():
    """The large single mesh as stated: 320^3 nodes (32.8M dofs, 876M stored
    entries), z graded at ratio 1.02 with a 4:1 x-stretch, 8 right-hand sides
    in one multi-column solve. Its coarsening stalls far above the dense
    limit, so the iterative coarsest solve runs. Every column meets rtol by
    the host's own residual, and a column solved alone (single-column
    kernels) agrees to 1e-6."""
    N = 320
    prob = W.make_problem(N, 1.02, seed=6, lx=4.0)
    Bm, _ = W.make_rhs(prob, 8, seed=1006)
    Bm = np.ascontiguousarray(Bm)
    amg = B.AMG.from_csr(prob.A, mode="fcg32")
    assert amg.coarse_info()["kind"] == "iter"
    X = torch.zeros((prob.A.n, 8), dtype=torch.float64, device="cuda")
    st, it, _, sts, tr = amg.solve_multi(torch.from_numpy(Bm).cuda(), X, rtol=RTOL, hist=False)
    assert st == 0 and np.all(sts == 0) and np.all(tr <= RTOL)
    Xh = X.cpu().numpy()
    for c in (0, 7):
        b = Bm[:, c]
        assert np.linalg.norm(b - W.spmv(prob.A, Xh[:, c])) <= RTOL * np.linalg.norm(b)
    b0 = torch.from_numpy(Bm[:, 0].copy()).cuda()
    x0 = torch.zeros_like(b0)
    r = amg.solve(b0, x0, hist=False)
    assert r.status == 0 and abs(r.iters - int(it[0])) <= 1
    assert (x0 - X[:, 0]).norm().item() <= 1e-6 * x0.norm().item()
    amg.close()


def test_full_size_160_thirty_two_rhs():
    """The benchmark's multi-column case: 32 right-hand sides of the 160^3
    mesh (4.1M dofs, z graded at 1.04, whose coarsening stalls above the
    dense limit: iterative coarsest solve) in one call. Every column meets
    rtol (library and, for two columns, the host's own residual) and a
    column solved alone agrees to 1e-6."""
    N = 160
    prob = W.make_problem(N, 1.04, seed=4)
    Bm, _ = W.make_rhs(prob, 32, seed=2002)
    Bm = np.ascontiguousarray(Bm)
    amg = B.AMG.from_csr(prob.A, mode="fcg32")
    X = torch.zeros((prob.A.n, 32), dtype=torch.float64, device="cuda")
    st, it, _, sts, tr = amg.solve_multi(torch.from_numpy(Bm).cuda(), X, rtol=RTOL, maxit=500, hist=False)
    assert st == 0 and np.all(sts == 0) and np.all(tr <= RTOL)
    Xh = X.cpu().numpy()
    for c in (0, 31):
        b = Bm[:, c]
        assert np.linalg.norm(b - W.spmv(prob.A, Xh[:, c])) <= RTOL * np.linalg.norm(b)
    b0 = torch.from_numpy(Bm[:, 31].copy()).cuda()
    x0 = torch.zeros_like(b0)
    r = amg.solve(b0, x0, rtol=RTOL, maxit=500, hist=False)
    assert r.status == 0 and abs(r.iters - int(it[31])) <= 1
    assert (x0 - X[:, 31]).norm().item() <= 1e-6 * x0.norm().item()
    amg.close()
