"""Batched solves of independent systems (pcg_solve_batch) in one launch.

Each system keeps its own hierarchy and mode; its batched result must equal
its own pcg_solve bit for bit (same kernels), and meet the oracle's bar.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2210_16660_gb300 import binding as B  # noqa: E402
from paper_2210_16660_gb300 import workloads as W  # noqa: E402

RTOL = 1e-8


def _systems(sizes, modes):
    probs = [W.make_problem(N, 1.04, seed=40 + k) for k, N in enumerate(sizes)]
    amgs = [B.AMG.from_csr(p.A, mode=m) for p, m in zip(probs, modes)]
    return probs, amgs


def test_batch_equals_single_solves_and_oracle():
    sizes = [8, 13, 17, 22, 29, 35]
    modes = ["fcg32", "pcg64", "fcg32", "fcg32", "pcg64", "fcg32"]
    probs, amgs = _systems(sizes, modes)
    batch = B.Batch(amgs)
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    st, it, sts = batch.solve(bs, xs, rtol=RTOL)
    assert st == 0 and list(sts) == [0] * len(sizes)
    for k, (p, a, m) in enumerate(zip(probs, amgs, modes)):
        x1 = torch.zeros_like(bs[k])
        r = a.solve(bs[k], x1, rtol=RTOL)
        assert r.iters == it[k]
        assert torch.equal(x1, xs[k]), k
        if k in (1, 3, 5):
            ref = O.Hierarchy(p.A, n_pass=2).solve(p.b, rtol=RTOL, maxit=1000, mode=m)
            xh = xs[k].cpu().numpy()
            assert abs(ref["iters"] - int(it[k])) <= 1
            assert np.linalg.norm(xh - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])
    # a second call reuses the graph and gives the same answers
    xs2 = [torch.zeros_like(b) for b in bs]
    st2, it2, _ = batch.solve(bs, xs2, rtol=RTOL)
    assert st2 == 0 and list(it2) == list(it)
    assert all(torch.equal(a, b) for a, b in zip(xs, xs2))
    batch.close()


def test_batch_mixed_outcomes_and_host_vectors():
    probs, amgs = _systems([10, 16, 12], ["fcg32", "fcg32", "pcg64"])
    batch = B.Batch(amgs)
    bs = [p.b.copy() for p in probs]
    bs[1][:] = 0.0                       # b = 0 -> x = 0, no iterations
    xs = [np.ones_like(b) for b in bs]
    st, it, sts = batch.solve(bs, xs, rtol=RTOL, maxit=500)
    assert st == 0 and list(sts) == [0, 0, 0]
    assert it[1] == 0 and not xs[1].any()
    for k in (0, 2):
        rel = np.linalg.norm(probs[k].b - W.spmv(probs[k].A, xs[k])) / np.linalg.norm(probs[k].b)
        assert rel <= RTOL
    # maxit exhausted in every system
    xs = [np.zeros_like(b) for b in bs]
    st, it, sts = batch.solve([p.b.copy() for p in probs], xs, rtol=1e-15, maxit=2)
    assert st == B.ERR_NOCONV and list(sts) == [B.ERR_NOCONV] * 3 and list(it) == [2, 2, 2]


def test_batch_rejects_duplicate_handles():
    probs, amgs = _systems([9], ["fcg32"])
    with pytest.raises(B.AmgError):
        B.Batch([amgs[0], amgs[0]])


def test_full_size_48_systems():
    """The benchmark's batch: 48 graded systems of 24^3..112^3 nodes (23.0M
    dofs) in one launch. Every system meets rtol by the host's own residual,
    equals its own pcg_solve bit for bit, and the three smallest agree with
    the oracle."""
    sizes = W.batch_sizes(48, 24, 112, seed=3)
    probs = [W.make_problem(Nn, 1.04, seed=3000 + k) for k, Nn in enumerate(sizes)]
    amgs = [B.AMG.from_csr(p.A, mode="fcg32") for p in probs]
    batch = B.Batch(amgs)
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    xs = [torch.zeros_like(b) for b in bs]
    st, it, sts = batch.solve(bs, xs, rtol=RTOL, maxit=500)
    assert st == 0 and list(sts) == [0] * 48
    smallest = sorted(range(48), key=lambda k: sizes[k])[:3]
    for k, p in enumerate(probs):
        xh = xs[k].cpu().numpy()
        assert np.linalg.norm(p.b - W.spmv(p.A, xh)) <= RTOL * np.linalg.norm(p.b), k
        x1 = torch.zeros_like(bs[k])
        r = amgs[k].solve(bs[k], x1, rtol=RTOL, maxit=500, hist=False)
        assert r.iters == it[k] and torch.equal(x1, xs[k]), k
        if k in smallest:
            ref = O.Hierarchy(p.A, n_pass=2).solve(p.b, rtol=RTOL, maxit=1000, mode="fcg32")
            assert abs(ref["iters"] - int(it[k])) <= 1
            assert np.linalg.norm(xh - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])
    batch.close()
