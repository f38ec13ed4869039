"""The entry point that allocates no device memory (amg_residual_noalloc).

It serves callers that cannot allocate device memory while they solve (an
application that owns the whole GPU through its own pool, or a loop that
cannot take an allocation's device synchronisation). Checked against the
library's own true residual after a solve (amg_last_true_residual) and the
residual vector formed on the host, on two calls in a row, since every call
reuses the same fixed scratch array. Kept in its own file so pytest runs it
after every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2210_16660_gb300 import binding as B  # noqa: E402
from paper_2210_16660_gb300 import workloads as W  # noqa: E402


@pytest.mark.parametrize("N,col16", [(24, True), (33, False)])
def test_residual_noalloc_matches_solver(N, col16):
    import os
    if not col16:
        os.environ["PCGAMG_COL16"] = "0"
    try:
        prob = W.make_problem(N, 1.04, seed=12)
        amg = B.AMG.from_csr(prob.A, mode="fcg32")
    finally:
        os.environ.pop("PCGAMG_COL16", None)
    assert amg.level_layout(0)["index_bytes"] == (2 if col16 else 4)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    res = amg.solve(b, x, rtol=1e-8)
    assert res.status == 0
    # the existing entry point's answer: ||b - A x|| / ||b|| of the final x
    ref_rel = res.true_rel
    r_host = prob.b - W.spmv(prob.A, x.cpu().numpy())
    outs = []
    for _ in range(2):
        r = torch.full_like(b, np.nan)
        rn, bn = amg.residual_noalloc(b, x, r)
        torch.cuda.synchronize()
        assert bn == pytest.approx(np.linalg.norm(prob.b), rel=1e-12)
        assert rn / bn == pytest.approx(ref_rel, rel=1e-9)
        rv = r.cpu().numpy()
        assert np.all(np.isfinite(rv))
        assert np.linalg.norm(rv - r_host) <= 1e-6 * np.linalg.norm(r_host)
        outs.append((rn, bn, rv))
    # the shared scratch gives the same result on the second call
    assert outs[0][0] == outs[1][0] and outs[0][1] == outs[1][1]
    assert np.array_equal(outs[0][2], outs[1][2])


def test_residual_noalloc_rejects_host_vectors():
    prob = W.make_problem(8, 1.0, seed=1)
    amg = B.AMG.from_csr(prob.A)
    b = prob.b.copy()
    with pytest.raises(B.AmgError) as e:
        amg.residual_noalloc(b, np.zeros_like(b), np.zeros_like(b))
    assert e.value.status == B.ERR_ARG
