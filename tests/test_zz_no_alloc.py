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


def _counting_allocator():
    """An allocator hook for the library that refuses every request and
    counts calls: any allocation inside a call would make it fail."""
    import ctypes as C
    calls = {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, ctx):
        calls["alloc"] += 1
        return None

    def _free(ptr, stream, ctx):
        calls["free"] += 1

    refs = (B.ALLOC_FN(_alloc), B.FREE_FN(_free))
    lib = B.load()
    assert lib.amg_set_allocator(C.cast(refs[0], C.c_void_p), C.cast(refs[1], C.c_void_p), None) == B.OK
    return calls, refs


def test_residual_noalloc_allocates_nothing():
    """With an allocator hook that refuses every request installed, two calls
    succeed and the hook is never called; the device's free memory is the
    same before and after them (measured after a first call, which may load
    the library's device code)."""
    prob = W.make_problem(20, 1.04, seed=13)
    amg = B.AMG.from_csr(prob.A, mode="pcg64")
    b = torch.from_numpy(prob.b).cuda()
    x = torch.from_numpy(prob.x_star * 0.999).cuda()
    r = torch.empty_like(b)
    norms_dev = torch.empty(2, dtype=torch.float64, device="cuda")
    ref = amg.residual_noalloc(b, x, r)
    torch.cuda.synchronize()
    lib = B.load()
    calls, refs = _counting_allocator()
    try:
        free0 = torch.cuda.mem_get_info()[0]
        outs = []
        for _ in range(2):
            st = lib.amg_residual_noalloc(amg._h, b.data_ptr(), x.data_ptr(), r.data_ptr(), norms_dev.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream or None)
            assert st == B.OK, B.last_error()
            torch.cuda.synchronize()
            outs.append(norms_dev.clone())
        free1 = torch.cuda.mem_get_info()[0]
    finally:
        lib.amg_set_allocator(None, None, None)
    assert calls == {"alloc": 0, "free": 0}
    assert free1 == free0
    assert torch.equal(outs[0], outs[1])
    assert outs[0][0].item() == ref[0] and outs[0][1].item() == ref[1]
    amg.close()


def test_residual_noalloc_on_a_side_stream():
    prob = W.make_problem(18, 1.04, seed=14)
    amg = B.AMG.from_csr(prob.A)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.linspace(-1.0, 1.0, prob.A.n, dtype=torch.float64, device="cuda")
    r0 = torch.empty_like(b)
    n0 = amg.residual_noalloc(b, x, r0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    r1 = torch.empty_like(b)
    with torch.cuda.stream(side):
        n1 = amg.residual_noalloc(b, x, r1, stream=side)
    side.synchronize()
    assert n0 == n1 and torch.equal(r0, r1)
    amg.close()


def test_residual_noalloc_rejects_overlap_and_wrong_sizes():
    prob = W.make_problem(10, 1.0, seed=2)
    amg = B.AMG.from_csr(prob.A)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    lib = B.load()
    norms = np.zeros(2)
    for rp in (b.data_ptr(), x.data_ptr() + 8):
        st = lib.amg_residual_noalloc(amg._h, b.data_ptr(), x.data_ptr(), rp, norms.ctypes.data, None)
        assert st == B.ERR_ARG
    with pytest.raises(ValueError):
        amg.residual_noalloc(b, x, torch.empty(prob.A.n - 1, dtype=torch.float64, device="cuda"))
    amg.close()


def test_residual_noalloc_row_limit():
    """The fixed scratch holds one partial-sum pair per 256 rows: 204^3 =
    8,489,664 rows is above its 8,388,608-row limit and is refused before
    anything is launched."""
    A, _, _ = W.q1_laplacian(204, 1.0)
    amg = B.AMG.from_csr(A)
    v = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = torch.empty_like(v)
    with pytest.raises(B.AmgError) as e:
        amg.residual_noalloc(v, v, r)
    assert e.value.status == B.ERR_ARG and "limit" in str(e.value)
    amg.close()
