"""GPU path vs the CPU oracle, through the C ABI.

Bar: aggregate maps of every pass and level bit-exact; coarse matrices bit
exact (same canonical summation order on both sides); iteration counts
within +-1; true float64 relative residual <= rtol; and
||x - x_oracle|| / ||x_oracle|| <= 1e-6 at rtol 1e-8 for both the float64
PCG and the float32-V-cycle FCG(1) path.
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


def _setup_both(A, **kw):
    h_or = O.Hierarchy(A, coarse_max=kw.get("coarse_max", 200), n_pass=kw.get("n_pass", 2),
                       max_levels=kw.get("max_levels", 30))
    amg = B.AMG.from_csr(A, **kw)
    return h_or, amg


def _compare_hierarchy(h_or, amg):
    info = amg.info()
    assert len(info) == h_or.nlevels
    for l in range(h_or.nlevels):
        n, z, npass = h_or.level_size(l)
        assert info[l] == (n, z)
        lv = h_or.level(l)
        rp, ci, v = amg.level_csr(l)
        assert np.array_equal(rp, lv["row_ptr"]) and np.array_equal(ci, lv["col"])
        assert np.array_equal(v.view(np.int64), lv["val"].view(np.int64)), f"level {l} values differ"
        if l + 1 < h_or.nlevels:
            for ps in range(npass):
                a_or, nc_or = h_or.pass_agg(l, ps)
                a_gpu, nc_gpu = amg.level_agg(l, ps)
                assert nc_gpu == nc_or
                assert np.array_equal(a_gpu, a_or), f"level {l} pass {ps} aggregates differ"
            agg_or, _ = h_or.level_agg(l)
            agg_gpu, _ = amg.level_agg(l, -1)
            assert np.array_equal(agg_gpu, agg_or)


@pytest.mark.parametrize("N,ratio,cmax", [(7, 1.0, 20), (13, 1.04, 50), (32, 1.0, 200), (33, 1.04, 200)])
def test_hierarchy_bit_exact(N, ratio, cmax):
    A, _, _ = W.q1_laplacian(N, ratio)
    h_or, amg = _setup_both(A, coarse_max=cmax)
    _compare_hierarchy(h_or, amg)


@pytest.mark.parametrize("npass", [1, 3, 4])
def test_hierarchy_bit_exact_npass(npass):
    A, _, _ = W.q1_laplacian(24, 1.04, lx=4.0)
    h_or, amg = _setup_both(A, n_pass=npass)
    _compare_hierarchy(h_or, amg)


def _solve_parity(prob, mode, device_vectors=True, x0=None, **kw):
    h_or = O.Hierarchy(prob.A, coarse_max=kw.get("coarse_max", 200), n_pass=kw.get("n_pass", 2))
    ref = h_or.solve(prob.b, x0=x0, rtol=RTOL, maxit=1000, mode=mode)
    amg = B.AMG.from_csr(prob.A, mode=mode, **kw)
    if device_vectors:
        b = torch.from_numpy(prob.b).cuda()
        x = torch.zeros_like(b) if x0 is None else torch.from_numpy(x0.copy()).cuda()
    else:
        b = prob.b.copy()
        x = np.zeros_like(b) if x0 is None else x0.copy()
    res = amg.solve(b, x, rtol=RTOL, maxit=1000)
    xs = x.cpu().numpy() if device_vectors else x
    assert res.status == 0, res.message
    assert abs(res.iters - ref["iters"]) <= 1, (res.iters, ref["iters"])
    true_rel = np.linalg.norm(prob.b - W.spmv(prob.A, xs)) / np.linalg.norm(prob.b)
    assert true_rel <= RTOL and res.true_rel <= RTOL
    err = np.linalg.norm(xs - ref["x"]) / np.linalg.norm(ref["x"])
    assert err <= X_TOL, err
    # history: same length as the iterations, starts at ||r0||/||b||, ends below rtol
    assert len(res.hist) == res.iters + 1
    assert res.hist[0] == pytest.approx(ref["hist"][0], rel=1e-12)
    assert res.hist[-1] <= RTOL
    return res, ref, xs, amg


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
@pytest.mark.parametrize("N,ratio", [(7, 1.0), (13, 1.04), (32, 1.0), (40, 1.04)])
def test_solve_parity(N, ratio, mode):
    prob = W.make_problem(N, ratio, seed=1)
    _solve_parity(prob, mode)


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_host_vectors_and_warm_start(mode):
    prob = W.make_problem(20, 1.04, seed=7)
    x0 = 0.9 * prob.x_star
    r1, _, x1, amg = _solve_parity(prob, mode, device_vectors=False, x0=x0)
    # the same call with device vectors gives bitwise the same iterate
    b = torch.from_numpy(prob.b).cuda()
    x = torch.from_numpy(x0.copy()).cuda()
    r2 = amg.solve(b, x, rtol=RTOL, maxit=1000)
    assert r2.iters == r1.iters
    assert np.array_equal(x.cpu().numpy(), x1)


def test_single_level_converges_in_one_iteration():
    # one level: B = A^{-1}; in float64 one iteration suffices, while the
    # float32 V-cycle rounds r and z to float32 (~1e-7), so it takes two
    prob = W.make_problem(5, 1.04, seed=2)
    res, ref, _, _ = _solve_parity(prob, "pcg64", coarse_max=200)
    assert res.iters == 1 and ref["iters"] == 1
    res, ref, _, _ = _solve_parity(prob, "fcg32", coarse_max=200)
    assert res.iters <= 2 and ref["iters"] <= 2


def test_special_cases():
    prob = W.make_problem(12, 1.04, seed=3)
    amg = B.AMG.from_csr(prob.A)
    n = prob.A.n
    # b = 0: x = 0, no iteration
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    res = amg.solve(torch.zeros(n, dtype=torch.float64, device="cuda"), x)
    assert res.status == 0 and res.iters == 0 and not x.any()
    # converged initial guess
    xs = np.linalg.solve(prob.A.to_dense(), prob.b)
    x = torch.from_numpy(xs).cuda()
    res = amg.solve(torch.from_numpy(prob.b).cuda(), x, rtol=1e-8)
    assert res.status == 0 and res.iters == 0
    # maxit exhausted
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = amg.solve(torch.from_numpy(prob.b).cuda(), x, rtol=1e-15, maxit=3)
    assert res.status == B.ERR_NOCONV and res.iters == 3
    # NaN in b
    b = prob.b.copy()
    b[5] = np.nan
    res = amg.solve(torch.from_numpy(b).cuda(), torch.zeros(n, dtype=torch.float64, device="cuda"))
    assert res.status == B.ERR_NAN
    # bad arguments
    res = amg.solve(torch.from_numpy(prob.b).cuda(), x, rtol=-1.0)
    assert res.status == B.ERR_ARG


def test_invalid_matrices_rejected():
    A, _, _ = W.q1_laplacian(6, 1.04)
    bad = W.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    bad.col[[1, 2]] = bad.col[[2, 1]]
    with pytest.raises(B.AmgError) as e:
        B.AMG.from_csr(bad)
    assert e.value.status == B.ERR_ARG
    asym = W.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    k = int(np.nonzero(asym.col[asym.row_ptr[100]:asym.row_ptr[101]] != 100)[0][0]) + asym.row_ptr[100]
    asym.val[k] *= 1.0000001
    with pytest.raises(B.AmgError) as e:
        B.AMG.from_csr(asym)
    assert e.value.status == B.ERR_ARG
    with pytest.raises(B.AmgError) as e:
        B.AMG.from_csr(A, hbm_budget=1 << 16)
    assert e.value.status == B.ERR_OOM


def test_deterministic_repeat():
    prob = W.make_problem(24, 1.04, seed=4)
    amg = B.AMG.from_csr(prob.A, mode="fcg32")
    outs = []
    for _ in range(3):
        x = torch.zeros(prob.A.n, dtype=torch.float64, device="cuda")
        amg.solve(torch.from_numpy(prob.b).cuda(), x)
        outs.append(x.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_graph_and_stream_launch_paths_agree():
    """The whole-solve graph and plain stream launches run the same kernels."""
    prob = W.make_problem(28, 1.04, seed=6)
    b = torch.from_numpy(prob.b).cuda()
    for mode in ("pcg64", "fcg32"):
        amg = B.AMG.from_csr(prob.A, mode=mode)
        x1 = torch.zeros_like(b)
        n0 = amg.launch_count()
        r1 = amg.solve(b, x1)
        n_graph = amg.launch_count() - n0
        amg.profile(True)
        x2 = torch.zeros_like(b)
        r2 = amg.solve(b, x2)
        prof = amg.profile_read()
        amg.profile(False)
        assert r1.status == r2.status == 0 and r1.iters == r2.iters
        assert torch.equal(x1, x2)
        assert np.array_equal(r1.hist, r2.hist)
        assert n_graph >= 5 * r1.iters
        assert prof["spmv"][1] >= r1.iters and prof["spmv"][0] > 0


def _with_env(key, val, fn):
    import os
    old = os.environ.get(key)
    os.environ[key] = val
    try:
        return fn()
    finally:
        if old is None:
            del os.environ[key]
        else:
            os.environ[key] = old


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_int16_and_int32_columns_agree(mode):
    """Columns stored as int16 offsets and as int32 give bitwise the same solve."""
    prob = W.make_problem(30, 1.04, seed=8)
    b = torch.from_numpy(prob.b).cuda()
    a16 = B.AMG.from_csr(prob.A, mode=mode)
    a32 = _with_env("PCGAMG_COL16", "0", lambda: B.AMG.from_csr(prob.A, mode=mode))
    assert a16.level_layout(0)["index_bytes"] == 2
    assert all(a32.level_layout(l)["index_bytes"] == 4 for l in range(len(a32.info())))
    x16, x32 = torch.zeros_like(b), torch.zeros_like(b)
    r16, r32 = a16.solve(b, x16), a32.solve(b, x32)
    assert r16.status == r32.status == 0 and r16.iters == r32.iters
    assert torch.equal(x16, x32)


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
@pytest.mark.parametrize("N", [32, 64])
def test_cluster_tail_matches_separate_launches(mode, N):
    """Small levels in one thread-block cluster with their data in shared
    memory (the default) give the same solve, bit for bit, as one launch per
    sweep (PCGAMG_TAIL=0)."""
    prob = W.make_problem(N, 1.04, seed=10)
    b = torch.from_numpy(prob.b).cuda()
    a1 = B.AMG.from_csr(prob.A, mode=mode)
    a2 = _with_env("PCGAMG_TAIL", "0", lambda: B.AMG.from_csr(prob.A, mode=mode))
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    n1, n2 = a1.launch_count(), a2.launch_count()
    r1, r2 = a1.solve(b, x1), a2.solve(b, x2)
    assert r1.status == r2.status == 0 and r1.iters == r2.iters
    assert a1.launch_count() - n1 < a2.launch_count() - n2      # the tail replaced launches
    assert torch.equal(x1, x2)
    # and the path without the tail meets the oracle too
    _with_env("PCGAMG_TAIL", "0", lambda: _solve_parity(prob, mode))


def _add_long_coupling(A, i, j, v):
    """A with one extra symmetric pair a_ij = a_ji = v (columns kept sorted)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    r = np.concatenate([rows, [i, j]])
    c = np.concatenate([A.col, [j, i]]).astype(np.int64)
    val = np.concatenate([A.val, [v, v]])
    order = np.lexsort((c, r))
    r, c, val = r[order], c[order], val[order]
    rp = np.zeros(A.n + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=A.n), out=rp[1:])
    return W.CSR(A.n, rp.astype(np.int32), c.astype(np.int32), val)


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_wide_columns_fall_back_to_int32(mode):
    """A coupling further than 2^15 rows apart keeps int32 columns; parity holds."""
    N = 33
    A, wall, _ = W.q1_laplacian(N, 1.04)
    i, j = N * N, A.n - 1
    A2 = _add_long_coupling(A, i, j, -1e-3)
    xs = W.normals(9, A2.n)
    xs[wall] = 0.0
    prob = W.Problem("long", N, A2, W.spmv(A2, xs), xs, wall, None)
    res, ref, _, amg = _solve_parity(prob, mode)
    assert amg.level_layout(0)["index_bytes"] == 4


def test_torch_allocator_route():
    prob = W.make_problem(10, 1.04, seed=5)
    B.use_torch_allocator(True)
    try:
        b = torch.from_numpy(prob.b).cuda()
        x = torch.zeros(prob.A.n, dtype=torch.float64, device="cuda")
        before = torch.cuda.memory_allocated()
        amg = B.AMG.from_csr(prob.A)
        assert torch.cuda.memory_allocated() > before
        assert amg.solve(b, x).status == 0
        amg.close()
        assert torch.cuda.memory_allocated() == before
    finally:
        B.use_torch_allocator(False)


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_full_size_128_graded(mode):
    """128^3 nodes, z graded 1.04 (2.1M dofs, 55M nnz): the benchmarked system."""
    prob = W.make_problem(128, 1.04, seed=2)
    h_or = O.Hierarchy(prob.A, n_pass=2)
    amg = B.AMG.from_csr(prob.A, mode=mode)
    # aggregates of every level and pass bit-exact
    for l in range(h_or.nlevels - 1):
        for ps in range(2):
            assert np.array_equal(amg.level_agg(l, ps)[0], h_or.pass_agg(l, ps)[0])
    ref = h_or.solve(prob.b, rtol=RTOL, maxit=1000, mode=mode)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    res = amg.solve(b, x, rtol=RTOL, maxit=1000)
    xs = x.cpu().numpy()
    assert res.status == 0 and abs(res.iters - ref["iters"]) <= 1
    assert np.linalg.norm(prob.b - W.spmv(prob.A, xs)) / np.linalg.norm(prob.b) <= RTOL
    assert np.linalg.norm(xs - ref["x"]) / np.linalg.norm(ref["x"]) <= X_TOL


@pytest.mark.parametrize("mode", ["pcg64", "fcg32"])
def test_every_launch_shape_gives_the_same_bits(mode):
    """Sweep launch shapes (chunk depth x grid form x fused or separate
    launches, and rows read by 4 lanes) change speed only: each
    forced shape, and the tuner's pick, reproduce the default solve bit for
    bit (rows are summed in storage order whatever the shape)."""
    prob = W.make_problem(40, 1.04, seed=12)
    b = torch.from_numpy(prob.b).cuda()
    amg = B.AMG.from_csr(prob.A, mode=mode)
    L = len(amg.info())
    assert amg.level_shape(0) == [0, 0, 0, 0]
    x0 = torch.zeros_like(b)
    r0 = amg.solve(b, x0)
    assert r0.status == 0
    for shape in range(9):
        for lvl in range(1, L):
            amg.set_level_shape(lvl, [shape] * 4)
        x = torch.zeros_like(b)
        r = amg.solve(b, x)
        assert r.iters == r0.iters and torch.equal(x, x0), shape
    before = [amg.level_shape(lvl) for lvl in range(L)]
    changed = amg.autotune(reps=2)
    after = [amg.level_shape(lvl) for lvl in range(L)]
    assert changed == sum(u != v for a, c in zip(before, after) for u, v in zip(a, c))
    assert after[0] == [0, 0, 0, 0] and all(0 <= v <= 8 for s in after for v in s)
    x = torch.zeros_like(b)
    r = amg.solve(b, x)
    assert r.iters == r0.iters and torch.equal(x, x0)
    with pytest.raises(B.AmgError):
        amg.set_level_shape(0, [0, 0, 0, 0])
    with pytest.raises(B.AmgError):
        amg.set_level_shape(1, [9, 0, 0, 0])


def test_hand_worked_pairwise_aggregation_on_gpu():
    """The device setup on the example worked by hand from Sec. 3.1
    (tests/golden/path5_pairwise_aggregation.json): pass aggregates, the
    composed map and the level-1 Galerkin matrix."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "path5_pairwise_aggregation.json")))
    Ad = np.array(g["matrix_dense"], float)
    n = Ad.shape[0]
    rows, cols = np.nonzero(Ad)
    rp = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    A = W.CSR(n, rp, cols.astype(np.int32), Ad[rows, cols])
    amg = B.AMG.from_csr(A, coarse_max=1, n_pass=2)
    assert len(amg.info()) == g["levels"]
    a0, nc0 = amg.level_agg(0, 0)
    assert list(a0) == g["pass0"]["agg"] and nc0 == len(g["pass0"]["w_c"])
    a1, nc1 = amg.level_agg(0, 1)
    assert list(a1) == g["pass1"]["agg"] and nc1 == g["pass1"]["n_c"]
    ac, _ = amg.level_agg(0)
    assert list(ac) == g["level0_composed"]["agg"]
    rp1, ci1, v1 = amg.level_csr(1)
    A1 = np.zeros((2, 2))
    for i in range(2):
        A1[i, ci1[rp1[i]:rp1[i + 1]]] = v1[rp1[i]:rp1[i + 1]]
    np.testing.assert_allclose(A1, g["level1"]["A"], rtol=1e-15, atol=1e-15)
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    r = amg.solve(b, x, rtol=1e-12)
    assert r.status == 0
    np.testing.assert_allclose(x.cpu().numpy(), np.linalg.solve(Ad, np.ones(n)), rtol=1e-10)
