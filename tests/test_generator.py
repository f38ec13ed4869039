"""Pins of the synthetic input generator (graded-hex Q1 Laplacian).

Checked against facts fixed by the discretisation, not by re-running the
generator's own formulas: the closed-form pattern size, exact symmetry, zero
row sums under Neumann conditions, and the tensor-product eigenpairs (with
the textbook closed form of the 1D eigenvalues on a uniform grid).
"""
import numpy as np
import pytest

from paper_2210_16660_gb300 import workloads as W


def _pattern_count(N):
    # full 27-point pattern: (3N-2)^3 entries; the Dirichlet plane iz=0 drops
    # its in-plane off-diagonals ((3N-2)^2 - N^2), and both directions of its
    # couplings to the plane iz=1 (2 (3N-2)^2 entries).
    full = (3 * N - 2) ** 3
    plane = (3 * N - 2) ** 2
    return full - (plane - N * N) - 2 * plane


@pytest.mark.parametrize("N", [2, 3, 5, 8, 32])
def test_nnz_closed_form(N):
    A, _, _ = W.q1_laplacian(N, 1.04)
    assert A.n == N ** 3
    assert A.nnz == _pattern_count(N)
    if N == 32:
        assert A.nnz == 805_100


def test_bitwise_symmetric_sorted():
    A, _, _ = W.q1_laplacian(9, 1.04, lx=4.0)
    d = A.to_dense()
    assert np.array_equal(d, d.T)
    for i in range(A.n):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)
        assert i in c


def test_neumann_row_sums_vanish():
    # K 1 = 0 along every axis, so rows away from the wall sum to zero.
    N = 10
    A, _, _ = W.q1_laplacian(N, 1.04)
    rs = W.spmv(A, np.ones(A.n)).reshape(N, N, N)
    scale = np.abs(A.val).max()
    assert np.abs(rs[2:]).max() <= 1e-13 * scale
    # wall rows keep a positive diagonal only
    for i in range(N * N):
        s, e = A.row_ptr[i], A.row_ptr[i + 1]
        assert e - s == 1 and A.col[s] == i and A.val[s] > 0


def _dense_1d(h, dirichlet_first):
    n = h.size + 1
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    for e, he in enumerate(h):
        K[e:e + 2, e:e + 2] += np.array([[1, -1], [-1, 1]]) / he
        M[e:e + 2, e:e + 2] += np.array([[2, 1], [1, 2]]) * he / 6
    if dirichlet_first:
        K, M = K[1:, 1:], M[1:, 1:]
    return K, M


def _geig(K, M):
    from scipy.linalg import eigh
    return eigh(K, M)


@pytest.mark.parametrize("N,ratio,lx", [(7, 1.0, 1.0), (9, 1.04, 1.0), (8, 1.02, 4.0)])
def test_tensor_eigenpairs(N, ratio, lx):
    """A u = (lx + ly + lz) M3 u for u = vx (x) vy (x) vz (generalised 1D pairs)."""
    A, wall, (hx, hy, hz) = W.q1_laplacian(N, ratio, lx=lx)
    Kx, Mx = _dense_1d(hx, False)
    Ky, My = _dense_1d(hy, False)
    Kz, Mz = _dense_1d(hz, True)
    lxv, Vx = _geig(Kx, Mx)
    lyv, Vy = _geig(Ky, My)
    lzv, Vz = _geig(Kz, Mz)
    rng = np.random.default_rng(0)
    for _ in range(6):
        a, b, c = rng.integers(0, N), rng.integers(0, N), rng.integers(0, N - 1)
        # node index ix + N*(iy + N*iz): z slowest, so u = vz (x) vy (x) vx
        uz = np.concatenate([[0.0], Vz[:, c]])
        u = np.kron(uz, np.kron(Vy[:, b], Vx[:, a]))
        Mz_full = np.zeros((N, N))
        Mz_full[1:, 1:] = Mz
        Mu = np.kron(Mz_full, np.kron(My, Mx)) @ u
        lam = lxv[a] + lyv[b] + lzv[c]
        Au = W.spmv(A, u)
        assert np.linalg.norm(Au - lam * Mu) <= 1e-10 * np.linalg.norm(Au)


@pytest.mark.parametrize("N", [6, 11])
def test_uniform_1d_closed_form(N):
    """Uniform 1D linear FE: lambda = 6 (1 - cos t) / (h^2 (2 + cos t))."""
    h = np.full(N - 1, 1.0 / (N - 1))
    K, M = _dense_1d(h, False)
    lam = np.sort(_geig(K, M)[0])
    t = np.arange(N) * np.pi / (N - 1)
    ref = np.sort(6 * (1 - np.cos(t)) / (h[0] ** 2 * (2 + np.cos(t))))
    assert np.allclose(lam, ref, rtol=1e-10, atol=1e-9)
    K, M = _dense_1d(h, True)
    lam = np.sort(_geig(K, M)[0])
    t = (np.arange(N - 1) + 0.5) * np.pi / (N - 1)
    ref = np.sort(6 * (1 - np.cos(t)) / (h[0] ** 2 * (2 + np.cos(t))))
    assert np.allclose(lam, ref, rtol=1e-10)
    # and the 3D operator inherits them: check one uniform tensor mode
    A, _, _ = W.q1_laplacian(N, 1.0)
    kx, ky, kz = 1, 2, 0
    v = lambda k: np.cos(k * np.pi * np.arange(N) / (N - 1))
    vz = np.sin((kz + 0.5) * np.pi * np.arange(N) / (N - 1))
    u = np.kron(vz, np.kron(v(ky), v(kx)))
    lam1 = lambda th: 6 * (1 - np.cos(th)) / (h[0] ** 2 * (2 + np.cos(th)))
    lam3 = lam1(kx * np.pi / (N - 1)) + lam1(ky * np.pi / (N - 1)) + lam1((kz + .5) * np.pi / (N - 1))
    _, M1 = _dense_1d(h, False)
    Mu = np.kron(M1, np.kron(M1, M1)) @ u
    Au = W.spmv(A, u)
    inner = np.arange(A.n) >= N * N
    # Dirichlet rows are replaced by the identity-like diagonal; compare the rest
    # with the z-mass coupling to the wall plane removed (vz vanishes there).
    M1z = M1.copy()
    M1z[0, :] = 0
    M1z[:, 0] = 0
    Mu = np.kron(M1z, np.kron(M1, M1)) @ u
    assert np.linalg.norm((Au - lam3 * Mu)[inner]) <= 1e-9 * np.linalg.norm(Au[inner])


def test_normals_reproducible_and_standard():
    z = W.normals(7, 200_001)
    assert np.array_equal(z, W.normals(7, 200_001))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    # offsets address the same stream
    assert np.array_equal(W.normals(7, 10, offset=5), z[5:15])
    # SplitMix64 reference value (seed 0, first output) from its published definition
    assert int(W.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


def test_problem_rhs():
    p = W.make_problem(6, 1.04, seed=3)
    assert np.all(p.x_star[p.wall] == 0)
    assert np.allclose(p.b, p.A.to_dense() @ p.x_star, rtol=1e-14, atol=1e-14)


def test_poisson_arrivals_and_choices():
    """The serving stream: arrivals start at 0, never go back, and their gaps
    have the exponential mean 1/rate; an infinite rate queues everything at
    0; mesh choices are uniform."""
    a = W.poisson_arrivals(20.0, 20000, seed=5)
    assert a[0] == 0.0 and np.all(np.diff(a) >= 0.0)
    gaps = np.diff(a)
    assert abs(gaps.mean() - 1 / 20.0) < 0.05 / 20.0
    assert abs(np.median(gaps) - np.log(2) / 20.0) < 0.05 / 20.0   # exponential median
    assert not W.poisson_arrivals(float("inf"), 7, seed=5).any()
    np.testing.assert_array_equal(a, W.poisson_arrivals(20.0, 20000, seed=5))
    c = W.uniform_choices(30000, 3, seed=5)
    assert set(np.unique(c)) == {0, 1, 2}
    assert np.all(np.abs(np.bincount(c) / 30000 - 1 / 3) < 0.01)


def test_time_step_chain():
    """Each step is warm-started from the previous exact solution, its
    right-hand side is A x*_t, and x*_t stays zero on the Dirichlet wall."""
    prob = W.make_problem(8, 1.04, seed=2)
    chain = W.time_steps(prob, prob.x_star, 3, seed=9)
    prev = prob.x_star
    for b, x0, xs in chain:
        np.testing.assert_array_equal(x0, prev)
        np.testing.assert_array_equal(b, W.spmv(prob.A, xs))
        assert not xs[prob.wall].any()
        rms = np.sqrt(np.mean(prev * prev))
        assert 0 < np.linalg.norm(xs - prev) / (rms * np.sqrt(prob.A.n)) < 0.02
        prev = xs
