"""Direct pin of the oracle's float32 V-cycle (the mixed mode's
preconditioner: matrix values, l1 diagonal, tentative weights, smoother,
residual and transfers in float32; the coarsest solve in float64).

The V-cycle is restated here with numpy float32 scalars in the documented
order: r rounded to float32 on entry; per level x = dinv32 * b,
t = A32 x (each row summed left to right in storage order),
b_c[agg(i)] += p32_i * (b_i - t_i) over increasing i; at the coarsest level
b widened to float64, solved with the float64 Cholesky factor (forward then
backward substitution, the factor read from the oracle) and rounded back;
then x += p32 * x_c[agg], t = A32 x, x = x + dinv32 * (b - t); z widened.
dinv32 is the float64 l1 diagonal's reciprocal rounded to float32, and
A32, p32 are the float64 values rounded. The oracle must agree bit for bit,
and planted float32 slips (dinv formed from a float32 row sum, the
restriction's product and sum contracted into one rounding) must not.
"""
import numpy as np
import pytest

import oracle as O
from paper_2210_16660_gb300 import workloads as W

f32 = np.float32


def _levels(h):
    out = []
    for l in range(h.nlevels):
        lv = h.level(l)
        agg, p = h.level_agg(l) if l + 1 < h.nlevels else (None, None)
        out.append((lv, agg, p))
    return out


def _spmv32(lv, v32, x):
    rp, ci = lv["row_ptr"], lv["col"]
    y = np.zeros(lv["n"], np.float32)
    for i in range(lv["n"]):
        s = f32(0.0)
        for k in range(rp[i], rp[i + 1]):
            s = f32(s + f32(v32[k] * x[ci[k]]))
        y[i] = s
    return y


def _dinv32(lv, from_f32_rowsum=False):
    rp, v = lv["row_ptr"], lv["val"]
    d = np.empty(lv["n"], np.float32)
    for i in range(lv["n"]):
        if from_f32_rowsum:
            s = f32(0.0)
            for k in range(rp[i], rp[i + 1]):
                s = f32(s + f32(abs(f32(v[k]))))
            d[i] = f32(f32(1.0) / s)
        else:
            s = 0.0
            for k in range(rp[i], rp[i + 1]):
                s = s + abs(float(v[k]))
            d[i] = f32(1.0 / s)
    return d


def _chol_solve(L, b):
    n = L.shape[0]
    x = np.zeros(n)
    for i in range(n):
        s = b[i]
        for k in range(i):
            s -= L[i, k] * x[k]
        x[i] = s / L[i, i]
    for i in range(n - 1, -1, -1):
        s = x[i]
        for k in range(i + 1, n):
            s -= L[k, i] * x[k]
        x[i] = s / L[i, i]
    return x


def vcycle32_numpy(h, r, slip=None):
    levs = _levels(h)
    Lc = len(levs) - 1
    v32 = [lv["val"].astype(np.float32) for lv, _, _ in levs]
    d32 = [_dinv32(lv, from_f32_rowsum=(slip == "f32_rowsum")) for lv, _, _ in levs]
    b = [None] * (Lc + 1)
    x = [None] * (Lc + 1)
    b[0] = np.asarray(r).astype(np.float32)
    for l in range(Lc):
        lv, agg, p = levs[l]
        p32 = p.astype(np.float32)
        x[l] = (d32[l] * b[l]).astype(np.float32)
        t = _spmv32(lv, v32[l], x[l])
        nc = levs[l + 1][0]["n"]
        bc = np.zeros(nc, np.float32)
        for i in range(lv["n"]):
            if agg[i] >= 0:
                res = f32(b[l][i] - t[i])
                if slip == "fused_restrict":
                    # the product not rounded before the sum (a contracted multiply-add)
                    bc[agg[i]] = f32(float(bc[agg[i]]) + float(p32[i]) * float(res))
                else:
                    bc[agg[i]] = f32(bc[agg[i]] + f32(p32[i] * res))
        b[l + 1] = bc
    L = h.coarse_factor()
    x[Lc] = _chol_solve(L, b[Lc].astype(np.float64)).astype(np.float32)
    for l in range(Lc - 1, -1, -1):
        lv, agg, p = levs[l]
        p32 = p.astype(np.float32)
        xl = x[l].copy()
        for i in range(lv["n"]):
            if agg[i] >= 0:
                xl[i] = f32(xl[i] + f32(p32[i] * x[l + 1][agg[i]]))
        t = _spmv32(lv, v32[l], xl)
        x[l] = np.array([f32(xl[i] + f32(d32[l][i] * f32(b[l][i] - t[i]))) for i in range(lv["n"])],
                        np.float32)
    return x[0].astype(np.float64)


@pytest.mark.parametrize("N,ratio,cmax", [(5, 1.04, 8), (6, 1.0, 12)])
def test_float32_vcycle_bit_for_bit(N, ratio, cmax):
    A, _, _ = W.q1_laplacian(N, ratio)
    h = O.Hierarchy(A, coarse_max=cmax, n_pass=2)
    assert h.nlevels >= 3
    r = np.random.default_rng(N).standard_normal(A.n)
    z = h.vcycle(r, fp32=True)
    want = vcycle32_numpy(h, r)
    assert np.array_equal(z.view(np.int64), want.view(np.int64))
    # the pin is sensitive to float32 slips of the kind a restatement can make
    for slip in ("f32_rowsum", "fused_restrict"):
        assert not np.array_equal(vcycle32_numpy(h, r, slip=slip), z), slip
