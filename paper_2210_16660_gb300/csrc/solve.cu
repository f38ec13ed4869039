// Solve phase: PCG / FCG(1) preconditioned by one V-cycle per iteration
// (arxiv 2210.16660, Sec. 3.1 Eq. (multiplicative composition) with nu = 1
// and M = D_l1; Sec. 5 flexible CG with a relative-residual stop).
//
// Every sweep streams a sliced-ELL matrix (one warp per 32-row slice,
// coalesced value/column loads, 4 entries of a row loaded ahead of their
// gathers) and fuses the vector work around it.
//
// GB300 note: float64 FMA throughput (~1.25 TFLOP/s) is about what one FMA per
// stored entry needs at full HBM bandwidth, so every float64 sweep does
// exactly one float64 operation per stored entry; anything else is formed
// once per row (D^-1 b, D^-1 b + P x_c, p = z + beta p). The float32 V-cycle
// reads a float32 copy of r (and of D^-1 r) so no conversion happens per entry.
//
// V-cycle (T = float for FCG(1), double for PCG; one structure for both):
//   down   : t = p .* (b - A xpre), xpre = D^-1 b formed by the producer of b
//   restr  : b_{l+1}[I] = sum_{i in G_I} t_i (members in index order), and
//            xpre_{l+1} = D^-1 b_{l+1}
//   coarse : x_L = A_L^{-1} b_L (float64 dense inverse)
//   prolong: xp = xpre + P x_{l+1}
//   post   : z = xp + D^-1 (b - A xp)
// so every sweep gathers one vector per stored entry.
// Krylov (float64): p = z + beta p; q = A p, p.q; x += alpha p,
// r -= alpha q, ||r||^2 (+ r32 or xpre_0); true residual when rtol is met.
//
// Reductions are two-stage and deterministic: each block writes a partial,
// the last block to finish (atomic ticket) sums the partials in index order
// and updates the iteration's scalars in device memory (struct Ctl), so an
// iteration needs no host round trip.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <type_traits>

#include "internal.cuh"
#include "sell_row.cuh"

namespace pcgamg {

namespace {

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// Block-wide sum of two doubles (blockDim.x == kBlock); result in warp 0.
__device__ __forceinline__ void block_sum2(double &a, double &b) {
    __shared__ double sa[kBlock / 32], sb[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (w == 0) {
        a = lane < kBlock / 32 ? sa[lane] : 0.0;
        b = lane < kBlock / 32 ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// Writes this block's partials; returns true in every thread of the last
// block to finish, after which partials[0..gridDim) are complete.
__device__ __forceinline__ bool publish_partials(double a, double b, double *partials, unsigned *counter) {
    __shared__ bool last;
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = a;
        partials[gridDim.x + blockIdx.x] = b;
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return last;
}

// Sum of the partials in a fixed order (run by the whole last block).
__device__ __forceinline__ void final_sum2(const double *partials, double &a, double &b) {
    __threadfence();
    a = 0.0;
    b = 0.0;
    int nb = gridDim.x;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        a += __ldcg(partials + k);
        b += __ldcg(partials + nb + k);
    }
    block_sum2(a, b);
}

__device__ __forceinline__ void fail(Ctl *c, int status) {
    c->done = 2;
    c->status = status;
}

// rho = r.z and beta of the next direction (last block of the kernel that
// produced z): PCG beta = rho / rho_old, FCG(1) beta = -(z.q_old) / (p.q)_old
// (the float32 V-cycle, and either precision when the iterative coarsest
// solve makes the V-cycle vary from one application to the next).
__device__ __forceinline__ void finish_rho(Ctl *ctl, double rz, double zq) {
    ctl->counter[0] = 0;
    if (!isfinite(rz) || !isfinite(zq)) { fail(ctl, AMG_ERR_NAN); return; }
    if (!(rz > 0.0)) { fail(ctl, AMG_ERR_BREAKDOWN); return; }
    ctl->rho = rz;
    ctl->zq = zq;
    double beta = 0.0;
    if (!ctl->restart) beta = ctl->mode == AMG_MODE_FCG32 || ctl->flex ? -zq / ctl->pq_old : rz / ctl->rho_old;
    ctl->beta = beta;
}

#define SELL_ROW_BEGIN                                               \
    int s_ = i >> 5, lane_ = i & 31;                                 \
    int32_t base_ = ldg(sptr + s_);                                  \
    int w_ = (ldg(sptr + s_ + 1) - base_) >> 5;                      \
    const IDX *c_ = col + base_ + lane_;                             \
    const auto *a_ = val + base_ + lane_;

// ------------------------------------------------------------ V-cycle sweeps
template <typename T>
struct Occ { static constexpr int kMinBlocks = sizeof(T) == 4 ? 6 : 4; };
// Sweeps with 16-entry chunks hold two chunks (the current one and the one
// in flight) in registers: two float32 blocks per SM, one float64.
template <typename T, int U>
struct SweepOcc {
    static constexpr int kMinBlocks = U <= 4 ? Occ<T>::kMinBlocks
                                      : U == kPatRow ? (sizeof(T) == 4 ? 3 : 1)
                                                     : (sizeof(T) == 4 ? 2 : 1);
};

// The V-cycle sweeps, restriction and prolongation read their first row's
// static data (matrix entries, weights, aggregate maps: written only by
// setup and refresh) before pdl_enter(), so it arrives while the preceding
// kernel drains; what a preceding kernel wrote is read through after_wait()
// pointers once the wait has returned.

// Pre-smooth from zero, residual, weighted restriction input:
// t_i = p_i (b_i - sum_j a_ij xpre_j), xpre = D^-1 b.
template <typename T, typename IDX, int U, bool STREAM>
__global__ void __launch_bounds__(kBlock, SweepOcc<T, U>::kMinBlocks) k_down(
    int n, const int32_t *__restrict__ sptr, const IDX *__restrict__ col, const T *__restrict__ val,
    const IDX *__restrict__ upat, const T *__restrict__ xpre, const T *__restrict__ b,
    const T *__restrict__ p, T *__restrict__ t, const Ctl *__restrict__ ctl) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    RowOf<U, STREAM, IDX, T> R;
    T pi = 0;
    if (i < n) {
        R.load(sptr, col, val, i, upat);
        pi = ldg(p + i);
    }
    pdl_enter();
    xpre = after_wait(xpre);
    b = after_wait(b);
    ctl = after_wait(ctl);
    if (ctl->done) return;
    for (; i < n; i += stride) {
        T acc = R.dot(i, [&](int j) { return ldg(xpre + j); });
        t[i] = pi * (ldg(b + i) - acc);
        if (i + stride < n) {
            R.load(sptr, col, val, i + stride, upat);
            pi = ldg(p + i + stride);
        }
    }
}

// The multi-lane launch shape of the coarse levels: k_down and k_post with
// kMlL lanes per row (MlRow), one row per lane group, the whole of a row's
// first pass (columns and values) loaded before the wait. Same values and
// summation order as k_down / k_post. A warp whose rows lie past the last
// slice leaves before any shuffle; the others keep every lane to the end.
template <typename T, typename IDX>
__global__ void __launch_bounds__(kBlock) k_down_ml(int n, const int32_t *__restrict__ sptr,
                                                    const IDX *__restrict__ col, const T *__restrict__ val,
                                                    const T *__restrict__ xpre, const T *__restrict__ b,
                                                    const T *__restrict__ p, T *__restrict__ t,
                                                    const Ctl *__restrict__ ctl) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = gid / kMlL, q = gid % kMlL;
    if ((row >> 5) >= (n + 31) >> 5) return;
    const bool live = row < n;
    MlRow<false, IDX, T> R;
    R.load(sptr, col, val, row, q, live);
    T pi = 0;
    if (live && q == 0) pi = ldg(p + row);
    pdl_enter();
    xpre = after_wait(xpre);
    b = after_wait(b);
    ctl = after_wait(ctl);
    if (ctl->done) return;
    T acc = R.dot(row, [&](int j) { return ldg(xpre + j); });
    if (live && q == 0) t[row] = pi * (ldg(b + row) - acc);
}

template <typename T, typename IDX>
__global__ void __launch_bounds__(kBlock) k_post_ml(int n, const int32_t *__restrict__ sptr,
                                                    const IDX *__restrict__ col, const T *__restrict__ val,
                                                    const T *__restrict__ xp, const T *__restrict__ b,
                                                    const T *__restrict__ dinv, T *__restrict__ z,
                                                    const Ctl *__restrict__ ctl) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = gid / kMlL, q = gid % kMlL;
    if ((row >> 5) >= (n + 31) >> 5) return;
    const bool live = row < n;
    MlRow<false, IDX, T> R;
    R.load(sptr, col, val, row, q, live);
    T di = 0;
    if (live && q == 0) di = ldg(dinv + row);
    pdl_enter();
    xp = after_wait(xp);
    b = after_wait(b);
    ctl = after_wait(ctl);
    if (ctl->done) return;
    T acc = R.dot(row, [&](int j) { return ldg(xp + j); });
    if (live && q == 0) z[row] = ldg(xp + row) + di * (ldg(b + row) - acc);
}

// xp_i = xpre_i + p_i xc[agg_i].
template <typename T>
__global__ void __launch_bounds__(kBlock) k_prolong(int n, const T *__restrict__ xpre, const T *__restrict__ p,
                                                    const int32_t *__restrict__ agg, const T *__restrict__ xc,
                                                    T *__restrict__ xp, const Ctl *__restrict__ ctl) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    int a = -1;
    T pw = 0;
    if (i < n) {
        a = ldg(agg + i);
        pw = ldg(p + i);
    }
    pdl_enter();
    xpre = after_wait(xpre);
    xc = after_wait(xc);
    ctl = after_wait(ctl);
    if (ctl->done) return;
    for (; i < n; i += stride) {
        T x = ldg(xpre + i);
        if (a >= 0) x += pw * ldg(xc + a);
        xp[i] = x;
        if (i + stride < n) {
            a = ldg(agg + i + stride);
            pw = ldg(p + i + stride);
        }
    }
}

// Post-smooth z_i = xp_i + dinv_i (b_i - sum_j a_ij xp_j). On level 0 (DOT)
// z is written in float64 and the kernel also forms r.z (float64 r) and, for
// FCG(1), z.q_old; its last block turns them into rho and beta.
template <typename T, typename TZ, bool DOT, bool FCG, typename IDX, int U, bool STREAM>
__global__ void __launch_bounds__(kBlock, SweepOcc<T, U>::kMinBlocks) k_post(
    int n, const int32_t *__restrict__ sptr, const IDX *__restrict__ col, const T *__restrict__ val,
    const IDX *__restrict__ upat, const T *__restrict__ xp, const T *__restrict__ b,
    const T *__restrict__ dinv, TZ *__restrict__ z, const double *__restrict__ r64,
    const double *__restrict__ qold, double *partials, Ctl *ctl) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    RowOf<U, STREAM, IDX, T> R;
    T di = 0;
    if (i < n) {
        R.load(sptr, col, val, i, upat);
        di = ldg(dinv + i);
    }
    pdl_enter();
    xp = after_wait(xp);
    b = after_wait(b);
    r64 = after_wait(r64);
    qold = after_wait(qold);
    ctl = after_wait(ctl);
    if (ctl->done) return;
    double rz = 0.0, zq = 0.0;
    for (; i < n; i += stride) {
        T acc = R.dot(i, [&](int j) { return ldg(xp + j); });
        TZ zo = (TZ)(ldg(xp + i) + di * (ldg(b + i) - acc));
        z[i] = zo;
        if (DOT) {
            rz += ldg(r64 + i) * (double)zo;
            if (FCG) zq += (double)zo * ldg(qold + i);
        }
        if (i + stride < n) {
            R.load(sptr, col, val, i + stride, upat);
            di = ldg(dinv + i + stride);
        }
    }
    if (DOT) {
        if (publish_partials(rz, zq, partials, &ctl->counter[0])) {
            double a, bb;
            final_sum2(partials, a, bb);
            if (threadIdx.x == 0) finish_rho(ctl, a, bb);
        }
    }
}

// ------------------------------------------------------------ shared pieces
// b_c[I] = sum of t over the members of aggregate I, in increasing index
// order; PRE also forms xpre_c = dinv_c b_c for the next float64 down sweep.
template <typename T, typename TO, bool PRE>
__global__ void __launch_bounds__(kBlock) k_restrict(int nc, const int32_t *__restrict__ rptr,
                                                     const int32_t *__restrict__ ridx, const T *__restrict__ t,
                                                     TO *__restrict__ bc, const T *__restrict__ dinvc,
                                                     T *__restrict__ xprec, const Ctl *__restrict__ ctl) {
    constexpr int M = 4;  // members read before the wait
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t k0 = 0, k1 = 0;
    int m[M];
    T dc = 0;
    if (I < nc) {
        k0 = ldg(rptr + I);
        k1 = ldg(rptr + I + 1);
#pragma unroll
        for (int u = 0; u < M; u++) m[u] = k0 + u < k1 ? ldg(ridx + k0 + u) : 0;
        if (PRE) dc = ldg(dinvc + I);
    }
    pdl_enter();
    t = after_wait(t);
    ctl = after_wait(ctl);
    if (ctl->done || I >= nc) return;
    T tv[M];
#pragma unroll
    for (int u = 0; u < M; u++) tv[u] = k0 + u < k1 ? ldg(t + m[u]) : T(0);
    T s = 0;
#pragma unroll
    for (int u = 0; u < M; u++)
        if (k0 + u < k1) s += tv[u];
    for (int32_t k = k0 + M; k < k1; k++) s += ldg(t + ldg(ridx + k));
    bc[I] = (TO)s;
    if (PRE) xprec[I] = dc * s;
}

// Smoothed aggregation: b_c[I] = sum over the rows i of P's column I
// (increasing i) of P_iI res_i, res = b - A xpre left by the down sweep
// (launched with unit weights); PRE also forms xpre_c = dinv_c b_c.
template <typename T, typename TO, bool PRE>
__global__ void __launch_bounds__(kBlock) k_restrict_sa(int nc, const int32_t *__restrict__ trp,
                                                        const int32_t *__restrict__ tri, const T *__restrict__ tv,
                                                        const T *__restrict__ res, TO *__restrict__ bc,
                                                        const T *__restrict__ dinvc, T *__restrict__ xprec,
                                                        const Ctl *__restrict__ ctl) {
    pdl_enter();
    if (ctl->done) return;
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    T s = 0;
    for (int32_t q = ldg(trp + I); q < ldg(trp + I + 1); q++) s += ldg(tv + q) * ldg(res + ldg(tri + q));
    bc[I] = (TO)s;
    if (PRE) xprec[I] = ldg(dinvc + I) * s;
}

// Smoothed aggregation: xp_i = xpre_i + sum over row i of P of P_iJ xc_J.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_prolong_sa(int n, const int32_t *__restrict__ prp,
                                                       const int32_t *__restrict__ pci, const T *__restrict__ pv,
                                                       const T *__restrict__ xpre, const T *__restrict__ xc,
                                                       T *__restrict__ xp, const Ctl *__restrict__ ctl) {
    pdl_enter();
    if (ctl->done) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T s = 0;
        for (int32_t q = ldg(prp + i); q < ldg(prp + i + 1); q++) s += ldg(pv + q) * ldg(xc + ldg(pci + q));
        xp[i] = ldg(xpre + i) + s;
    }
}

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Down sweep fused with the restriction it feeds, one thread per coarse row
// I: t_i = p_i (b_i - sum_j a_ij xpre_j) for each member i of aggregate I
// (members in increasing index order), summed into b_c[I] (and, with PRE,
// xpre_c = dinv_c b_c). Same arithmetic, in the same order, as k_down
// followed by k_restrict; t is never stored.
template <typename T, typename TO, bool PRE, typename IDX, int U>
__global__ void __launch_bounds__(kBlock) k_down_restrict(int nc, const int32_t *__restrict__ rptr,
                                                          const int32_t *__restrict__ ridx,
                                                          const int32_t *__restrict__ sptr,
                                                          const IDX *__restrict__ col, const T *__restrict__ val,
                                                          const T *__restrict__ xpre, const T *__restrict__ b,
                                                          const T *__restrict__ p, TO *__restrict__ bc,
                                                          const T *__restrict__ dinvc, T *__restrict__ xprec,
                                                          const Ctl *__restrict__ ctl) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t q0 = 0, q1 = 0;
    int i = 0;
    SellRow<U, false, IDX, T> R;
    T pi = 0;
    if (I < nc) {
        q0 = ldg(rptr + I);
        q1 = ldg(rptr + I + 1);
        if (q0 < q1) {
            i = ldg(ridx + q0);
            R.load(sptr, col, val, i);
            pi = ldg(p + i);
        }
    }
    pdl_enter();
    xpre = after_wait(xpre);
    b = after_wait(b);
    ctl = after_wait(ctl);
    if (ctl->done || I >= nc) return;
    T sum = 0;
    for (int32_t q = q0; q < q1; q++) {
        T acc = R.dot(i, [&](int j) { return ldg(xpre + j); });
        // rounded product (never contracted into the sum), as k_down stores t
        T t = mul_rn(pi, ldg(b + i) - acc);
        sum += t;
        if (q + 1 < q1) {
            i = ldg(ridx + q + 1);
            R.load(sptr, col, val, i);
            pi = ldg(p + i);
        }
    }
    bc[I] = (TO)sum;
    if (PRE) xprec[I] = ldg(dinvc + I) * sum;
}

// Prolongation fused into the post sweep: xp_j = xpre_j + p_j x_c[agg_j] is
// formed for every gathered entry (and for the row itself), then
// z_i = xp_i + dinv_i (b_i - sum_j a_ij xp_j). Same values as k_prolong
// followed by k_post; xp is never stored.
template <typename T, typename IDX, int U>
__global__ void __launch_bounds__(kBlock) k_prolong_post(int n, const int32_t *__restrict__ sptr,
                                                         const IDX *__restrict__ col, const T *__restrict__ val,
                                                         const T *__restrict__ xpre, const T *__restrict__ p,
                                                         const int32_t *__restrict__ agg, const T *__restrict__ xc,
                                                         const T *__restrict__ b, const T *__restrict__ dinv,
                                                         T *__restrict__ z, const Ctl *__restrict__ ctl) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    SellRow<U, false, IDX, T> R;
    T di = 0;
    if (i < n) {
        R.load(sptr, col, val, i);
        di = ldg(dinv + i);
    }
    pdl_enter();
    xpre = after_wait(xpre);
    xc = after_wait(xc);
    b = after_wait(b);
    ctl = after_wait(ctl);
    if (ctl->done) return;
    auto xp = [&](int j) {
        T x = ldg(xpre + j);
        int a = ldg(agg + j);
        if (a >= 0) x += ldg(p + j) * ldg(xc + a);
        return x;
    };
    for (; i < n; i += stride) {
        T acc = R.dot(i, xp);
        z[i] = xp(i) + di * (ldg(b + i) - acc);
        if (i + stride < n) {
            R.load(sptr, col, val, i + stride);
            di = ldg(dinv + i + stride);
        }
    }
}

// ------------------------------------------------------------ hybrid Gauss-Seidel
// One sweep of the l1 hybrid Gauss-Seidel smoother (Sec. 3.1, l1 reading):
// xn = xo + M^{-1} (b - A xo), M = blockdiag(L_pp + D_l1) for FWD (rows of a
// block in increasing order) or its transpose (decreasing order). One thread
// per block of nb contiguous rows: it first copies its rows of xo into xn,
// then updates them in order, reading its own block's values from xn (the
// ones already updated) and every other block's from xo (block Jacobi).
// ZERO: xo = 0 (the first pre-smoothing sweep), x_r = d_r (b_r - acc).
// Entries are summed in storage order; with one row per block and one sweep
// the values are those of the l1-Jacobi sweeps (k_down's xpre, k_post).
template <typename T, bool FWD, bool ZERO>
__global__ void __launch_bounds__(kBlock) k_gs_sweep(int n, int nb, const int32_t *__restrict__ rp,
                                                     const int32_t *__restrict__ ci, const T *__restrict__ v,
                                                     const T *__restrict__ dinv, const T *__restrict__ b,
                                                     const T *__restrict__ xo, T *xn, const Ctl *__restrict__ ctl) {
    pdl_enter();
    if (ctl->done) return;
    int64_t lo64 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * nb;
    if (lo64 >= n) return;
    const int lo = (int)lo64, hi = (int)min((int64_t)n, lo64 + nb);
    for (int r = lo; r < hi; r++) xn[r] = ZERO ? T(0) : ldg(xo + r);
    for (int q = 0; q < hi - lo; q++) {
        const int r = FWD ? lo + q : hi - 1 - q;
        T acc = 0;
        const int32_t e = ldg(rp + r + 1);
        for (int32_t k = ldg(rp + r); k < e; k++) {
            const int j = ldg(ci + k);
            T xj = (j >= lo && j < hi) ? xn[j] : (ZERO ? T(0) : ldg(xo + j));
            acc += ldg(v + k) * xj;
        }
        if (ZERO)
            xn[r] = ldg(dinv + r) * (ldg(b + r) - acc);
        else
            xn[r] = xn[r] + ldg(dinv + r) * (ldg(b + r) - acc);
    }
}

// Two-phase form of the same sweep, for blocks of at most 32 rows. Phase one,
// one thread per row over the sliced-ELL layout: acc_r = sum of a_rj x_old_j
// over every entry of row r except the in-block ones the pass has already
// updated when it reaches r (FWD: j in [lo, r); backward: j in (r, hi)),
// which contribute 0 here. Phase two, one thread per block: the recurrence
// over those entries alone (k_gs_block). Same values as k_gs_sweep up to the
// order of the sums; with one row per block the sums are k_post's.
template <typename T, typename IDX, int U, bool FWD, bool STREAM>
__global__ void __launch_bounds__(kBlock, Occ<T>::kMinBlocks) k_gs_offsum(
    int n, int nb, const int32_t *__restrict__ sptr, const IDX *__restrict__ col, const T *__restrict__ val,
    const T *__restrict__ xo, T *__restrict__ acc, const Ctl *__restrict__ ctl) {
    pdl_enter();
    if (ctl->done) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        SELL_ROW_BEGIN
        const int lo = (i / nb) * nb, hi = min(n, lo + nb);
        T a = sell_row<U, STREAM>(c_, a_, w_, i, [&](int j) {
            bool done = FWD ? (j >= lo && j < i) : (j > i && j < hi);
            return done ? T(0) : ldg(xo + j);
        });
        acc[i] = a;
    }
}

constexpr int kGsThreads = 128;  // threads per CTA of k_gs_block (window: 33 values each)

// Phase two: one thread per block of nb <= 32 rows, rows in pass order. The
// block's new values live in a shared-memory window (33-value stride per
// thread, so threads at the same row offset use different banks);
// x_r = x_old_r + d_r (b_r - (acc_r + sum over the row's part entries of
// a_rj x_new_j)). ZERO (first pre-smoothing pass, x_old = 0): acc = 0 and
// x_r = d_r (b_r - sum).
template <typename T, bool FWD, bool ZERO>
__global__ void __launch_bounds__(kGsThreads) k_gs_block(int n, int nb, int w, const int32_t *__restrict__ pci,
                                                         const T *__restrict__ pv, const T *__restrict__ dinv,
                                                         const T *__restrict__ b, const T *__restrict__ xo,
                                                         const T *__restrict__ acc, T *__restrict__ xn,
                                                         const Ctl *__restrict__ ctl) {
    __shared__ T win[kGsThreads * 33];
    pdl_enter();
    if (ctl->done) return;
    int64_t lo64 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * nb;
    if (lo64 >= n) return;
    const int lo = (int)lo64, hi = (int)min((int64_t)n, lo64 + nb);
    T *wv = win + threadIdx.x * 33;
    for (int q = 0; q < hi - lo; q++) {
        const int r = FWD ? lo + q : hi - 1 - q;
        T sum = ZERO ? T(0) : ldg(acc + r);
        const int64_t e = (int64_t)r * w;
        for (int k = 0; k < w; k++) {
            const int j = ldg(pci + e + k);
            if (j >= 0) sum += ldg(pv + e + k) * wv[j - lo];
        }
        T x;
        if (ZERO)
            x = ldg(dinv + r) * (ldg(b + r) - sum);
        else
            x = ldg(xo + r) + ldg(dinv + r) * (ldg(b + r) - sum);
        wv[r - lo] = x;
        xn[r] = x;
    }
}

// Both phases of a sweep in one warp per 32-row slice, for blocks whose size
// divides 32 (so no block crosses a slice) and rows with at most kGsPart
// already-updated in-block entries. Phase one as in k_gs_offsum, one lane per
// row; phase two over the slice in 32 steps in pass order (FWD: rows
// increasing, else decreasing): at step t lane t finishes its row,
// x_t = x_old_t + d_t (b_t - acc_t), the value is broadcast by a shuffle, and
// every lane whose next in-block entry (in pass order) is column t adds
// a_rt x_t to its acc. Blocks of fewer rows run side by side in the same
// steps. Same values as k_gs_block up to the order of the sums.
constexpr int kGsPartMax = 8;

template <typename T, typename IDX, int U, bool FWD, bool ZERO, bool STREAM>
__global__ void __launch_bounds__(kBlock, Occ<T>::kMinBlocks) k_gs_warp(
    int n, int nb, int w, const int32_t *__restrict__ sptr, const IDX *__restrict__ col, const T *__restrict__ val,
    const int32_t *__restrict__ pci, const T *__restrict__ pv, const T *__restrict__ dinv, const T *__restrict__ b,
    const T *__restrict__ xo, T *__restrict__ xn, const Ctl *__restrict__ ctl) {
    pdl_enter();
    if (ctl->done) return;
    const int lane = threadIdx.x & 31;
    const int nsl = (n + 31) >> 5;
    const int wstride = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int sl = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); sl < nsl; sl += wstride) {
        const int i = (sl << 5) + lane;
        const bool valid = i < n;
        T acc = 0;
        if (!ZERO && valid) {
            const int lo = (i / nb) * nb, hi = min(n, lo + nb);
            SELL_ROW_BEGIN
            acc = sell_row<U, STREAM>(c_, a_, w_, i, [&](int j) {
                bool done = FWD ? (j >= lo && j < i) : (j > i && j < hi);
                return done ? T(0) : ldg(xo + j);
            });
        }
        // the row's in-block entries in pass order (padding -1 never matches)
        int rj[kGsPartMax];
        T ra[kGsPartMax];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < kGsPartMax; k++) {
            bool ok = valid && k < w;
            rj[k] = ok ? ldg(pci + (int64_t)i * w + k) : -1;
            ra[k] = ok ? ldg(pv + (int64_t)i * w + k) : T(0);
            cnt += rj[k] >= 0 ? 1 : 0;
        }
        int pj[kGsPartMax];
        T pa[kGsPartMax];
#pragma unroll
        for (int k = 0; k < kGsPartMax; k++) {
            if (FWD) {
                pj[k] = rj[k];
                pa[k] = ra[k];
            } else {
                pj[k] = -1;
                pa[k] = T(0);
#pragma unroll
                for (int m = 0; m < kGsPartMax; m++)
                    if (m == cnt - 1 - k) {
                        pj[k] = rj[m];
                        pa[k] = ra[m];
                    }
            }
        }
        const T bi = valid ? ldg(b + i) : T(0), di = valid ? ldg(dinv + i) : T(0);
        const T xold = (!ZERO && valid) ? ldg(xo + i) : T(0);
        T x = 0;
#pragma unroll 4
        for (int step = 0; step < 32; step++) {
            const int t = FWD ? step : 31 - step;
            if (lane == t) x = ZERO ? di * (bi - acc) : xold + di * (bi - acc);
            const T xt = __shfl_sync(0xffffffffu, x, t);
            if (pj[0] == (sl << 5) + t) {
                acc += pa[0] * xt;
#pragma unroll
                for (int k = 0; k + 1 < kGsPartMax; k++) {
                    pj[k] = pj[k + 1];
                    pa[k] = pa[k + 1];
                }
                pj[kGsPartMax - 1] = -1;
            }
        }
        if (valid) xn[i] = x;
    }
}

// Level 0 after the Gauss-Seidel post-smoothing: z = x (widened), r.z and,
// for FCG(1), z.q_old; the last block forms rho and beta. Same grid and row
// order as the level-0 k_post, so the sums are formed in the same order.
template <typename T, bool FCG>
__global__ void __launch_bounds__(kBlock, Occ<T>::kMinBlocks) k_gs_finish0(int n, const T *__restrict__ x,
                                                                           const double *__restrict__ r64,
                                                                           const double *__restrict__ qold,
                                                                           double *__restrict__ z, double *partials,
                                                                           Ctl *ctl) {
    pdl_enter();
    if (ctl->done) return;
    double rz = 0.0, zq = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double zo = (double)ldg(x + i);
        z[i] = zo;
        rz += ldg(r64 + i) * zo;
        if (FCG) zq += zo * ldg(qold + i);
    }
    if (publish_partials(rz, zq, partials, &ctl->counter[0])) {
        double a, bb;
        final_sum2(partials, a, bb);
        if (threadIdx.x == 0) finish_rho(ctl, a, bb);
    }
}

// x_L = A_L^{-1} b_L, one warp per row; TO = float rounds the float64 result.
template <typename TO>
__global__ void __launch_bounds__(kBlock) k_coarse(int nL, const double *__restrict__ ainv,
                                                   const double *__restrict__ bL, TO *__restrict__ xL,
                                                   const Ctl *__restrict__ ctl) {
    pdl_enter();
    if (ctl->done) return;
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= nL) return;
    const double *a = ainv + (int64_t)row * nL;
    double s = 0.0;
    for (int j = lane; j < nL; j += 32) s += ldg(a + j) * ldg(bL + j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) xL[row] = (TO)s;
}

// Single-level hierarchy: z = A^{-1} r (through float32 as the float32
// V-cycle would round it when F32), then r.z / z.q_old as on level 0.
template <bool F32, bool FCG>
__global__ void __launch_bounds__(kBlock) k_coarse_only(int n, const double *__restrict__ ainv,
                                                        const double *__restrict__ r, double *__restrict__ z,
                                                        const double *__restrict__ qold, double *partials,
                                                        Ctl *ctl) {
    pdl_enter();
    if (ctl->done) return;
    double rz = 0.0, zq = 0.0;
    int lane = threadIdx.x & 31;
    int wpb = blockDim.x >> 5;
    for (int row = blockIdx.x * wpb + (threadIdx.x >> 5); row < n; row += gridDim.x * wpb) {
        const double *a = ainv + (int64_t)row * n;
        double s = 0.0;
        for (int j = lane; j < n; j += 32) {
            double rj = ldg(r + j);
            if (F32) rj = (double)(float)rj;
            s += ldg(a + j) * rj;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            double zo = F32 ? (double)(float)s : s;
            z[row] = zo;
            rz += r[row] * zo;
            if (FCG) zq += zo * qold[row];
        }
    }
    if (publish_partials(rz, zq, partials, &ctl->counter[0])) {
        double a, bb;
        final_sum2(partials, a, bb);
        if (threadIdx.x == 0) finish_rho(ctl, a, bb);
    }
}

// ------------------------------------------------------------ Krylov kernels
// p = z + beta p (beta = 0 on a restart gives p = z).
__global__ void __launch_bounds__(kBlock) k_axpy_p(int n, const double *__restrict__ z, double *__restrict__ p,
                                                   const Ctl *__restrict__ ctl) {
    pdl_enter();
    if (ctl->done) return;
    double beta = ctl->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

// q = A p and p.q; the last block forms alpha = rho / p.q.
template <typename IDX>
__global__ void __launch_bounds__(kBlock, 4) k_spmv(int n, const int32_t *__restrict__ sptr,
                                                    const IDX *__restrict__ col, const double *__restrict__ val,
                                                    const IDX *__restrict__ upat, const double *__restrict__ p,
                                                    double *__restrict__ q, double *partials, Ctl *ctl) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    SellRow<kUnroll, true, IDX, double> R;
    if (i < n) R.load(sptr, col, val, i, upat);
    pdl_enter();
    p = after_wait(p);
    ctl = after_wait(ctl);
    if (ctl->done) return;
    double pq = 0.0;
    for (; i < n; i += stride) {
        double acc = R.dot(i, [&](int j) { return ldg(p + j); });
        q[i] = acc;
        pq += ldg(p + i) * acc;
        if (i + stride < n) R.load(sptr, col, val, i + stride, upat);
    }
    if (publish_partials(pq, 0.0, partials, &ctl->counter[1])) {
        double a, unused;
        final_sum2(partials, a, unused);
        if (threadIdx.x == 0) {
            ctl->counter[1] = 0;
            if (!isfinite(a)) { fail(ctl, AMG_ERR_NAN); return; }
            if (!(a > 0.0)) { fail(ctl, AMG_ERR_BREAKDOWN); return; }
            ctl->pq = a;
            ctl->alpha = ctl->rho / a;
        }
    }
}

// What the V-cycle of the mode reads besides r: FCG32 a float32 copy of r
// and xpre_0 = D_0^{-1} r in float32 (as the float32 V-cycle forms them);
// PCG64 xpre_0 = D_0^{-1} r in float64.
struct REmit {
    float *r32;
    const float *dinv32;
    float *xpre32;
    const double *dinv64;
    double *xpre64;
};

template <int MODE>
__device__ __forceinline__ void emit_r(int i, double ri, const REmit &e) {
    if (MODE == AMG_MODE_FCG32) {
        float r = (float)ri;
        e.r32[i] = r;
        e.xpre32[i] = ldg(e.dinv32 + i) * r;
    } else {
        e.xpre64[i] = ldg(e.dinv64 + i) * ri;
    }
}

// x += alpha p, r -= alpha q, ||r||^2; the last block records the relative
// residual, advances the iteration and decides whether to check the true one.
template <int MODE>
__global__ void __launch_bounds__(kBlock) k_update(int n, const double *__restrict__ p,
                                                   const double *__restrict__ q, double *__restrict__ x,
                                                   double *__restrict__ r, REmit em, double *partials, Ctl *ctl,
                                                   double *hist) {
    pdl_enter();
    if (ctl->done) return;
    double alpha = ctl->alpha;
    double rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = x[i] + alpha * p[i];
        double ri = r[i] - alpha * q[i];
        r[i] = ri;
        emit_r<MODE>(i, ri, em);
        rr += ri * ri;
    }
    if (publish_partials(rr, 0.0, partials, &ctl->counter[2])) {
        double a, unused;
        final_sum2(partials, a, unused);
        if (threadIdx.x == 0) {
            ctl->counter[2] = 0;
            int it = ctl->iter + 1;
            ctl->iter = it;
            double rel = sqrt(a) / ctl->bnorm;
            ctl->rel = rel;
            hist[it] = rel;
            ctl->rho_old = ctl->rho;
            ctl->pq_old = ctl->pq;
            ctl->restart = 0;
            if (!isfinite(rel)) { fail(ctl, AMG_ERR_NAN); return; }
            if (rel <= ctl->rtol) ctl->check = 1;
            else if (it >= ctl->maxit) fail(ctl, AMG_ERR_NOCONV);
        }
    }
}

// r = b - A x, ||r||^2 (and ||b||^2 on INIT); also the mode's copy of r.
// Otherwise (not INIT) it runs only when the recursive residual met rtol.
template <bool INIT, int MODE, typename IDX>
__global__ void __launch_bounds__(kBlock, 4) k_residual(int n, const int32_t *__restrict__ sptr,
                                                        const IDX *__restrict__ col,
                                                        const double *__restrict__ val, const double *__restrict__ b,
                                                        const double *__restrict__ x, double *__restrict__ r,
                                                        REmit em, double *partials, Ctl *ctl, double *hist) {
    pdl_enter();
    if (ctl->done) return;
    if (!INIT && !ctl->check) return;
    double rr = 0.0, bb = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        SELL_ROW_BEGIN
        double acc = sell_row<kUnroll, true>(c_, a_, w_, i, [&](int j) { return ldg(x + j); });
        double bi = ldg(b + i);
        double ri = bi - acc;
        r[i] = ri;
        emit_r<MODE>(i, ri, em);
        rr += ri * ri;
        if (INIT) bb += bi * bi;
    }
    if (publish_partials(rr, bb, partials, &ctl->counter[3])) {
        double a, bsq;
        final_sum2(partials, a, bsq);
        if (threadIdx.x == 0) {
            ctl->counter[3] = 0;
            if (INIT) {
                double bn = sqrt(bsq);
                ctl->bnorm = bn;
                if (!isfinite(bn) || !isfinite(a)) { fail(ctl, AMG_ERR_NAN); return; }
                if (bn == 0.0) { ctl->done = 1; ctl->status = AMG_OK; ctl->true_rel = 0.0; hist[0] = 0.0; return; }
                double rel = sqrt(a) / bn;
                ctl->rel = rel;
                ctl->true_rel = rel;
                hist[0] = rel;
                if (rel <= ctl->rtol) { ctl->done = 1; ctl->status = AMG_OK; }
                else if (ctl->maxit <= 0) fail(ctl, AMG_ERR_NOCONV);
            } else {
                double rel = sqrt(a) / ctl->bnorm;
                ctl->true_rel = rel;
                ctl->check = 0;
                if (!isfinite(rel)) { fail(ctl, AMG_ERR_NAN); return; }
                if (rel <= ctl->rtol) { ctl->done = 1; ctl->status = AMG_OK; return; }
                ctl->restart = 1;
                hist[ctl->iter] = rel;
                if (ctl->iter >= ctl->maxit) fail(ctl, AMG_ERR_NOCONV);
            }
        }
    }
}

__global__ void k_zero(double *a, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 0.0;
}

// Loop condition of the solve graph: run another body while not done. The
// body count is bounded independently of the kernels' own bookkeeping: past
// (maxit + 1) / 2 + 1 bodies the solve is ended as not converged.
__global__ void k_set_cond(cudaGraphConditionalHandle hc, Ctl *ctl, int count_body) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (count_body) {
        int b = ctl->bodies + 1;
        ctl->bodies = b;
        if (!ctl->done && b > (ctl->maxit + 1) / 2 + 1) {
            ctl->done = 2;
            ctl->status = AMG_ERR_NOCONV;
        }
    }
    cudaGraphSetConditional(hc, ctl->done ? 0u : 1u);
}

inline int grid_rows(int64_t n) { return (int)((n + kBlock - 1) / kBlock); }


// ------------------------------------------------------------ profiling
// CUDA-event spans around kernel launches (only when profiling is on).
// kinds: 0 down0, 1 post0 (the whole up phase of level 0 with the
// Gauss-Seidel smoother), 2 q = A p, 3 update, 4 true residual, 5 levels >= 1
// and the coarsest solve, 6 p = z + beta p, 7 prolong0.
constexpr int kEvPairs = 256;

// Opens a span of `kind` (kinds < kKinds: the kernel kinds above; kinds
// kLevelSpan + 3 l + phase: level l's down (0: down + restriction), up (1:
// prolongation + post) or coarsest (2) phase). Returns the span's slot or -1.
constexpr int kLevelSpan = 100;

int prof_begin(amg_hier *h, int kind, cudaStream_t s) {
    if (!h->profile || h->ev_used + 2 > (int)h->ev.size()) return -1;
    int slot = h->ev_used;
    h->ev_kind[slot / 2] = kind;
    cudaEventRecord(h->ev[slot], s);
    h->ev_used += 2;
    return slot;
}

void prof_end(amg_hier *h, int slot, cudaStream_t s) {
    if (slot < 0) return;
    cudaEventRecord(h->ev[slot + 1], s);
}

// Fold the recorded spans into the totals (stream already synchronised).
void prof_collect(amg_hier *h) {
    for (int k = 0; k + 1 < h->ev_used; k += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]) != cudaSuccess) continue;
        int kind = h->ev_kind[k / 2];
        if (kind >= kLevelSpan) {
            int l = (kind - kLevelSpan) / 3, ph = (kind - kLevelSpan) % 3;
            if (l < amg_hier::kMaxProfLevels) {
                h->lev_ms[l][ph] += ms;
                h->lev_n[l][ph] += 1;
            }
        } else {
            h->prof_ms[kind] += ms;
            h->prof_n[kind] += 1;
        }
    }
    h->ev_used = 0;
}

// ------------------------------------------------------------ one iteration
template <typename T>
struct LP;
template <>
struct LP<float> {
    static const float *val(const Level &l) { return l.S.v32; }
    static const float *dinv(const Level &l) { return l.dinv32; }
    static const float *p(const Level &l) { return l.p32; }
    static float *b(Level &l) { return l.b32; }
    static float *x(Level &l) { return l.x32; }
    static float *t(Level &l) { return l.t32; }
    static float *xpre(Level &l) { return l.xpre32; }
    static float *xp(Level &l) { return l.xp32; }
    static const float *r0(const amg_hier *h) { return h->r32; }
    static const float *Pv(const Level &l) { return l.P32; }
    static const float *Ptv(const Level &l) { return l.Pt32; }
    static const float *ones(const Level &l) { return l.ones32; }
    static const float *csr(const Level &l) { return l.v32csr; }
    static const float *part(const Level &l, int d) { return l.gs_v32[d]; }
    static float *acc(const Level &l) { return reinterpret_cast<float *>(l.gs_acc); }
};
template <>
struct LP<double> {
    static const double *val(const Level &l) { return l.S.v64; }
    static const double *dinv(const Level &l) { return l.dinv; }
    static const double *p(const Level &l) { return l.p; }
    static double *b(Level &l) { return l.b64; }
    static double *x(Level &l) { return l.x64; }
    static double *t(Level &l) { return l.t64; }
    static double *xpre(Level &l) { return l.xpre64; }
    static double *xp(Level &l) { return l.xp64; }
    static const double *r0(const amg_hier *h) { return h->r; }
    static const double *Pv(const Level &l) { return l.P.v; }
    static const double *Ptv(const Level &l) { return l.Pt.v; }
    static const double *ones(const Level &l) { return l.ones64; }
    static const double *csr(const Level &l) { return l.A.v; }
    static const double *part(const Level &l, int d) { return l.gs_v64[d]; }
    static double *acc(const Level &l) { return l.gs_acc; }
};

REmit remit(amg_hier *h) {
    Level &l0 = h->lev[0];
    return REmit{h->r32, l0.dinv32, l0.xpre32, l0.dinv, l0.xpre64};
}

// Launch with the level's column array: int16 offsets when present.
// BODY sees IDX (the column type), cols (the columns) and pats (the shared
// offset patterns in the column type, or null).
#define WITH_COLS(S, BODY)                          \
    do {                                            \
        if ((S).col16) {                            \
            using IDX = int16_t;                    \
            const IDX *cols = (S).col16;            \
            [[maybe_unused]] const IDX *pats = (S).upat16; \
            BODY;                                   \
        } else {                                    \
            using IDX = int32_t;                    \
            const IDX *cols = (S).col;              \
            [[maybe_unused]] const IDX *pats = (S).upat; \
            BODY;                                   \
        }                                           \
    } while (0)

template <typename T>
constexpr int prec_index() { return sizeof(T) == 4 ? 0 : 1; }

int shape_grid(const amg_hier *h, int n, int pi, int sweep, unsigned char shape) {
    int g = grid_rows(n);
    if (shape & 2) return g;
    int w = h->wave[pi][sweep][shape & 1];
    return w > 0 && w < g ? w : g;
}

// Weight of the down sweep's output t = w (b - A xpre): the tentative
// prolongator's p (restriction by the aggregate map), or ones with
// smoothed aggregation (the restriction then applies P^T).
template <typename T>
const T *pdown(const amg_hier *h, const Level &lv) {
    return h->smoothed ? LP<T>::ones(lv) : LP<T>::p(lv);
}

// Prolongation to level l: xp = xpre + P x_{l+1} (through the aggregate map,
// or the explicit smoothed P).
template <typename T>
void launch_prolong(amg_hier *h, int l, int grid, cudaStream_t s) {
    using P = LP<T>;
    auto &lev = h->lev;
    Level &lv = lev[l];
    int n = lv.A.n;
    if (h->smoothed)
        launch_k(h->pdl, k_prolong_sa<T>, grid, kBlock, s, n, (const int32_t *)lv.P.rp, (const int32_t *)lv.P.ci,
                 P::Pv(lv), (const T *)P::xpre(lv), (const T *)P::x(lev[l + 1]), P::xp(lv), (const Ctl *)h->ctl);
    else
        launch_k(h->pdl, k_prolong<T>, grid, kBlock, s, n, (const T *)P::xpre(lv), P::p(lv), lv.agg,
                 (const T *)P::x(lev[l + 1]), P::xp(lv), (const Ctl *)h->ctl);
}

// Down sweep of level l >= 1 with the given launch shape (bits 0 and 1).
template <typename T>
void launch_down(amg_hier *h, int l, unsigned char shape, cudaStream_t s) {
    using P = LP<T>;
    Level &lv = h->lev[l];
    int n = lv.A.n;
    if (shape & 8) {
        WITH_COLS(lv.S, (launch_k(h->pdl, k_down_ml<T, IDX>, grid_rows((int64_t)n * kMlL), kBlock, s, n, lv.S.sptr,
                                  cols, P::val(lv), (const T *)P::xpre(lv), (const T *)P::b(lv), pdown<T>(h, lv),
                                  P::t(lv), (const Ctl *)h->ctl)));
        return;
    }
    int g = shape_grid(h, n, prec_index<T>(), 0, shape);
    if (shape & 1)
        WITH_COLS(lv.S, (launch_k(h->pdl, k_down<T, IDX, kUnrollSmall, false>, g, kBlock, s, n, lv.S.sptr, cols,
                                  P::val(lv), pats, P::xpre(lv), P::b(lv), pdown<T>(h, lv), P::t(lv), (const Ctl *)h->ctl)));
    else
        WITH_COLS(lv.S, (launch_k(h->pdl, k_down<T, IDX, kUnroll, false>, g, kBlock, s, n, lv.S.sptr, cols,
                                  P::val(lv), pats, P::xpre(lv), P::b(lv), pdown<T>(h, lv), P::t(lv), (const Ctl *)h->ctl)));
}

// Restriction from level l to l+1 (the coarsest gets float64 b_L).
template <typename T>
void launch_restrict(amg_hier *h, int l, cudaStream_t s) {
    using P = LP<T>;
    auto &lev = h->lev;
    Level &lv = lev[l];
    const Ctl *ctl = h->ctl;
    if (h->smoothed) {
        if (l + 2 == (int)lev.size())
            launch_k(h->pdl, k_restrict_sa<T, double, false>, grid_rows(lv.nc), kBlock, s, lv.nc,
                     (const int32_t *)lv.Pt.rp, (const int32_t *)lv.Pt.ci, P::Ptv(lv), (const T *)P::t(lv), h->bL,
                     (const T *)nullptr, (T *)nullptr, ctl);
        else
            launch_k(h->pdl, k_restrict_sa<T, T, true>, grid_rows(lv.nc), kBlock, s, lv.nc,
                     (const int32_t *)lv.Pt.rp, (const int32_t *)lv.Pt.ci, P::Ptv(lv), (const T *)P::t(lv),
                     P::b(lev[l + 1]), P::dinv(lev[l + 1]), P::xpre(lev[l + 1]), ctl);
        return;
    }
    if (l + 2 == (int)lev.size())
        launch_k(h->pdl, k_restrict<T, double, false>, grid_rows(lv.nc), kBlock, s, lv.nc, lv.rptr, lv.ridx,
                 (const T *)P::t(lv), h->bL, (const T *)nullptr, (T *)nullptr, ctl);
    else
        launch_k(h->pdl, k_restrict<T, T, true>, grid_rows(lv.nc), kBlock, s, lv.nc, lv.rptr, lv.ridx,
                 (const T *)P::t(lv), P::b(lev[l + 1]), P::dinv(lev[l + 1]), P::xpre(lev[l + 1]), ctl);
}

// Down phase of level l >= 1: down sweep then restriction, or (shape bit 2)
// both in one launch by aggregate.
template <typename T>
void launch_down_phase(amg_hier *h, int l, unsigned char shape, cudaStream_t s) {
    using P = LP<T>;
    if (!(shape & 4) || h->smoothed) {
        launch_down<T>(h, l, shape, s);
        launch_restrict<T>(h, l, s);
        return;
    }
    auto &lev = h->lev;
    Level &lv = lev[l];
    const Ctl *ctl = h->ctl;
    int g = grid_rows(lv.nc);
    bool last = l + 2 == (int)lev.size();
#define PCG_DR(U)                                                                                                   \
    do {                                                                                                            \
        if (last)                                                                                                   \
            WITH_COLS(lv.S, (launch_k(h->pdl, k_down_restrict<T, double, false, IDX, U>, g, kBlock, s, lv.nc,      \
                                      lv.rptr, lv.ridx, lv.S.sptr, cols, P::val(lv), P::xpre(lv), P::b(lv),         \
                                      P::p(lv), h->bL, (const T *)nullptr, (T *)nullptr, ctl)));                    \
        else                                                                                                        \
            WITH_COLS(lv.S, (launch_k(h->pdl, k_down_restrict<T, T, true, IDX, U>, g, kBlock, s, lv.nc, lv.rptr,   \
                                      lv.ridx, lv.S.sptr, cols, P::val(lv), P::xpre(lv), P::b(lv), P::p(lv),        \
                                      P::b(lev[l + 1]), P::dinv(lev[l + 1]), P::xpre(lev[l + 1]), ctl)));           \
    } while (0)
    if (shape & 1) PCG_DR(kUnrollSmall);
    else PCG_DR(kUnroll);
#undef PCG_DR
}

// Post sweep of level l >= 1 (z = x_l) with the given launch shape.
template <typename T>
void launch_post(amg_hier *h, int l, unsigned char shape, cudaStream_t s) {
    using P = LP<T>;
    Level &lv = h->lev[l];
    int n = lv.A.n;
    if (shape & 8) {
        WITH_COLS(lv.S, (launch_k(h->pdl, k_post_ml<T, IDX>, grid_rows((int64_t)n * kMlL), kBlock, s, n, lv.S.sptr,
                                  cols, P::val(lv), (const T *)P::xp(lv), (const T *)P::b(lv), P::dinv(lv), P::x(lv),
                                  (const Ctl *)h->ctl)));
        return;
    }
    int g = shape_grid(h, n, prec_index<T>(), 1, shape);
    if (shape & 1)
        WITH_COLS(lv.S, (launch_k(h->pdl, k_post<T, T, false, false, IDX, kUnrollSmall, false>, g, kBlock, s, n,
                                  lv.S.sptr, cols, P::val(lv), pats, P::xp(lv), P::b(lv), P::dinv(lv), P::x(lv),
                                  (const double *)nullptr, (const double *)nullptr, (double *)nullptr, h->ctl)));
    else
        WITH_COLS(lv.S, (launch_k(h->pdl, k_post<T, T, false, false, IDX, kUnroll, false>, g, kBlock, s, n,
                                  lv.S.sptr, cols, P::val(lv), pats, P::xp(lv), P::b(lv), P::dinv(lv), P::x(lv),
                                  (const double *)nullptr, (const double *)nullptr, (double *)nullptr, h->ctl)));
}

// Up phase of level l >= 1: prolongation then post sweep, or (shape bit 2)
// the prolongation formed per gathered entry inside the post sweep.
template <typename T>
void launch_up_phase(amg_hier *h, int l, unsigned char shape, cudaStream_t s) {
    using P = LP<T>;
    auto &lev = h->lev;
    Level &lv = lev[l];
    int n = lv.A.n;
    const Ctl *ctl = h->ctl;
    if (!(shape & 4) || h->smoothed) {
        launch_prolong<T>(h, l, grid_rows(n), s);
        launch_post<T>(h, l, shape, s);
        return;
    }
    int g = shape_grid(h, n, prec_index<T>(), 1, shape);
    if (shape & 1)
        WITH_COLS(lv.S, (launch_k(h->pdl, k_prolong_post<T, IDX, kUnrollSmall>, g, kBlock, s, n, lv.S.sptr, cols,
                                  P::val(lv), (const T *)P::xpre(lv), P::p(lv), lv.agg, (const T *)P::x(lev[l + 1]),
                                  (const T *)P::b(lv), P::dinv(lv), P::x(lv), ctl)));
    else
        WITH_COLS(lv.S, (launch_k(h->pdl, k_prolong_post<T, IDX, kUnroll>, g, kBlock, s, n, lv.S.sptr, cols,
                                  P::val(lv), (const T *)P::xpre(lv), P::p(lv), lv.agg, (const T *)P::x(lev[l + 1]),
                                  (const T *)P::b(lv), P::dinv(lv), P::x(lv), ctl)));
}

// Coarsest solve of the single-column V-cycle: x_L = A_L^{-1} b_L with the
// dense inverse, or the iterative solve (FCG + block-Jacobi ILU(1)). Adds
// the kernels launched to *kernels.
template <typename T>
int launch_coarsest(amg_hier *h, cudaStream_t s, int *kernels) {
    using P = LP<T>;
    Level &lc = h->lev.back();
    if (h->coarse_iter) {
        PCG_TRY(launch_coarse_iter<T>(h, h->cws, h->bL, P::x(lc), &h->ctl->done, nullptr, s));
        *kernels += coarse_iter_launches(h);
        return AMG_OK;
    }
    launch_k(h->pdl, k_coarse<T>, (h->nL * 32 + kBlock - 1) / kBlock, kBlock, s, h->nL, h->Ainv, h->bL, P::x(lc),
             (const Ctl *)h->ctl);
    *kernels += 1;
    return AMG_OK;
}

// One wave of the level-0 sweeps of precision T.
template <typename T>
int grid0(const amg_hier *h) { return sizeof(T) == 4 ? h->grid32 : h->grid64; }

// Float32 level-0 sweeps read whole rows at once where level 0 has shared
// offset patterns (PatRow), else 4-entry chunks.
inline bool pat_rows(const amg_hier *h) { return h->lev[0].S.upat != nullptr; }

// Level-0 down sweep t = p (b - A xpre) (evict-first matrix stream, shared
// offset patterns where level 0 has them).
template <typename T>
void launch_down0(amg_hier *h, const T *b0, cudaStream_t s) {
    using P = LP<T>;
    Level &l0 = h->lev[0];
    if constexpr (sizeof(T) == 4) {
        if (pat_rows(h)) {
            WITH_COLS(l0.S, (launch_k(h->pdl, k_down<T, IDX, kPatRow, true>, grid0<T>(h), kBlock, s, l0.A.n,
                                      l0.S.sptr, cols, P::val(l0), pats, (const T *)P::xpre(l0), b0,
                                      pdown<T>(h, l0), P::t(l0), (const Ctl *)h->ctl)));
            return;
        }
    }
    WITH_COLS(l0.S, (launch_k(h->pdl, k_down<T, IDX, kUnroll, true>, grid0<T>(h), kBlock, s, l0.A.n,
                                  l0.S.sptr, cols, P::val(l0), pats, (const T *)P::xpre(l0), b0, pdown<T>(h, l0),
                                  P::t(l0), (const Ctl *)h->ctl)));
}

// Level-0 post sweep z = xp + dinv (b - A xp) with r.z (and z.q_old).
template <typename T, bool FCG>
void launch_post0(amg_hier *h, const T *b0, cudaStream_t s) {
    using P = LP<T>;
    Level &l0 = h->lev[0];
    if constexpr (sizeof(T) == 4) {
        if (pat_rows(h)) {
            WITH_COLS(l0.S, (launch_k(h->pdl, k_post<T, double, true, FCG, IDX, kPatRow, true>, grid0<T>(h), kBlock,
                                      s, l0.A.n, l0.S.sptr, cols, P::val(l0), pats, P::xp(l0), b0, P::dinv(l0), h->z,
                                      h->r, h->q, h->partials, h->ctl)));
            return;
        }
    }
    WITH_COLS(l0.S, (launch_k(h->pdl, k_post<T, double, true, FCG, IDX, kUnroll, true>, grid0<T>(h), kBlock, s,
                                  l0.A.n, l0.S.sptr, cols, P::val(l0), pats, P::xp(l0), b0, P::dinv(l0), h->z, h->r,
                                  h->q, h->partials, h->ctl)));
}

// z = B r (one V-cycle in precision T), including rho / beta. Kernels are
// launched with programmatic dependent launch when h->pdl (see pdl_enter).
template <typename T, bool FCG>
int launch_vcycle(amg_hier *h, cudaStream_t s) {
    using P = LP<T>;
    auto &lev = h->lev;
    int L = (int)lev.size() - 1;
    const T *b0 = P::r0(h);
    int sp1 = prof_begin(h, 0, s);
    launch_down0<T>(h, b0, s);
    prof_end(h, sp1, s);
    int sp2 = prof_begin(h, 5, s);
    // levels handled by separate launches: 0..F-1; the tail runs F..L
    int tf = h->no_tail ? 0 : h->tail_first[prec_index<T>()];
    int F = tf > 0 ? tf : L;
    // per-level spans (profiling only): level l's down phase is its down
    // sweep and the restriction that leaves it (level 0: the restriction)
    int kernels = 1;  // down sweep of level 0
    for (int l = 0; l < F; l++) {
        Level &lv = lev[l];
        int spl = prof_begin(h, kLevelSpan + 3 * l, s);
        unsigned char sh = lv.shape[prec_index<T>()][0];
        if (l == 0) {
            launch_restrict<T>(h, 0, s);
            kernels += 1;
        } else {
            launch_down_phase<T>(h, l, sh, s);
            kernels += (sh & 4) ? 1 : 2;
        }
        prof_end(h, spl, s);
    }
    int spc = prof_begin(h, kLevelSpan + 3 * F + 2, s);
    if (F < L) {
        PCG_TRY(launch_smem_tail<T>(h, s));
        kernels += 1;
    } else {
        PCG_TRY(launch_coarsest<T>(h, s, &kernels));
    }
    prof_end(h, spc, s);
    for (int l = F - 1; l >= 1; l--) {
        Level &lv = lev[l];
        int spl = prof_begin(h, kLevelSpan + 3 * l + 1, s);
        unsigned char sh = lv.shape[prec_index<T>()][1];
        launch_up_phase<T>(h, l, sh, s);
        kernels += (sh & 4) ? 1 : 2;
        prof_end(h, spl, s);
    }
    kernels += 2;  // prolongation and post sweep of level 0
    prof_end(h, sp2, s);
    int sp7 = prof_begin(h, 7, s);
    launch_prolong<T>(h, 0, h->gridv, s);
    prof_end(h, sp7, s);
    int sp3 = prof_begin(h, 1, s);
    launch_post0<T, FCG>(h, b0, s);
    prof_end(h, sp3, s);
    h->launches += kernels;
    PCG_LAUNCH_CK();
    return AMG_OK;
}

// gs_nu Gauss-Seidel sweeps on level l: pre-smoothing (forward, from zero,
// into xpre) or post-smoothing (backward, from xp, into x). Successive sweeps
// alternate between the target and t (free at both points), arranged so the
// last one writes the target. A level with a two-phase table for the pass
// (blocks of at most 32 rows) sweeps with k_gs_offsum + k_gs_block (the first
// pre-smoothing pass with k_gs_block alone); any other with k_gs_sweep.
// Returns the kernels launched.
template <typename T>
int launch_gs(amg_hier *h, int l, bool pre, const T *b, T *target, cudaStream_t s) {
    using P = LP<T>;
    Level &lv = h->lev[l];
    const int n = lv.A.n, nu = h->gs_nu, nb = gs_rows(n, h->gs_blocks);
    const unsigned g = (unsigned)((((int64_t)n + nb - 1) / nb + kBlock - 1) / kBlock);
    const Ctl *ctl = h->ctl;
    const T *src = pre ? nullptr : (const T *)P::xp(lv);
    const int d = pre ? 0 : 1;  // the forward (pre) or backward (post) pass
    // float32 only: a float64 warp instruction occupies the float64 pipe for
    // all 32 lanes, and the one-warp recurrence issues two per step with one
    // lane active; k_gs_block keeps a block per lane instead
    if (sizeof(T) == 4 && lv.gs_w[d] >= 0 && lv.gs_w[d] <= kGsPartMax && nb <= 32 && 32 % nb == 0 &&
        h->gs_fused) {
        // both phases in one launch (one warp per slice)
        const int w = lv.gs_w[d];
        const int gr = grid_rows(n);
        const bool big = n > kSmallRows;
        const int32_t *pci = lv.gs_ci[d];
        const T *pv = P::part(lv, d);
        for (int sw = 1; sw <= nu; sw++) {
            T *dst = (nu - sw) % 2 == 0 ? target : P::t(lv);
            const bool zero = pre && sw == 1;
#define PCG_GSW(UU, ST)                                                                                            \
    do {                                                                                                            \
        if (zero)                                                                                                   \
            WITH_COLS(lv.S, (launch_k(h->pdl, k_gs_warp<T, IDX, UU, true, true, ST>, gr, kBlock, s, n, nb, w,       \
                                      lv.S.sptr, cols, P::val(lv), pci, pv, P::dinv(lv), b, src, dst, ctl)));       \
        else if (pre)                                                                                               \
            WITH_COLS(lv.S, (launch_k(h->pdl, k_gs_warp<T, IDX, UU, true, false, ST>, gr, kBlock, s, n, nb, w,      \
                                      lv.S.sptr, cols, P::val(lv), pci, pv, P::dinv(lv), b, src, dst, ctl)));       \
        else                                                                                                        \
            WITH_COLS(lv.S, (launch_k(h->pdl, k_gs_warp<T, IDX, UU, false, false, ST>, gr, kBlock, s, n, nb, w,     \
                                      lv.S.sptr, cols, P::val(lv), pci, pv, P::dinv(lv), b, src, dst, ctl)));       \
    } while (0)
            if (l == 0) PCG_GSW(kUnroll, true);
            else if (big) PCG_GSW(kUnroll, false);
            else PCG_GSW(kUnrollSmall, false);
#undef PCG_GSW
            src = dst;
        }
        return nu;
    }
    if (lv.gs_w[d] >= 0) {
        // two-phase sweeps
        const int w = lv.gs_w[d];
        const unsigned gb = (unsigned)((((int64_t)n + nb - 1) / nb + kGsThreads - 1) / kGsThreads);
        const int gr = grid_rows(n);
        const bool big = n > kSmallRows;
        int kernels = 0;
        for (int sw = 1; sw <= nu; sw++) {
            T *dst = (nu - sw) % 2 == 0 ? target : P::t(lv);
            const bool zero = pre && sw == 1;
            if (!zero) {
#define PCG_OFFSUM(UU, ST)                                                                                          \
    WITH_COLS(lv.S, (launch_k(h->pdl, k_gs_offsum<T, IDX, UU, true, ST>, gr, kBlock, s, n, nb, lv.S.sptr, cols,     \
                              P::val(lv), src, P::acc(lv), ctl)))
#define PCG_OFFSUM_B(UU, ST)                                                                                        \
    WITH_COLS(lv.S, (launch_k(h->pdl, k_gs_offsum<T, IDX, UU, false, ST>, gr, kBlock, s, n, nb, lv.S.sptr, cols,    \
                              P::val(lv), src, P::acc(lv), ctl)))
                if (pre) {
                    if (l == 0) PCG_OFFSUM(kUnroll, true);
                    else if (big) PCG_OFFSUM(kUnroll, false);
                    else PCG_OFFSUM(kUnrollSmall, false);
                } else {
                    if (l == 0) PCG_OFFSUM_B(kUnroll, true);
                    else if (big) PCG_OFFSUM_B(kUnroll, false);
                    else PCG_OFFSUM_B(kUnrollSmall, false);
                }
#undef PCG_OFFSUM
#undef PCG_OFFSUM_B
                kernels++;
            }
            const int32_t *pci = lv.gs_ci[d];
            const T *pv = P::part(lv, d);
            if (zero)
                launch_k(h->pdl, k_gs_block<T, true, true>, gb, kGsThreads, s, n, nb, w, pci, pv, P::dinv(lv), b,
                         (const T *)nullptr, (const T *)nullptr, dst, ctl);
            else if (pre)
                launch_k(h->pdl, k_gs_block<T, true, false>, gb, kGsThreads, s, n, nb, w, pci, pv, P::dinv(lv), b,
                         src, (const T *)P::acc(lv), dst, ctl);
            else
                launch_k(h->pdl, k_gs_block<T, false, false>, gb, kGsThreads, s, n, nb, w, pci, pv, P::dinv(lv), b,
                         src, (const T *)P::acc(lv), dst, ctl);
            kernels++;
            src = dst;
        }
        return kernels;
    }
    for (int sw = 1; sw <= nu; sw++) {
        T *dst = (nu - sw) % 2 == 0 ? target : P::t(lv);
        if (pre && sw == 1)
            launch_k(h->pdl, k_gs_sweep<T, true, true>, g, kBlock, s, n, nb, (const int32_t *)lv.A.rp,
                     (const int32_t *)lv.A.ci, P::csr(lv), P::dinv(lv), b, (const T *)nullptr, dst, ctl);
        else if (pre)
            launch_k(h->pdl, k_gs_sweep<T, true, false>, g, kBlock, s, n, nb, (const int32_t *)lv.A.rp,
                     (const int32_t *)lv.A.ci, P::csr(lv), P::dinv(lv), b, src, dst, ctl);
        else
            launch_k(h->pdl, k_gs_sweep<T, false, false>, g, kBlock, s, n, nb, (const int32_t *)lv.A.rp,
                     (const int32_t *)lv.A.ci, P::csr(lv), P::dinv(lv), b, src, dst, ctl);
        src = dst;
    }
    return nu;
}

// z = B r with the hybrid Gauss-Seidel smoother (gs_nu sweeps each side):
// the l1-Jacobi V-cycle with its smoothing steps replaced, the coarsest solve
// by launch_coarsest (no cluster tail), rho and beta by k_gs_finish0.
template <typename T, bool FCG>
int launch_vcycle_gs(amg_hier *h, cudaStream_t s) {
    using P = LP<T>;
    auto &lev = h->lev;
    int L = (int)lev.size() - 1;
    Ctl *ctl = h->ctl;
    Level &l0 = lev[0];
    const T *b0 = P::r0(h);
    const bool pdl = h->pdl;
    int kernels = 0;
    int sp1 = prof_begin(h, 0, s);
    kernels += launch_gs<T>(h, 0, true, b0, P::xpre(l0), s);
    launch_down0<T>(h, b0, s);
    kernels += 1;
    prof_end(h, sp1, s);
    int sp2 = prof_begin(h, 5, s);
    for (int l = 0; l < L; l++) {
        int spl = prof_begin(h, kLevelSpan + 3 * l, s);
        unsigned char sh = lev[l].shape[prec_index<T>()][0];
        if (l == 0) {
            launch_restrict<T>(h, 0, s);
            kernels += 1;
        } else {
            kernels += launch_gs<T>(h, l, true, P::b(lev[l]), P::xpre(lev[l]), s);
            launch_down_phase<T>(h, l, sh, s);
            kernels += (sh & 4) ? 1 : 2;
        }
        prof_end(h, spl, s);
    }
    int spc = prof_begin(h, kLevelSpan + 3 * L + 2, s);
    PCG_TRY(launch_coarsest<T>(h, s, &kernels));
    prof_end(h, spc, s);
    for (int l = L - 1; l >= 1; l--) {
        Level &lv = lev[l];
        int spl = prof_begin(h, kLevelSpan + 3 * l + 1, s);
        launch_prolong<T>(h, l, grid_rows(lv.A.n), s);
        kernels += 1 + launch_gs<T>(h, l, false, P::b(lv), P::x(lv), s);
        prof_end(h, spl, s);
    }
    prof_end(h, sp2, s);
    int sp3 = prof_begin(h, 1, s);
    launch_prolong<T>(h, 0, h->gridv, s);
    kernels += 1 + launch_gs<T>(h, 0, false, b0, P::x(l0), s);
    // the post sweep's grid, so rho is summed in the same order as there
    launch_k(pdl, k_gs_finish0<T, FCG>, grid0<T>(h), kBlock, s, l0.A.n, (const T *)P::x(l0), (const double *)h->r,
             (const double *)h->q, h->z, h->partials, ctl);
    kernels += 1;
    prof_end(h, sp3, s);
    h->launches += kernels;
    PCG_LAUNCH_CK();
    return AMG_OK;
}

template <int MODE>
int launch_iteration_t(amg_hier *h, cudaStream_t s) {
    int L = (int)h->lev.size() - 1;
    Level &l0 = h->lev[0];
    int n = l0.A.n;
    const bool pdl = h->pdl;
    if (L == 0) {
        launch_k(pdl, k_coarse_only<MODE == AMG_MODE_FCG32, MODE == AMG_MODE_FCG32>, h->gridv, kBlock, s, h->nL,
                 h->Ainv, h->r, h->z, h->q, h->partials, h->ctl);
        h->launches += 1;
    } else if (MODE == AMG_MODE_FCG32) {
        if (h->gs_nu) PCG_TRY((launch_vcycle_gs<float, true>(h, s)));
        else PCG_TRY((launch_vcycle<float, true>(h, s)));
    } else if (h->coarse_iter) {
        // the float64 V-cycle is not a fixed operator either: FCG(1) beta
        if (h->gs_nu) PCG_TRY((launch_vcycle_gs<double, true>(h, s)));
        else PCG_TRY((launch_vcycle<double, true>(h, s)));
    } else {
        if (h->gs_nu) PCG_TRY((launch_vcycle_gs<double, false>(h, s)));
        else PCG_TRY((launch_vcycle<double, false>(h, s)));
    }
    int sp4 = prof_begin(h, 6, s);
    launch_k(pdl, k_axpy_p, h->gridv, kBlock, s, n, h->z, h->p, h->ctl);
    prof_end(h, sp4, s);
    int sp5 = prof_begin(h, 2, s);
    WITH_COLS(l0.S, (launch_k(pdl, k_spmv<IDX>, h->grid64, kBlock, s, n, l0.S.sptr, cols, l0.S.v64,
                              pats, h->p, h->q,
                              h->partials, h->ctl)));
    prof_end(h, sp5, s);
    int sp6 = prof_begin(h, 3, s);
    launch_k(pdl, k_update<MODE>, h->gridv, kBlock, s, n, h->p, h->q, h->x, h->r, remit(h), h->partials, h->ctl,
             h->hist);
    prof_end(h, sp6, s);
    int sp7 = prof_begin(h, 4, s);
    WITH_COLS(l0.S, (launch_k(pdl, k_residual<false, MODE, IDX>, h->grid64, kBlock, s, n, l0.S.sptr, cols, l0.S.v64,
                              h->b, h->x, h->r, remit(h), h->partials, h->ctl, h->hist)));
    prof_end(h, sp7, s);
    h->launches += 4;
    PCG_LAUNCH_CK();
    return AMG_OK;
}

int launch_iteration(amg_hier *h, cudaStream_t s) {
    if (h->mode == AMG_MODE_FCG32) return launch_iteration_t<AMG_MODE_FCG32>(h, s);
    return launch_iteration_t<AMG_MODE_PCG64>(h, s);
}

int launch_prefix(amg_hier *h, cudaStream_t s) {
    Level &l0 = h->lev[0];
    int n = l0.A.n;
    k_zero<<<grid_rows(n), kBlock, 0, s>>>(h->p, n);
    k_zero<<<grid_rows(n), kBlock, 0, s>>>(h->q, n);
    if (h->mode == AMG_MODE_FCG32)
        WITH_COLS(l0.S, (launch_k(h->pdl, k_residual<true, AMG_MODE_FCG32, IDX>, h->grid64, kBlock, s, n, l0.S.sptr,
                                  cols, l0.S.v64, h->b, h->x, h->r, remit(h), h->partials, h->ctl, h->hist)));
    else
        WITH_COLS(l0.S, (launch_k(h->pdl, k_residual<true, AMG_MODE_PCG64, IDX>, h->grid64, kBlock, s, n, l0.S.sptr,
                                  cols, l0.S.v64, h->b, h->x, h->r, remit(h), h->partials, h->ctl, h->hist)));
    h->launches += 3;
    PCG_LAUNCH_CK();
    return AMG_OK;
}

}  // namespace

// Captures the prefix of one whole solve of h in `mode` onto cs, which must
// be capturing (possibly as a forked branch of a larger capture): zero p/q,
// first residual, the loop-condition kernel, and a while node whose body is
// filled later by capture_solve_body. Kernel counts go to *prefix_k.
int capture_solve_prefix(amg_hier *h, int mode, cudaStream_t cs, PendingBody *pb, int *prefix_k) {
    int saved_mode = h->mode;
    h->mode = mode;
    int64_t l0 = h->launches;
    int st = launch_prefix(h, cs);
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle hc = 0;
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t cnode = nullptr;
    cudaError_t e = cudaSuccess;
    if (!st) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr);
    if (!st && e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault);
    if (!st && e == cudaSuccess) {
        k_set_cond<<<1, 32, 0, cs>>>(hc, h->ctl, 0);
        e = cudaGetLastError();
    }
    if (!st && e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd);
    if (!st && e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hc;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&cnode, g, deps, nullptr, nd, &cp);
    }
    if (!st && e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    *prefix_k = (int)(h->launches - l0) + 1;
    h->launches = l0;
    h->mode = saved_mode;
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "solve graph capture", __FILE__, __LINE__);
    pb->h = h;
    pb->mode = mode;
    pb->body = cp.conditional.phGraph_out[0];
    pb->hc = hc;
    return AMG_OK;
}

// Fills the while node's body: two iterations and the condition kernel,
// captured on s (not capturing). Kernel count of one body to *body_k.
int capture_solve_body(const PendingBody &pb, cudaStream_t s, int *body_k) {
    amg_hier *h = pb.h;
    int saved_mode = h->mode;
    h->mode = pb.mode;
    int64_t l1 = h->launches;
    int st = AMG_OK;
    cudaError_t e = cudaStreamBeginCaptureToGraph(s, pb.body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = launch_iteration(h, s);
        if (!st) st = launch_iteration(h, s);
        if (!st) k_set_cond<<<1, 32, 0, s>>>(pb.hc, h->ctl, 1);
        cudaGraph_t bout = pb.body;
        cudaError_t e2 = cudaStreamEndCapture(s, &bout);
        if (e2 != cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    *body_k = (int)(h->launches - l1) + 1;
    h->launches = l1;
    h->mode = saved_mode;
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "solve graph body capture", __FILE__, __LINE__);
    return AMG_OK;
}

namespace {

// Whole solve as one graph: prefix (zero p/q, first residual, condition),
// then a while node whose body is two iterations plus the condition kernel.
// tail = false builds the variant without the shared-memory tail.
int build_graph(amg_hier *h, int mode, bool tail = true) {
    if (!h->cap_stream) PCG_CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = h->cap_stream;
    PendingBody pb;
    int prefix = 0, body_k = 0;
    cudaGraphExec_t &exec = tail ? h->gexec[mode] : h->gexec_nt[mode];
    h->no_tail = tail ? 0 : 1;
    PCG_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int st = capture_solve_prefix(h, mode, cs, &pb, &prefix);
    cudaGraph_t full = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &full);
    if (!st && e != cudaSuccess) st = cuda_fail(e, "solve graph capture", __FILE__, __LINE__);
    if (!st) st = capture_solve_body(pb, cs, &body_k);
    h->no_tail = 0;
    if (st) {
        if (full) cudaGraphDestroy(full);
        return st;
    }
    e = cudaGraphInstantiate(&exec, full, 0);
    cudaGraphDestroy(full);
    if (e != cudaSuccess) {
        exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
    h->graph_prefix_kernels = prefix;
    (tail ? h->graph_body_kernels : h->graph_body_kernels_nt)[mode] = body_k;
    return AMG_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// Shared-memory cluster tail (tail.cu); PCGAMG_TAIL=0 launches every level
// separately instead.
int setup_tail(amg_hier *h) {
    h->tail_first[0] = h->tail_first[1] = 0;
    // the tail holds a dense coarsest inverse and aggregate-map transfers
    if (h->coarse_iter || h->smoothed) return AMG_OK;
    const char *e = getenv("PCGAMG_TAIL");
    if (e && e[0] == '0') return AMG_OK;
    return setup_smem_tail(h);
}

int set_profile(amg_hier *h, int enable) {
    if (enable && h->ev.empty()) {
        h->ev.resize(2 * kEvPairs);
        for (auto &e : h->ev) PCG_CK(cudaEventCreate(&e));
    }
    h->profile = enable ? 1 : 0;
    h->ev_used = 0;
    return AMG_OK;
}

void free_profile(amg_hier *h) {
    for (auto &e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
    drop_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
}

int alloc_solve_workspace(amg_hier *h) {
    Mem &M = h->mem;
    int n = h->lev[0].A.n;
    int dev = 0, sms = 0;
    PCG_CK(cudaGetDevice(&dev));
    PCG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    h->device = dev;
    // One wave of resident blocks per level-0 kernel family (grid = SMs x
    // blocks resident per SM), capped by the rows available.
    auto wave = [&](const void *fn, int *grid) -> int {
        int per = 0;
        PCG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kBlock, 0));
        int64_t want = ((int64_t)n + kBlock - 1) / kBlock;
        int64_t g = (int64_t)sms * (per > 0 ? per : 1);
        *grid = (int)(want < g ? want : g);
        if (*grid < 1) *grid = 1;
        return AMG_OK;
    };
    PCG_TRY(wave((const void *)k_down<float, int32_t, kUnroll, true>, &h->grid32));
    if (pat_rows(h)) {
        // the whole-row sweeps: one wave of the fewer of their resident blocks
        int gd = 0, gp = 0;
        if (h->lev[0].S.col16) {
            PCG_TRY(wave((const void *)k_down<float, int16_t, kPatRow, true>, &gd));
            PCG_TRY(wave((const void *)k_post<float, double, true, true, int16_t, kPatRow, true>, &gp));
        } else {
            PCG_TRY(wave((const void *)k_down<float, int32_t, kPatRow, true>, &gd));
            PCG_TRY(wave((const void *)k_post<float, double, true, true, int32_t, kPatRow, true>, &gp));
        }
        h->grid32 = std::min(gd, gp);
    }
    PCG_TRY(wave((const void *)k_spmv<int32_t>, &h->grid64));
    PCG_TRY(wave((const void *)k_update<AMG_MODE_FCG32>, &h->gridv));
    h->nblk = std::max(h->grid32, std::max(h->grid64, h->gridv));
    // One wave of each coarse-level sweep variant, and the fixed shape rule.
    const void *fns[2][2][2] = {
        {{(const void *)k_down<float, int16_t, kUnroll, false>, (const void *)k_down<float, int16_t, kUnrollSmall, false>},
         {(const void *)k_post<float, float, false, false, int16_t, kUnroll, false>,
          (const void *)k_post<float, float, false, false, int16_t, kUnrollSmall, false>}},
        {{(const void *)k_down<double, int16_t, kUnroll, false>, (const void *)k_down<double, int16_t, kUnrollSmall, false>},
         {(const void *)k_post<double, double, false, false, int16_t, kUnroll, false>,
          (const void *)k_post<double, double, false, false, int16_t, kUnrollSmall, false>}}};
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int c = 0; c < 2; c++) {
                int per = 0;
                PCG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fns[a][b][c], kBlock, 0));
                h->wave[a][b][c] = sms * (per > 0 ? per : 1);
            }
    for (size_t l = 1; l < h->lev.size(); l++) {
        unsigned char d = (unsigned char)((h->lev[l].A.n <= kSmallRows ? 1 : 0) | 2);
        for (auto &pr : h->lev[l].shape) pr[0] = pr[1] = d;
    }
    PCG_TRY(alloc(M, &h->b, n));
    PCG_TRY(alloc(M, &h->x, n));
    PCG_TRY(alloc(M, &h->r, n));
    PCG_TRY(alloc(M, &h->r32, n));
    PCG_TRY(alloc(M, &h->z, n));
    PCG_TRY(alloc(M, &h->q, n));
    PCG_TRY(alloc(M, &h->p, n));
    PCG_TRY(alloc(M, &h->partials, 2 * (size_t)h->nblk));
    PCG_TRY(alloc(M, &h->ctl, 1));
    PCG_CK(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), M.stream));
    PCG_CK(cudaMallocHost(&h->ctl_host, sizeof(Ctl)));
    h->hist_cap = 1001;
    PCG_TRY(alloc(M, &h->hist, h->hist_cap));
    if (h->coarse_iter) PCG_TRY(cws_alloc(h, M, h->cws, 1));
    PCG_TRY(setup_tail(h));
    return AMG_OK;
}

// Launch-shape tuner: for every level l in 1..L-1 (the levels with down and
// post sweeps), each V-cycle precision and each phase (down: down sweep +
// restriction; up: prolongation + post sweep), times the eight shapes
// (4- or 16-entry chunks x one-wave or one-thread-per-row grid x separate or
// fused launches) on this device, `reps` runs each after one warm-up run,
// and moves to the fastest only if it beats the current shape by more than
// 3% (so timing noise does not flip shapes). Work vectors are zeroed first;
// the inputs only set the timing. Captured solve graphs are dropped.
constexpr int kShapes = 9;  // 0..7, and 8: multi-lane rows
template <typename T>
int tune_level(amg_hier *h, int l, cudaStream_t s, int reps, cudaEvent_t e0, cudaEvent_t e1, int *changed) {
    int pi = prec_index<T>();
    Level &lv = h->lev[l];
    for (int sweep = 0; sweep < 2; sweep++) {
        float best = 0.0f, cur = 0.0f;
        int pick = -1;
        for (int shape = 0; shape < kShapes; shape++) {
            for (int r = -1; r < reps; r++) {
                if (r == 0) PCG_CK(cudaEventRecord(e0, s));
                if (sweep == 0) launch_down_phase<T>(h, l, (unsigned char)shape, s);
                else launch_up_phase<T>(h, l, (unsigned char)shape, s);
            }
            PCG_CK(cudaEventRecord(e1, s));
            PCG_CK(cudaEventSynchronize(e1));
            PCG_LAUNCH_CK();
            float ms = 0.0f;
            PCG_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (shape == lv.shape[pi][sweep]) cur = ms;
            if (pick < 0 || ms < best) {
                best = ms;
                pick = shape;
            }
        }
        if (best > 0.97f * cur) pick = lv.shape[pi][sweep];
        if (lv.shape[pi][sweep] != pick) (*changed)++;
        lv.shape[pi][sweep] = (unsigned char)pick;
    }
    return AMG_OK;
}

int autotune_impl(amg_hier *h, cudaStream_t s, int reps, int *changed) {
    int L = (int)h->lev.size() - 1;
    *changed = 0;
    // the shapes tune the l1-Jacobi sweeps and the tentative transfers only
    if (h->gs_nu || h->smoothed) return AMG_OK;
    if (reps < 1) reps = 1;
    PCG_CK(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), s));
    for (int l = 1; l <= L; l++) {
        Level &lv = h->lev[l];
        size_t n = (size_t)lv.A.n;
        for (float *v : {lv.b32, lv.x32, lv.t32, lv.xpre32, lv.xp32})
            if (v) PCG_CK(cudaMemsetAsync(v, 0, n * sizeof(float), s));
        for (double *v : {lv.b64, lv.x64, lv.t64, lv.xpre64, lv.xp64})
            if (v) PCG_CK(cudaMemsetAsync(v, 0, n * sizeof(double), s));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = AMG_OK;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) st = cuda_fail(ce, "autotune events", __FILE__, __LINE__);
    for (int l = 1; l < L && !st; l++) {
        st = tune_level<float>(h, l, s, reps, e0, e1, changed);
        if (!st) st = tune_level<double>(h, l, s, reps, e0, e1, changed);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    drop_graphs(h);
    PCG_CK(cudaStreamSynchronize(s));
    return st;
}

// Drops every captured whole-solve graph of h (they are rebuilt on the next
// solve) and marks batch graphs holding h as stale.
void drop_graphs(amg_hier *h) {
    for (auto *set : {h->gexec, h->gexec_nt, h->multi.gexec})
        for (int m = 0; m < 2; m++) {
            if (set[m]) cudaGraphExecDestroy(set[m]);
            set[m] = nullptr;
        }
    h->graph_gen++;
}

// Makes room for maxit+1 history values (invalidates captured graphs).
int ensure_hist(amg_hier *h, int maxit) {
    if (maxit + 1 <= h->hist_cap) return AMG_OK;
    release(h->mem, h->hist);
    h->hist_cap = maxit + 1;
    PCG_TRY(alloc(h->mem, &h->hist, h->hist_cap));
    drop_graphs(h);
    return AMG_OK;
}

// Serving lane. solve_prepare makes the whole-solve graph of `mode` (and a
// history of maxit + 1) ready; solve_launch starts one solve on s without
// waiting (b, x0: host or device, copied into h's own vectors) and copies the
// final state to the pinned mirror; once s has passed it, solve_collect
// writes x (host or device; zeros when b = 0) and the outcome.
int solve_prepare(amg_hier *h, int mode, int maxit) {
    PCG_TRY(ensure_hist(h, maxit));
    if (!h->gexec_nt[mode]) PCG_TRY(build_graph(h, mode, false));
    return AMG_OK;
}

int solve_launch(amg_hier *h, int mode, const double *b, const double *x0, double rtol, int maxit, cudaStream_t s) {
    int n = h->lev[0].A.n;
    h->mem.stream = s;
    PCG_TRY(solve_prepare(h, mode, maxit));
    PCG_CK(cudaMemcpyAsync(h->b, b, sizeof(double) * n, cudaMemcpyDefault, s));
    PCG_CK(cudaMemcpyAsync(h->x, x0, sizeof(double) * n, cudaMemcpyDefault, s));
    Ctl c0;
    memset(&c0, 0, sizeof(c0));
    c0.rtol = rtol;
    c0.maxit = maxit;
    c0.mode = mode;
    c0.flex = h->coarse_iter;
    c0.restart = 1;
    *h->ctl_host = c0;
    PCG_CK(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    PCG_CK(cudaGraphLaunch(h->gexec_nt[mode], s));
    PCG_CK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    return AMG_OK;
}

int solve_collect(amg_hier *h, int mode, double *x, cudaStream_t s, int *status, int *iters, double *true_rel,
                  int64_t *kernels) {
    int n = h->lev[0].A.n;
    const Ctl &c = *h->ctl_host;
    if (c.done == 1 && c.bnorm == 0.0) {
        k_zero<<<grid_rows(n), kBlock, 0, s>>>(h->x, n);
        PCG_LAUNCH_CK();
    }
    PCG_CK(cudaMemcpyAsync(x, h->x, sizeof(double) * n, cudaMemcpyDefault, s));
    int64_t k = h->graph_prefix_kernels + (int64_t)c.bodies * h->graph_body_kernels_nt[mode];
    h->launches += k;
    if (kernels) *kernels = k;
    if (status) *status = c.done ? c.status : AMG_ERR_NOCONV;
    if (iters) *iters = c.iter;
    if (true_rel) *true_rel = c.true_rel;
    h->last_true_rel = c.true_rel;
    return AMG_OK;
}

int solve_impl(amg_hier *h, const double *b, double *x, double rtol, int maxit, int *iters, double *res_hist,
               cudaStream_t s) {
    if (!b || !x || !(rtol >= 0.0) || maxit < 0) {
        set_error("pcg_solve: bad arguments");
        return AMG_ERR_ARG;
    }
    Level &l0 = h->lev[0];
    int n = l0.A.n;
    h->mem.stream = s;
    if (maxit + 1 > h->hist_cap) {
        release(h->mem, h->hist);
        h->hist_cap = maxit + 1;
        PCG_TRY(alloc(h->mem, &h->hist, h->hist_cap));
        drop_graphs(h);
    }
    bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    PCG_CK(cudaMemcpyAsync(h->b, b, sizeof(double) * n, bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    PCG_CK(cudaMemcpyAsync(h->x, x, sizeof(double) * n, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    Ctl c0;
    memset(&c0, 0, sizeof(c0));
    c0.rtol = rtol;
    c0.maxit = maxit;
    c0.mode = h->mode;
    c0.flex = h->coarse_iter;
    c0.restart = 1;
    *h->ctl_host = c0;
    PCG_CK(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    bool graph = h->use_graph && !h->profile;
    if (graph && !h->gexec[h->mode]) {
        if (build_graph(h, h->mode) != AMG_OK) {
            h->use_graph = 0;  // keep solving with stream launches; the reason stays in amg_last_error
            graph = false;
        }
    }
    if (graph) {
        PCG_CK(cudaGraphLaunch(h->gexec[h->mode], s));
        PCG_CK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaStreamSynchronize(s));
        h->launches += h->graph_prefix_kernels + (int64_t)h->ctl_host->bodies * h->graph_body_kernels[h->mode];
    } else {
        PCG_TRY(launch_prefix(h, s));
        // Iterate in chunks; once done, every later kernel returns at once.
        const int chunk = 4;
        int launched = 0;
        for (;;) {
            PCG_CK(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            PCG_CK(cudaStreamSynchronize(s));
            if (h->profile) prof_collect(h);
            if (h->ctl_host->done || launched >= maxit) break;
            for (int k = 0; k < chunk && launched < maxit; k++, launched++) PCG_TRY(launch_iteration(h, s));
        }
    }
    Ctl &c = *h->ctl_host;
    if (c.done == 1 && c.bnorm == 0.0) k_zero<<<grid_rows(n), kBlock, 0, s>>>(h->x, n);
    PCG_LAUNCH_CK();
    PCG_CK(cudaMemcpyAsync(x, h->x, sizeof(double) * n, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (res_hist) PCG_CK(cudaMemcpyAsync(res_hist, h->hist, sizeof(double) * (c.iter + 1), cudaMemcpyDefault, s));
    PCG_CK(cudaStreamSynchronize(s));
    if (iters) *iters = c.iter;
    h->last_true_rel = c.true_rel;
    int st = c.done ? c.status : AMG_ERR_NOCONV;
    if (st == AMG_ERR_NOCONV) set_error("pcg_solve: no convergence in %d iterations (rel %.3e)", maxit, c.rel);
    else if (st == AMG_ERR_BREAKDOWN) set_error("pcg_solve: breakdown (r.z <= 0 or p.Ap <= 0) at iteration %d", c.iter);
    else if (st == AMG_ERR_NAN) set_error("pcg_solve: NaN/Inf at iteration %d", c.iter);
    return st;
}

}  // namespace pcgamg
