// Multi right-hand-side solve: k systems A x_c = b_c (c < k <= 32) sharing
// one hierarchy, advanced together (arxiv 2210.16660, Sec. 3.1 / Sec. 5 per
// column; the hierarchy is built once and reused, Sec. 2 / Sec. 4).
//
// Every vector is an n x K row-major block (the K values of a row are
// contiguous; K = k rounded up to a power of two, at least 4, padding
// columns are zero and inactive). One thread per (row, column): the K threads of a row read
// the same matrix entry (one broadcast load) and K consecutive vector values
// (one coalesced load), so each stored entry is read once per sweep for all
// columns (SpMM). Each column keeps its own Krylov scalars, iteration count,
// residual history and status; a column that has converged or failed stops
// changing (alpha = 0) while the others go on. Same V-cycle structure and
// reading of the method as the single right-hand-side path.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "sell_row.cuh"

namespace pcgamg {

namespace {

constexpr int kMB = 256;         // threads per block
constexpr int kMaxK = 32;

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// Each thread owns V consecutive columns of one row (one 16-byte vector: 4
// floats or 2 doubles), so a row takes K / V threads, a warp covers 32V/K
// consecutive rows, a neighbour row's column group is one vector load, and
// the matrix entry of a row is one broadcast load shared by its threads.
template <typename T>
struct VW {
    static constexpr int V = 16 / (int)sizeof(T);
};

template <typename T, int V>
__device__ __forceinline__ void ld_vec(const T *p, T (&o)[V]) {
    if constexpr (sizeof(T) == 4) {
        float4 u = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = u.x; o[1] = u.y; o[2] = u.z; o[3] = u.w;
    } else {
        double2 u = __ldg(reinterpret_cast<const double2 *>(p));
        o[0] = u.x; o[1] = u.y;
    }
}

template <typename T, int V>
__device__ __forceinline__ void ld_vec_cg(const T *p, T (&o)[V]) {
    if constexpr (sizeof(T) == 4) {
        float4 u = __ldcg(reinterpret_cast<const float4 *>(p));
        o[0] = u.x; o[1] = u.y; o[2] = u.z; o[3] = u.w;
    } else {
        double2 u = __ldcg(reinterpret_cast<const double2 *>(p));
        o[0] = u.x; o[1] = u.y;
    }
}

template <typename T, int V>
__device__ __forceinline__ void st_vec(T *p, const T (&o)[V]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
    }
}

// acc[v] += sum_k a_k x(j_k)[v] over one sliced-ELL row, entries in storage
// order; U entries' columns and values are loaded before their gathers.
template <int U, bool STREAM, int V, typename IDX, typename T, typename F>
__device__ __forceinline__ void sell_row_vec(const IDX *__restrict__ c, const T *__restrict__ a, int w, int row,
                                             F xvec, T (&acc)[V]) {
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = 0;
    int k = 0;
    for (; k + U <= w; k += U) {
        int j[U];
        T av[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            j[u] = col_of(ld_mat<STREAM>(c + 32 * (k + u)), row);
            av[u] = ld_mat<STREAM>(a + 32 * (k + u));
        }
        T x[U][V];
#pragma unroll
        for (int u = 0; u < U; u++) xvec(j[u], x[u]);
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
            for (int v = 0; v < V; v++) acc[v] += av[u] * x[u][v];
    }
    for (; k < w; k++) {
        int j = col_of(ld_mat<STREAM>(c + 32 * k), row);
        T av = ld_mat<STREAM>(a + 32 * k);
        T x[V];
        xvec(j, x);
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] += av * x[v];
    }
}

// Thread (row i, first column c0) of a K-column block; grid-stride over
// n * (K / V) threads.
#define MK_FOR(nrows, V)                                                                      \
    for (int64_t g_ = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;                         \
         g_ < (int64_t)(nrows) * (K / (V)); g_ += (int64_t)gridDim.x * blockDim.x)
#define MK_IDX(V)                                                                             \
    int i = (int)(g_ / (K / (V)));                                                            \
    int c0 = (int)(g_ % (K / (V))) * (V);                                                     \
    int64_t e0 = (int64_t)i * K + c0;

// Whether any of the V columns from c0 is still iterating.
template <int V>
__device__ __forceinline__ bool group_live(const CtlM *ctl, int c0) {
    int a = 0;
#pragma unroll
    for (int v = 0; v < V; v++) a |= ctl->active[c0 + v];
    return a != 0;
}

// A thread's column group is fixed over its grid-stride loop (the stride is a
// multiple of K / V); a group whose columns have all stopped skips its rows,
// so a block with few live columns moves only their vectors. The arithmetic
// of a live column does not depend on which other columns are live.
#define MK_LIVE(V)                                                                            \
    const bool live_ = group_live<V>(                                                         \
        ctl, (int)((((int64_t)blockIdx.x * blockDim.x + threadIdx.x) % (K / (V))) * (V)));

// Per-column block sums: a thread holds a[V] and b[V] for columns c0..c0+V-1
// (c0 fixed per thread). Result: threads 0..K-1 hold the block's sums for
// columns 0..K-1.
template <int K, int V>
__device__ __forceinline__ void block_sum_cols(double (&a)[V], double (&b)[V], double &ra, double &rb) {
    constexpr int TPR = K / V;
    __shared__ double sa[kMB / 32][kMaxK], sb[kMB / 32][kMaxK];
#pragma unroll
    for (int o = 16; o >= TPR; o >>= 1)
#pragma unroll
        for (int v = 0; v < V; v++) {
            a[v] += __shfl_down_sync(0xffffffffu, a[v], o);
            b[v] += __shfl_down_sync(0xffffffffu, b[v], o);
        }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < TPR)
#pragma unroll
        for (int v = 0; v < V; v++) {
            sa[w][lane * V + v] = a[v];
            sb[w][lane * V + v] = b[v];
        }
    __syncthreads();
    ra = rb = 0.0;
    if (threadIdx.x < K) {
        for (int q = 0; q < kMB / 32; q++) { ra += sa[q][threadIdx.x]; rb += sb[q][threadIdx.x]; }
    }
}

// Writes the block's per-column partials (layout [slot][column][block]) and
// returns true in every thread of the last block to finish.
template <int K, int V>
__device__ __forceinline__ bool publish_cols(double (&a)[V], double (&b)[V], double *partials,
                                             unsigned *counter) {
    __shared__ bool last;
    double ra, rb;
    block_sum_cols<K, V>(a, b, ra, rb);
    int G = gridDim.x;
    if (threadIdx.x < K) {
        partials[(0 * K + threadIdx.x) * G + blockIdx.x] = ra;
        partials[(1 * K + threadIdx.x) * G + blockIdx.x] = rb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return last;
}

// Last block: res[q] = sum over blocks of partials[q][.] in block order, for
// q < 2K (slot 0 columns, then slot 1 columns). Loads are unrolled so each
// lane has several in flight.
template <int K>
__device__ __forceinline__ void final_cols(const double *partials, double *res) {
    __threadfence();
    int G = gridDim.x;
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = w; q < 2 * K; q += kMB / 32) {
        const double *src = partials + (int64_t)q * G;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int k = lane;
        for (; k + 96 < G; k += 128) {
            s0 += __ldcg(src + k);
            s1 += __ldcg(src + k + 32);
            s2 += __ldcg(src + k + 64);
            s3 += __ldcg(src + k + 96);
        }
        for (; k < G; k += 32) s0 += __ldcg(src + k);
        double s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) res[q] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void col_fail(CtlM *c, int col, int status) {
    c->status[col] = status;
    c->active[col] = 0;
}

__device__ __forceinline__ void update_done(CtlM *c) {
    int any = 0;
    for (int q = 0; q < c->K; q++) any |= c->active[q];
    if (!any) c->done = 1;
}

// ------------------------------------------------------------ V-cycle
template <typename T, typename IDX, int K, int U, bool STREAM>
__global__ void __launch_bounds__(kMB) k_down_m(int n, const int32_t *__restrict__ sptr,
                                               const IDX *__restrict__ col, const T *__restrict__ val,
                                               const T *__restrict__ xpre, const T *__restrict__ b,
                                               const T *__restrict__ p, T *__restrict__ t,
                                               const CtlM *__restrict__ ctl) {
    constexpr int V = VW<T>::V;
    if (ctl->done) return;
    MK_LIVE(V)
    MK_FOR(live_ ? n : 0, V) {
        MK_IDX(V)
        int s = i >> 5, lane = i & 31;
        int32_t base = ldg(sptr + s);
        int w = (ldg(sptr + s + 1) - base) >> 5;
        T acc[V];
        sell_row_vec<U, STREAM, V>(col + base + lane, val + base + lane, w, i,
                                   [&](int j, T (&x)[V]) { ld_vec<T, V>(xpre + (int64_t)j * K + c0, x); }, acc);
        T bv[V], o[V];
        ld_vec<T, V>(b + e0, bv);
        T pi = ldg(p + i);
#pragma unroll
        for (int v = 0; v < V; v++) o[v] = pi * (bv[v] - acc[v]);
        st_vec<T, V>(t + e0, o);
    }
}

template <typename T, typename TO, bool PRE, int K>
__global__ void __launch_bounds__(kMB) k_restrict_m(int nc, const int32_t *__restrict__ rptr,
                                                   const int32_t *__restrict__ ridx, const T *__restrict__ t,
                                                   TO *__restrict__ bc, const T *__restrict__ dinvc,
                                                   T *__restrict__ xprec, const CtlM *__restrict__ ctl) {
    constexpr int V = VW<T>::V;
    if (ctl->done) return;
    MK_LIVE(V)
    MK_FOR(live_ ? nc : 0, V) {
        MK_IDX(V)
        T s[V];
#pragma unroll
        for (int v = 0; v < V; v++) s[v] = 0;
        for (int32_t q = ldg(rptr + i); q < ldg(rptr + i + 1); q++) {
            T x[V];
            ld_vec<T, V>(t + (int64_t)ldg(ridx + q) * K + c0, x);
#pragma unroll
            for (int v = 0; v < V; v++) s[v] += x[v];
        }
#pragma unroll
        for (int v = 0; v < V; v++) bc[e0 + v] = (TO)s[v];
        if (PRE) {
            T d = ldg(dinvc + i), o[V];
#pragma unroll
            for (int v = 0; v < V; v++) o[v] = d * s[v];
            st_vec<T, V>(xprec + e0, o);
        }
    }
}

// x_L = A_L^{-1} b_L for K columns (float64): one warp per (row, pair of
// columns), lanes striding over the row with coalesced loads of A_L^{-1},
// then the shuffle tree -- the order of k_coarse, per column.
template <typename TO, int K>
__global__ void __launch_bounds__(kMB) k_coarse_m(int nL, const double *__restrict__ ainv,
                                                 const double *__restrict__ bL, TO *__restrict__ xL,
                                                 const CtlM *__restrict__ ctl) {
    constexpr int V = 2;
    if (ctl->done) return;
    int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= nL * (K / V)) return;  // whole warps
    int row = warp / (K / V), c0 = (warp % (K / V)) * V;
    if (!group_live<V>(ctl, c0)) return;
    const double *a = ainv + (int64_t)row * nL;
    double s0 = 0.0, s1 = 0.0;
    for (int j = lane; j < nL; j += 32) {
        double aj = ldg(a + j);
        double2 bj = __ldg(reinterpret_cast<const double2 *>(bL + (int64_t)j * K + c0));
        s0 += aj * bj.x;
        s1 += aj * bj.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) {
        xL[(int64_t)row * K + c0] = (TO)s0;
        xL[(int64_t)row * K + c0 + 1] = (TO)s1;
    }
}

template <typename T, int K>
__global__ void __launch_bounds__(kMB) k_prolong_m(int n, const T *__restrict__ xpre, const T *__restrict__ p,
                                                  const int32_t *__restrict__ agg, const T *__restrict__ xc,
                                                  T *__restrict__ xp, const CtlM *__restrict__ ctl) {
    constexpr int V = VW<T>::V;
    if (ctl->done) return;
    MK_LIVE(V)
    MK_FOR(live_ ? n : 0, V) {
        MK_IDX(V)
        T x[V];
        ld_vec<T, V>(xpre + e0, x);
        int a = ldg(agg + i);
        if (a >= 0) {
            T pi = ldg(p + i), y[V];
            ld_vec<T, V>(xc + (int64_t)a * K + c0, y);
#pragma unroll
            for (int v = 0; v < V; v++) x[v] += pi * y[v];
        }
        st_vec<T, V>(xp + e0, x);
    }
}

// z = xp + D^-1 (b - A xp); DOT on level 0: per-column r.z and z.q_old, and
// the last block forms rho_c and beta_c.
template <typename T, typename TZ, bool DOT, bool FCG, typename IDX, int K, int U, bool STREAM>
__global__ void __launch_bounds__(kMB) k_post_m(int n, const int32_t *__restrict__ sptr,
                                               const IDX *__restrict__ col, const T *__restrict__ val,
                                               const T *__restrict__ xp, const T *__restrict__ b,
                                               const T *__restrict__ dinv, TZ *__restrict__ z,
                                               const double *__restrict__ r64, const double *__restrict__ qold,
                                               double *partials, CtlM *ctl) {
    constexpr int V = VW<T>::V;
    if (ctl->done) return;
    double rz[V], zq[V];
#pragma unroll
    for (int v = 0; v < V; v++) rz[v] = zq[v] = 0.0;
    MK_LIVE(V)
    MK_FOR(live_ ? n : 0, V) {
        MK_IDX(V)
        int s = i >> 5, lane = i & 31;
        int32_t base = ldg(sptr + s);
        int w = (ldg(sptr + s + 1) - base) >> 5;
        T acc[V];
        sell_row_vec<U, STREAM, V>(col + base + lane, val + base + lane, w, i,
                                   [&](int j, T (&x)[V]) { ld_vec<T, V>(xp + (int64_t)j * K + c0, x); }, acc);
        T xv[V], bv[V];
        ld_vec<T, V>(xp + e0, xv);
        ld_vec<T, V>(b + e0, bv);
        T d = ldg(dinv + i);
#pragma unroll
        for (int v = 0; v < V; v++) {
            TZ zo = (TZ)(xv[v] + d * (bv[v] - acc[v]));
            z[e0 + v] = zo;
            if (DOT) {
                rz[v] += ldg(r64 + e0 + v) * (double)zo;
                if (FCG) zq[v] += (double)zo * ldg(qold + e0 + v);
            }
        }
    }
    if (DOT) {
        __shared__ double res[2 * kMaxK];
        if (publish_cols<K, V>(rz, zq, partials, &ctl->counter[0])) {
            final_cols<K>(partials, res);
            if (threadIdx.x == 0) ctl->counter[0] = 0;
            int c = threadIdx.x;
            if (c < K && ctl->active[c]) {
                double rho = res[c], zqc = res[K + c];
                if (!isfinite(rho) || !isfinite(zqc)) {
                    col_fail(ctl, c, AMG_ERR_NAN);
                } else if (!(rho > 0.0)) {
                    col_fail(ctl, c, AMG_ERR_BREAKDOWN);
                } else {
                    ctl->rho[c] = rho;
                    double beta = 0.0;
                    if (!ctl->restart[c])
                        beta = ctl->mode == AMG_MODE_FCG32 || ctl->flex ? -zqc / ctl->pq_old[c]
                                                                        : rho / ctl->rho_old[c];
                    ctl->beta[c] = beta;
                }
            }
        }
    }
}

// ------------------------------------------------------------ hybrid Gauss-Seidel
// One sweep of the l1 hybrid Gauss-Seidel smoother for K columns (the
// single-column k_gs_warp per column group): one warp per (32-row slice,
// group of V columns), a lane per row. Phase one sums each row's entries with
// x_old except the in-block ones this pass has already updated; phase two
// runs the slice's rows in pass order in 32 steps, each finished value
// broadcast by a shuffle and added by the rows whose next in-block entry (in
// pass order) is that row. Needs blocks whose size divides 32 and rows with
// at most kGsPartM in-block entries of the pass.
constexpr int kGsPartM = 8;

template <typename T, typename IDX, int U, bool FWD, bool ZERO, bool STREAM, int K>
__global__ void __launch_bounds__(kMB) k_gs_warp_m(int n, int nb, int w, const int32_t *__restrict__ sptr,
                                                  const IDX *__restrict__ col, const T *__restrict__ val,
                                                  const int32_t *__restrict__ pci, const T *__restrict__ pv,
                                                  const T *__restrict__ dinv, const T *__restrict__ b,
                                                  const T *__restrict__ xo, T *__restrict__ xn,
                                                  const CtlM *__restrict__ ctl) {
    constexpr int V = VW<T>::V;
    constexpr int G = K / V;
    if (ctl->done) return;
    const int lane = threadIdx.x & 31;
    const int nsl = (n + 31) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < (int64_t)nsl * G; wi += nw) {
        const int sl = (int)(wi / G), c0 = (int)(wi % G) * V;
        if (!group_live<V>(ctl, c0)) continue;  // uniform over the warp
        const int i = (sl << 5) + lane;
        const bool valid = i < n;
        const int64_t e0 = (int64_t)i * K + c0;
        T acc[V];
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = 0;
        if (!ZERO && valid) {
            const int lo = (i / nb) * nb, hi = min(n, lo + nb);
            int32_t base = ldg(sptr + sl);
            int wd = (ldg(sptr + sl + 1) - base) >> 5;
            sell_row_vec<U, STREAM, V>(col + base + lane, val + base + lane, wd, i,
                                       [&](int j, T (&x)[V]) {
                                           bool done = FWD ? (j >= lo && j < i) : (j > i && j < hi);
                                           if (done) {
#pragma unroll
                                               for (int v = 0; v < V; v++) x[v] = 0;
                                           } else {
                                               ld_vec<T, V>(xo + (int64_t)j * K + c0, x);
                                           }
                                       },
                                       acc);
        }
        int rj[kGsPartM];
        T ra[kGsPartM];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < kGsPartM; k++) {
            bool ok = valid && k < w;
            rj[k] = ok ? ldg(pci + (int64_t)i * w + k) : -1;
            ra[k] = ok ? ldg(pv + (int64_t)i * w + k) : T(0);
            cnt += rj[k] >= 0 ? 1 : 0;
        }
        int pj[kGsPartM];
        T pa[kGsPartM];
#pragma unroll
        for (int k = 0; k < kGsPartM; k++) {
            if (FWD) {
                pj[k] = rj[k];
                pa[k] = ra[k];
            } else {
                pj[k] = -1;
                pa[k] = T(0);
#pragma unroll
                for (int m = 0; m < kGsPartM; m++)
                    if (m == cnt - 1 - k) {
                        pj[k] = rj[m];
                        pa[k] = ra[m];
                    }
            }
        }
        T bv[V], xold[V], x[V];
        const T di = valid ? ldg(dinv + i) : T(0);
#pragma unroll
        for (int v = 0; v < V; v++) bv[v] = xold[v] = x[v] = 0;
        if (valid) {
            ld_vec<T, V>(b + e0, bv);
            if (!ZERO) ld_vec<T, V>(xo + e0, xold);
        }
#pragma unroll 2
        for (int step = 0; step < 32; step++) {
            const int t = FWD ? step : 31 - step;
            if (lane == t)
#pragma unroll
                for (int v = 0; v < V; v++) x[v] = ZERO ? di * (bv[v] - acc[v]) : xold[v] + di * (bv[v] - acc[v]);
            T xt[V];
#pragma unroll
            for (int v = 0; v < V; v++) xt[v] = __shfl_sync(0xffffffffu, x[v], t);
            if (pj[0] == (sl << 5) + t) {
#pragma unroll
                for (int v = 0; v < V; v++) acc[v] += pa[0] * xt[v];
#pragma unroll
                for (int k = 0; k + 1 < kGsPartM; k++) {
                    pj[k] = pj[k + 1];
                    pa[k] = pa[k + 1];
                }
                pj[kGsPartM - 1] = -1;
            }
        }
        if (valid) st_vec<T, V>(xn + e0, x);
    }
}

// Level 0 after the Gauss-Seidel post-smoothing: z = x (widened), r.z and
// (FCG) z.q_old per column; the last block forms rho and beta per column.
template <typename T, bool FCG, int K>
__global__ void __launch_bounds__(kMB) k_gs_finish0_m(int n, const T *__restrict__ x, const double *__restrict__ r64,
                                                     const double *__restrict__ qold, double *__restrict__ z,
                                                     double *partials, CtlM *ctl) {
    constexpr int V = VW<T>::V;
    if (ctl->done) return;
    double rz[V], zq[V];
#pragma unroll
    for (int v = 0; v < V; v++) rz[v] = zq[v] = 0.0;
    MK_LIVE(V)
    MK_FOR(live_ ? n : 0, V) {
        MK_IDX(V)
        T xv[V];
        ld_vec<T, V>(x + e0, xv);
#pragma unroll
        for (int v = 0; v < V; v++) {
            double zo = (double)xv[v];
            z[e0 + v] = zo;
            rz[v] += ldg(r64 + e0 + v) * zo;
            if (FCG) zq[v] += zo * ldg(qold + e0 + v);
        }
    }
    __shared__ double res[2 * kMaxK];
    if (publish_cols<K, V>(rz, zq, partials, &ctl->counter[0])) {
        final_cols<K>(partials, res);
        if (threadIdx.x == 0) ctl->counter[0] = 0;
        int c = threadIdx.x;
        if (c < K && ctl->active[c]) {
            double rho = res[c], zqc = res[K + c];
            if (!isfinite(rho) || !isfinite(zqc)) {
                col_fail(ctl, c, AMG_ERR_NAN);
            } else if (!(rho > 0.0)) {
                col_fail(ctl, c, AMG_ERR_BREAKDOWN);
            } else {
                ctl->rho[c] = rho;
                double beta = 0.0;
                if (!ctl->restart[c])
                    beta = ctl->mode == AMG_MODE_FCG32 || ctl->flex ? -zqc / ctl->pq_old[c] : rho / ctl->rho_old[c];
                ctl->beta[c] = beta;
            }
        }
    }
}

// ------------------------------------------------------------ Krylov
template <int K>
__global__ void __launch_bounds__(kMB) k_axpy_m(int n, const double *__restrict__ z, double *__restrict__ p,
                                               const CtlM *__restrict__ ctl) {
    constexpr int V = 2;
    if (ctl->done) return;
    MK_LIVE(V)
    MK_FOR(live_ ? n : 0, V) {
        MK_IDX(V)
        double zv[V], pv[V], o[V];
        ld_vec<double, V>(z + e0, zv);
        ld_vec_cg<double, V>(p + e0, pv);
#pragma unroll
        for (int v = 0; v < V; v++) o[v] = ctl->active[c0 + v] ? zv[v] + ctl->beta[c0 + v] * pv[v] : 0.0;
        st_vec<double, V>(p + e0, o);
    }
}

template <typename IDX, int K>
__global__ void __launch_bounds__(kMB) k_spmm_m(int n, const int32_t *__restrict__ sptr,
                                               const IDX *__restrict__ col, const double *__restrict__ val,
                                               const double *__restrict__ p, double *__restrict__ q,
                                               double *partials, CtlM *ctl) {
    constexpr int V = 2;
    if (ctl->done) return;
    double pq[V] = {0.0, 0.0}, unused[V] = {0.0, 0.0};
    MK_LIVE(V)
    MK_FOR(live_ ? n : 0, V) {
        MK_IDX(V)
        int s = i >> 5, lane = i & 31;
        int32_t base = ldg(sptr + s);
        int w = (ldg(sptr + s + 1) - base) >> 5;
        double acc[V];
        sell_row_vec<kUnroll, true, V>(col + base + lane, val + base + lane, w, i,
                                       [&](int j, double (&x)[V]) { ld_vec<double, V>(p + (int64_t)j * K + c0, x); },
                                       acc);
        st_vec<double, V>(q + e0, acc);
        double pv[V];
        ld_vec<double, V>(p + e0, pv);
#pragma unroll
        for (int v = 0; v < V; v++) pq[v] += pv[v] * acc[v];
    }
    __shared__ double res[2 * kMaxK];
    if (publish_cols<K, V>(pq, unused, partials, &ctl->counter[1])) {
        final_cols<K>(partials, res);
        if (threadIdx.x == 0) ctl->counter[1] = 0;
        int c = threadIdx.x;
        if (c < K) {
            if (!ctl->active[c]) {
                ctl->alpha[c] = 0.0;
            } else {
                double a = res[c];
                if (!isfinite(a)) col_fail(ctl, c, AMG_ERR_NAN);
                else if (!(a > 0.0)) col_fail(ctl, c, AMG_ERR_BREAKDOWN);
                else {
                    ctl->pq[c] = a;
                    ctl->alpha[c] = ctl->rho[c] / a;
                }
                if (!ctl->active[c]) ctl->alpha[c] = 0.0;
            }
        }
    }
}

// The mode's copy of r for the V-cycle, two columns at a time.
template <int MODE>
__device__ __forceinline__ void emit_r_m(int64_t e, int i, const double (&ri)[2], float *r32, const float *dinv32,
                                         float *xpre32, const double *dinv64, double *xpre64) {
    if (MODE == AMG_MODE_FCG32) {
        float d = __ldg(dinv32 + i);
        float a = (float)ri[0], b = (float)ri[1];
        *reinterpret_cast<float2 *>(r32 + e) = make_float2(a, b);
        *reinterpret_cast<float2 *>(xpre32 + e) = make_float2(d * a, d * b);
    } else {
        double d = __ldg(dinv64 + i);
        *reinterpret_cast<double2 *>(xpre64 + e) = make_double2(d * ri[0], d * ri[1]);
    }
}

template <int MODE, int K>
__global__ void __launch_bounds__(kMB) k_update_m(int n, const double *__restrict__ p,
                                                 const double *__restrict__ q, double *__restrict__ x,
                                                 double *__restrict__ r, float *__restrict__ r32,
                                                 const float *__restrict__ dinv32, float *__restrict__ xpre32,
                                                 const double *__restrict__ dinv64, double *__restrict__ xpre64,
                                                 double *partials, CtlM *ctl, double *hist, int hstride) {
    constexpr int V = 2;
    if (ctl->done) return;
    double rr[V] = {0.0, 0.0}, unused[V] = {0.0, 0.0};
    MK_LIVE(V)
    MK_FOR(live_ ? n : 0, V) {
        MK_IDX(V)
        double rv[V], xv[V], pv[V], qv[V];
        ld_vec_cg<double, V>(r + e0, rv);
        ld_vec_cg<double, V>(x + e0, xv);
        ld_vec<double, V>(p + e0, pv);
        ld_vec<double, V>(q + e0, qv);
#pragma unroll
        for (int v = 0; v < V; v++) {
            if (ctl->active[c0 + v]) {
                double al = ctl->alpha[c0 + v];
                xv[v] = xv[v] + al * pv[v];
                rv[v] = rv[v] - al * qv[v];
                rr[v] += rv[v] * rv[v];
            }
        }
        st_vec<double, V>(x + e0, xv);
        st_vec<double, V>(r + e0, rv);
        emit_r_m<MODE>(e0, i, rv, r32, dinv32, xpre32, dinv64, xpre64);
    }
    __shared__ double res[2 * kMaxK];
    if (publish_cols<K, V>(rr, unused, partials, &ctl->counter[2])) {
        final_cols<K>(partials, res);
        __syncthreads();
        if (threadIdx.x == 0) {
            ctl->counter[2] = 0;
            ctl->iter_all += 1;
            int anycheck = 0;
            for (int c = 0; c < K; c++) {
                if (!ctl->active[c]) continue;
                int it = ctl->iter[c] + 1;
                ctl->iter[c] = it;
                double rel = sqrt(res[c]) / ctl->bnorm[c];
                ctl->rel[c] = rel;
                hist[(int64_t)c * hstride + it] = rel;
                ctl->rho_old[c] = ctl->rho[c];
                ctl->pq_old[c] = ctl->pq[c];
                ctl->restart[c] = 0;
                if (!isfinite(rel)) { col_fail(ctl, c, AMG_ERR_NAN); continue; }
                if (rel <= ctl->rtol) { ctl->check[c] = 1; anycheck = 1; }
                else if (it >= ctl->maxit) col_fail(ctl, c, AMG_ERR_NOCONV);
            }
            ctl->any_check = anycheck;
            update_done(ctl);
        }
    }
}

// r = b - A x. INIT: the columns marked pending (a new right-hand side),
// plus ||b||; otherwise only the columns whose recursive residual met rtol.
// The other columns keep their r.
template <bool INIT, int MODE, typename IDX, int K>
__global__ void __launch_bounds__(kMB) k_residual_m(int n, const int32_t *__restrict__ sptr,
                                                   const IDX *__restrict__ col, const double *__restrict__ val,
                                                   const double *__restrict__ b, const double *__restrict__ x,
                                                   double *__restrict__ r, float *__restrict__ r32,
                                                   const float *__restrict__ dinv32, float *__restrict__ xpre32,
                                                   const double *__restrict__ dinv64, double *__restrict__ xpre64,
                                                   double *partials, CtlM *ctl, double *hist, int hstride) {
    constexpr int V = 2;
    if (ctl->done) return;
    if (!INIT && !ctl->any_check) return;
    double rr[V] = {0.0, 0.0}, bb[V] = {0.0, 0.0};
    MK_FOR(n, V) {
        MK_IDX(V)
        bool use0 = INIT ? ctl->pending[c0] != 0 : ctl->check[c0] != 0;
        bool use1 = INIT ? ctl->pending[c0 + 1] != 0 : ctl->check[c0 + 1] != 0;
        if (!use0 && !use1) continue;
        int s = i >> 5, lane = i & 31;
        int32_t base = ldg(sptr + s);
        int w = (ldg(sptr + s + 1) - base) >> 5;
        double acc[V];
        sell_row_vec<kUnroll, true, V>(col + base + lane, val + base + lane, w, i,
                                       [&](int j, double (&xx)[V]) { ld_vec<double, V>(x + (int64_t)j * K + c0, xx); },
                                       acc);
        double bv[V], rv[V];
        ld_vec<double, V>(b + e0, bv);
        ld_vec_cg<double, V>(r + e0, rv);
        if (use0) rv[0] = bv[0] - acc[0];
        if (use1) rv[1] = bv[1] - acc[1];
        st_vec<double, V>(r + e0, rv);
        emit_r_m<MODE>(e0, i, rv, r32, dinv32, xpre32, dinv64, xpre64);
        if (use0) rr[0] += rv[0] * rv[0];
        if (use1) rr[1] += rv[1] * rv[1];
        if (INIT) {
            if (use0) bb[0] += bv[0] * bv[0];
            if (use1) bb[1] += bv[1] * bv[1];
        }
    }
    __shared__ double res[2 * kMaxK];
    if (publish_cols<K, V>(rr, bb, partials, &ctl->counter[3])) {
        final_cols<K>(partials, res);
        __syncthreads();
        if (threadIdx.x == 0) {
            ctl->counter[3] = 0;
            for (int c = 0; c < K; c++) {
                if (INIT) {
                    if (!ctl->pending[c]) continue;
                    ctl->pending[c] = 0;
                    double bn = sqrt(res[K + c]);
                    ctl->bnorm[c] = bn;
                    ctl->active[c] = 0;
                    ctl->status[c] = AMG_OK;
                    ctl->iter[c] = 0;
                    ctl->check[c] = 0;
                    if (c >= ctl->k) continue;
                    if (!isfinite(bn) || !isfinite(res[c])) { col_fail(ctl, c, AMG_ERR_NAN); continue; }
                    if (bn == 0.0) { ctl->true_rel[c] = 0.0; hist[(int64_t)c * hstride] = 0.0; continue; }
                    double rel = sqrt(res[c]) / bn;
                    ctl->rel[c] = rel;
                    ctl->true_rel[c] = rel;
                    hist[(int64_t)c * hstride] = rel;
                    if (rel <= ctl->rtol) continue;
                    if (ctl->maxit <= 0) { col_fail(ctl, c, AMG_ERR_NOCONV); continue; }
                    ctl->active[c] = 1;
                    ctl->restart[c] = 1;
                } else {
                    if (!ctl->check[c]) continue;
                    ctl->check[c] = 0;
                    double rel = sqrt(res[c]) / ctl->bnorm[c];
                    ctl->true_rel[c] = rel;
                    if (!isfinite(rel)) { col_fail(ctl, c, AMG_ERR_NAN); continue; }
                    if (rel <= ctl->rtol) { ctl->active[c] = 0; ctl->status[c] = AMG_OK; continue; }
                    ctl->restart[c] = 1;
                    hist[(int64_t)c * hstride + ctl->iter[c]] = rel;
                    if (ctl->iter[c] >= ctl->maxit) col_fail(ctl, c, AMG_ERR_NOCONV);
                }
            }
            ctl->any_check = 0;
            update_done(ctl);
        }
    }
}

__global__ void k_zero_m(double *a, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 0.0;
}

// Copies between the caller's n x k block and the internal n x K block.
__global__ void k_pack(const double *__restrict__ src, int k, double *__restrict__ dst, int K, int64_t n) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n * K) return;
    int64_t i = g / K;
    int c = (int)(g % K);
    dst[g] = c < k ? src[i * k + c] : 0.0;
}

// Unpack; columns with b = 0 get x = 0.
__global__ void k_unpack(const double *__restrict__ src, int K, double *__restrict__ dst, int k, int64_t n,
                         const CtlM *__restrict__ ctl) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n * k) return;
    int64_t i = g / k;
    int c = (int)(g % k);
    dst[g] = ctl->bnorm[c] == 0.0 ? 0.0 : src[i * K + c];
}

__global__ void k_set_cond_m(cudaGraphConditionalHandle hc, CtlM *ctl, int count_body) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (count_body) {
        int b = ctl->bodies + 1;
        ctl->bodies = b;
        if (!ctl->done && b > (ctl->maxit + 1) / 2 + 1) {
            for (int c = 0; c < ctl->K; c++)
                if (ctl->active[c]) col_fail(ctl, c, AMG_ERR_NOCONV);
            ctl->done = 1;
        }
    }
    cudaGraphSetConditional(hc, ctl->done ? 0u : 1u);
}

inline int grid_of(int64_t items) { return (int)((items + kMB - 1) / kMB); }

template <typename T>
struct MP;
template <>
struct MP<float> {
    static const float *val(const Level &l) { return l.S.v32; }
    static const float *dinv(const Level &l) { return l.dinv32; }
    static const float *p(const Level &l) { return l.p32; }
    static float *b(MultiLevel &m) { return m.b32; }
    static float *x(MultiLevel &m) { return m.x32; }
    static float *t(MultiLevel &m) { return m.t32; }
    static float *xpre(MultiLevel &m) { return m.xpre32; }
    static float *xp(MultiLevel &m) { return m.xp32; }
    static const float *part(const Level &l, int d) { return l.gs_v32[d]; }
};
template <>
struct MP<double> {
    static const double *val(const Level &l) { return l.S.v64; }
    static const double *dinv(const Level &l) { return l.dinv; }
    static const double *p(const Level &l) { return l.p; }
    static double *b(MultiLevel &m) { return m.b64; }
    static double *x(MultiLevel &m) { return m.x64; }
    static double *t(MultiLevel &m) { return m.t64; }
    static double *xpre(MultiLevel &m) { return m.xpre64; }
    static double *xp(MultiLevel &m) { return m.xp64; }
    static const double *part(const Level &l, int d) { return l.gs_v64[d]; }
};

#define WITH_COLS_M(S, BODY)              \
    do {                                  \
        if ((S).col16) {                  \
            using IDX = int16_t;          \
            const IDX *cols = (S).col16;  \
            BODY;                         \
        } else {                          \
            using IDX = int32_t;          \
            const IDX *cols = (S).col;    \
            BODY;                         \
        }                                 \
    } while (0)

// gs_nu Gauss-Seidel sweeps of level l for K columns: pre-smoothing
// (forward, from zero, into the level's xpre) or post-smoothing (backward,
// from xp, into x); sweeps alternate between the target and t so the last
// writes the target.
template <typename T, int K>
void launch_gs_m(amg_hier *h, MultiWS &W, int l, bool pre, const T *b, T *target, cudaStream_t s) {
    using P = MP<T>;
    constexpr int V = VW<T>::V;
    Level &lv = h->lev[l];
    MultiLevel &mv = W.lev[l];
    const int n = lv.A.n, nu = h->gs_nu, nb = gs_rows(n, h->gs_blocks), d = pre ? 0 : 1;
    const int w = lv.gs_w[d];
    const int grid = grid_of((((int64_t)n + 31) / 32) * (K / V) * 32);
    const T *src = pre ? nullptr : (const T *)P::xp(mv);
    const bool big = n > kSmallRows;
    for (int sw = 1; sw <= nu; sw++) {
        T *dst = (nu - sw) % 2 == 0 ? target : P::t(mv);
        const bool zero = pre && sw == 1;
#define PCG_GSM(UU, ST)                                                                                          \
    do {                                                                                                         \
        if (zero)                                                                                                \
            WITH_COLS_M(lv.S, (k_gs_warp_m<T, IDX, UU, true, true, ST, K><<<grid, kMB, 0, s>>>(                  \
                                  n, nb, w, lv.S.sptr, cols, P::val(lv), lv.gs_ci[d], P::part(lv, d), P::dinv(lv), \
                                  b, src, dst, W.ctl)));                                                         \
        else if (pre)                                                                                            \
            WITH_COLS_M(lv.S, (k_gs_warp_m<T, IDX, UU, true, false, ST, K><<<grid, kMB, 0, s>>>(                 \
                                  n, nb, w, lv.S.sptr, cols, P::val(lv), lv.gs_ci[d], P::part(lv, d), P::dinv(lv), \
                                  b, src, dst, W.ctl)));                                                         \
        else                                                                                                     \
            WITH_COLS_M(lv.S, (k_gs_warp_m<T, IDX, UU, false, false, ST, K><<<grid, kMB, 0, s>>>(                \
                                  n, nb, w, lv.S.sptr, cols, P::val(lv), lv.gs_ci[d], P::part(lv, d), P::dinv(lv), \
                                  b, src, dst, W.ctl)));                                                         \
    } while (0)
        if (l == 0) PCG_GSM(kUnroll, true);
        else if (big) PCG_GSM(kUnroll, false);
        else PCG_GSM(kUnrollSmall, false);
#undef PCG_GSM
        src = dst;
    }
}

template <typename T, bool FCG, int K>
int launch_vcycle_m(amg_hier *h, MultiWS &W, cudaStream_t s) {
    using P = MP<T>;
    constexpr int V = VW<T>::V;
    auto gv = [](int64_t rows) { return grid_of(rows * (K / V)); };
    auto &lev = h->lev;
    int L = (int)lev.size() - 1;
    CtlM *ctl = W.ctl;
    Level &l0 = lev[0];
    MultiLevel &m0 = W.lev[0];
    const T *b0;
    if constexpr (sizeof(T) == 4) b0 = W.r32;
    else b0 = W.r;
    int g0 = W.grid;
    if (L == 0) {
        // single level: z = A^{-1} r through the coarse kernel (float32 rounding as the V-cycle's)
        set_error("pcg_solve_multi: single-level hierarchy not supported by the multi-column path");
        return AMG_ERR_ARG;
    }
    const bool gs = h->gs_nu > 0;
    if (gs) launch_gs_m<T, K>(h, W, 0, true, b0, P::xpre(m0), s);
    WITH_COLS_M(l0.S, (k_down_m<T, IDX, K, kUnroll, true><<<g0, kMB, 0, s>>>(
                          l0.A.n, l0.S.sptr, cols, P::val(l0), P::xpre(m0), b0, P::p(l0), P::t(m0), ctl)));
    for (int l = 0; l < L; l++) {
        Level &lv = lev[l];
        MultiLevel &mv = W.lev[l];
        int n = lv.A.n;
        if (l > 0 && gs) launch_gs_m<T, K>(h, W, l, true, P::b(mv), P::xpre(mv), s);
        if (l > 0)
            WITH_COLS_M(lv.S, (k_down_m<T, IDX, K, kUnroll, false><<<gv(n), kMB, 0, s>>>(
                                  n, lv.S.sptr, cols, P::val(lv), P::xpre(mv), P::b(mv), P::p(lv), P::t(mv), ctl)));
        if (l + 1 == L)
            k_restrict_m<T, double, false, K><<<gv(lv.nc), kMB, 0, s>>>(
                lv.nc, lv.rptr, lv.ridx, P::t(mv), W.bL, nullptr, nullptr, ctl);
        else
            k_restrict_m<T, T, true, K><<<gv(lv.nc), kMB, 0, s>>>(
                lv.nc, lv.rptr, lv.ridx, P::t(mv), P::b(W.lev[l + 1]), P::dinv(lev[l + 1]), P::xpre(W.lev[l + 1]),
                ctl);
    }
    if (h->coarse_iter)
        PCG_TRY(launch_coarse_iter<T>(h, W.cws, W.bL, P::x(W.lev[L]), &ctl->done, ctl->active, s));
    else
        k_coarse_m<T, K><<<grid_of((int64_t)h->nL * (K / 2) * 32), kMB, 0, s>>>(h->nL, h->Ainv, W.bL,
                                                                                P::x(W.lev[L]), ctl);
    for (int l = L - 1; l >= 1; l--) {
        Level &lv = lev[l];
        MultiLevel &mv = W.lev[l];
        int n = lv.A.n;
        k_prolong_m<T, K><<<gv(n), kMB, 0, s>>>(n, P::xpre(mv), P::p(lv), lv.agg,
                                                                  P::x(W.lev[l + 1]), P::xp(mv), ctl);
        if (gs) {
            launch_gs_m<T, K>(h, W, l, false, P::b(mv), P::x(mv), s);
            continue;
        }
        WITH_COLS_M(lv.S, (k_post_m<T, T, false, false, IDX, K, kUnroll, false>
                           <<<gv(n), kMB, 0, s>>>(n, lv.S.sptr, cols, P::val(lv), P::xp(mv),
                                                                    P::b(mv), P::dinv(lv), P::x(mv), nullptr,
                                                                    nullptr, nullptr, ctl)));
    }
    k_prolong_m<T, K><<<g0, kMB, 0, s>>>(l0.A.n, P::xpre(m0), P::p(l0), l0.agg, P::x(W.lev[1]), P::xp(m0), ctl);
    if (gs) {
        launch_gs_m<T, K>(h, W, 0, false, b0, P::x(m0), s);
        k_gs_finish0_m<T, FCG, K><<<g0, kMB, 0, s>>>(l0.A.n, (const T *)P::x(m0), W.r, W.q, W.z, W.partials, ctl);
        PCG_LAUNCH_CK();
        return AMG_OK;
    }
    WITH_COLS_M(l0.S, (k_post_m<T, double, true, FCG, IDX, K, kUnroll, true><<<g0, kMB, 0, s>>>(
                          l0.A.n, l0.S.sptr, cols, P::val(l0), P::xp(m0), b0, P::dinv(l0), W.z, W.r, W.q,
                          W.partials, ctl)));
    PCG_LAUNCH_CK();
    return AMG_OK;
}

template <int K>
int launch_iteration_m(amg_hier *h, MultiWS &W, int mode, cudaStream_t s) {
    Level &l0 = h->lev[0];
    MultiLevel &m0 = W.lev[0];
    int n = l0.A.n;
    if (mode == AMG_MODE_FCG32) PCG_TRY((launch_vcycle_m<float, true, K>(h, W, s)));
    else if (h->coarse_iter) PCG_TRY((launch_vcycle_m<double, true, K>(h, W, s)));  // flexible: FCG(1) beta
    else PCG_TRY((launch_vcycle_m<double, false, K>(h, W, s)));
    k_axpy_m<K><<<W.grid, kMB, 0, s>>>(n, W.z, W.p, W.ctl);
    WITH_COLS_M(l0.S, (k_spmm_m<IDX, K><<<W.grid, kMB, 0, s>>>(n, l0.S.sptr, cols, l0.S.v64, W.p, W.q, W.partials,
                                                               W.ctl)));
    int hs = W.hist_cap;
    if (mode == AMG_MODE_FCG32) {
        k_update_m<AMG_MODE_FCG32, K><<<W.grid, kMB, 0, s>>>(n, W.p, W.q, W.x, W.r, W.r32, l0.dinv32, m0.xpre32,
                                                             l0.dinv, m0.xpre64, W.partials, W.ctl, W.hist, hs);
        WITH_COLS_M(l0.S, (k_residual_m<false, AMG_MODE_FCG32, IDX, K><<<W.grid, kMB, 0, s>>>(
                              n, l0.S.sptr, cols, l0.S.v64, W.b, W.x, W.r, W.r32, l0.dinv32, m0.xpre32, l0.dinv,
                              m0.xpre64, W.partials, W.ctl, W.hist, hs)));
    } else {
        k_update_m<AMG_MODE_PCG64, K><<<W.grid, kMB, 0, s>>>(n, W.p, W.q, W.x, W.r, W.r32, l0.dinv32, m0.xpre32,
                                                             l0.dinv, m0.xpre64, W.partials, W.ctl, W.hist, hs);
        WITH_COLS_M(l0.S, (k_residual_m<false, AMG_MODE_PCG64, IDX, K><<<W.grid, kMB, 0, s>>>(
                              n, l0.S.sptr, cols, l0.S.v64, W.b, W.x, W.r, W.r32, l0.dinv32, m0.xpre32, l0.dinv,
                              m0.xpre64, W.partials, W.ctl, W.hist, hs)));
    }
    PCG_LAUNCH_CK();
    return AMG_OK;
}

// First residual, ||b|| and state of the pending columns only.
template <int K>
int launch_init_residual_m(amg_hier *h, MultiWS &W, int mode, cudaStream_t s) {
    Level &l0 = h->lev[0];
    MultiLevel &m0 = W.lev[0];
    int n = l0.A.n;
    int hs = W.hist_cap;
    if (mode == AMG_MODE_FCG32)
        WITH_COLS_M(l0.S, (k_residual_m<true, AMG_MODE_FCG32, IDX, K><<<W.grid, kMB, 0, s>>>(
                              n, l0.S.sptr, cols, l0.S.v64, W.b, W.x, W.r, W.r32, l0.dinv32, m0.xpre32, l0.dinv,
                              m0.xpre64, W.partials, W.ctl, W.hist, hs)));
    else
        WITH_COLS_M(l0.S, (k_residual_m<true, AMG_MODE_PCG64, IDX, K><<<W.grid, kMB, 0, s>>>(
                              n, l0.S.sptr, cols, l0.S.v64, W.b, W.x, W.r, W.r32, l0.dinv32, m0.xpre32, l0.dinv,
                              m0.xpre64, W.partials, W.ctl, W.hist, hs)));
    PCG_LAUNCH_CK();
    return AMG_OK;
}

template <int K>
int launch_prefix_m(amg_hier *h, MultiWS &W, int mode, cudaStream_t s) {
    int64_t nk = (int64_t)h->lev[0].A.n * K;
    k_zero_m<<<grid_of(nk), kMB, 0, s>>>(W.p, nk);
    k_zero_m<<<grid_of(nk), kMB, 0, s>>>(W.q, nk);
    PCG_LAUNCH_CK();
    return launch_init_residual_m<K>(h, W, mode, s);
}

// Whole multi-column solve as one graph (prefix, then a device-side while
// loop of two iterations per body), as in the single-column path.
template <int K>
int build_graph_m(amg_hier *h, MultiWS &W, int mode) {
    if (!h->cap_stream) PCG_CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = h->cap_stream;
    PCG_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int st = launch_prefix_m<K>(h, W, mode, cs);
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
        k_set_cond_m<<<1, 32, 0, cs>>>(hc, W.ctl, 0);
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
    cudaGraph_t full = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &full);
    if (st || e != cudaSuccess || e2 != cudaSuccess) {
        if (full) cudaGraphDestroy(full);
        if (!st) st = cuda_fail(e != cudaSuccess ? e : e2, "multi solve graph capture", __FILE__, __LINE__);
        return st;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = launch_iteration_m<K>(h, W, mode, cs);
        if (!st) st = launch_iteration_m<K>(h, W, mode, cs);
        if (!st) k_set_cond_m<<<1, 32, 0, cs>>>(hc, W.ctl, 1);
        cudaGraph_t bout = body;
        e = cudaStreamEndCapture(cs, &bout);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (st || e != cudaSuccess) {
        cudaGraphDestroy(full);
        if (!st) st = cuda_fail(e, "multi solve graph body capture", __FILE__, __LINE__);
        return st;
    }
    e = cudaGraphInstantiate(&W.gexec[mode], full, 0);
    cudaGraphDestroy(full);
    if (e != cudaSuccess) {
        W.gexec[mode] = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate (multi)", __FILE__, __LINE__);
    }
    return AMG_OK;
}

bool is_dev(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Workspace of K columns (reallocated when K or the history length grows).
int ensure_ws(amg_hier *h, int K, int maxit) {
    MultiWS &W = h->multi;
    if (W.K == K && W.hist_cap >= maxit + 1) return AMG_OK;
    mws_free(h->mem, W);
    return mws_alloc(h, h->mem, W, K, maxit + 1 > 1001 ? maxit + 1 : 1001, 3);
}

template <int K>
int solve_multi_k(amg_hier *h, int k, const double *B, double *X, double rtol, int maxit, int *iters,
                  double *res_hist, cudaStream_t s) {
    PCG_TRY(ensure_ws(h, K, maxit));
    MultiWS &W = h->multi;
    int n = h->lev[0].A.n;
    int64_t nk = (int64_t)n * K;
    int64_t nkk = (int64_t)n * k;
    Mem &M = h->mem;
    M.stream = s;
    // inputs into the internal n x K block (through a device staging copy when on the host)
    const double *bsrc = B, *xsrc = X;
    double *stage = nullptr;
    bool bdev = is_dev(B), xdev = is_dev(X);
    if (!bdev || !xdev) PCG_TRY(alloc(M, &stage, (size_t)nkk));
    if (!bdev) {
        PCG_CK(cudaMemcpyAsync(stage, B, sizeof(double) * nkk, cudaMemcpyHostToDevice, s));
        bsrc = stage;
    }
    k_pack<<<grid_of(nk), kMB, 0, s>>>(bsrc, k, W.b, K, n);
    if (!xdev) {
        PCG_CK(cudaMemcpyAsync(stage, X, sizeof(double) * nkk, cudaMemcpyHostToDevice, s));
        xsrc = stage;
    }
    k_pack<<<grid_of(nk), kMB, 0, s>>>(xsrc, k, W.x, K, n);
    PCG_LAUNCH_CK();
    CtlM c0;
    memset(&c0, 0, sizeof(c0));
    c0.rtol = rtol;
    c0.maxit = maxit;
    c0.mode = h->mode;
    c0.flex = h->coarse_iter;
    c0.k = k;
    c0.K = K;
    for (int q = 0; q < K; q++) c0.pending[q] = 1;
    *W.ctl_host = c0;
    PCG_CK(cudaMemcpyAsync(W.ctl, W.ctl_host, sizeof(CtlM), cudaMemcpyHostToDevice, s));
    int mode = h->mode;
    bool graph = h->use_graph;
    if (graph && !W.gexec[mode]) {
        if (build_graph_m<K>(h, W, mode) != AMG_OK) graph = false;
    }
    if (graph) {
        PCG_CK(cudaGraphLaunch(W.gexec[mode], s));
        PCG_CK(cudaMemcpyAsync(W.ctl_host, W.ctl, sizeof(CtlM), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaStreamSynchronize(s));
    } else {
        PCG_TRY(launch_prefix_m<K>(h, W, mode, s));
        int launched = 0;
        for (;;) {
            PCG_CK(cudaMemcpyAsync(W.ctl_host, W.ctl, sizeof(CtlM), cudaMemcpyDeviceToHost, s));
            PCG_CK(cudaStreamSynchronize(s));
            if (W.ctl_host->done || launched >= maxit) break;
            for (int q = 0; q < 4 && launched < maxit; q++, launched++) PCG_TRY(launch_iteration_m<K>(h, W, mode, s));
        }
    }
    CtlM &c = *W.ctl_host;
    double *xdst = xdev ? X : stage;
    k_unpack<<<grid_of(nkk), kMB, 0, s>>>(W.x, K, xdst, k, n, W.ctl);
    PCG_LAUNCH_CK();
    if (!xdev) PCG_CK(cudaMemcpyAsync(X, stage, sizeof(double) * nkk, cudaMemcpyDeviceToHost, s));
    if (res_hist) {
        int hl = maxit + 1;
        for (int q = 0; q < k; q++)
            PCG_CK(cudaMemcpyAsync(res_hist + (int64_t)q * hl, W.hist + (int64_t)q * W.hist_cap,
                                   sizeof(double) * (c.iter[q] + 1), cudaMemcpyDefault, s));
    }
    PCG_CK(cudaStreamSynchronize(s));
    if (stage) release(M, stage);
    int st = AMG_OK;
    for (int q = 0; q < k; q++) {
        if (iters) iters[q] = c.iter[q];
        h->multi_status[q] = c.status[q];
        h->multi_true_rel[q] = c.true_rel[q];
        if (c.status[q] != AMG_OK && st == AMG_OK) st = c.status[q];
    }
    h->multi_k = k;
    if (st) set_error("pcg_solve_multi: some columns failed (status %d; see amg_multi_info)", st);
    return st;
}

}  // namespace

// Whether the multi-column kernels can smooth h by Gauss-Seidel: every level
// with sweeps has blocks whose size divides 32 and at most kGsPartM
// already-updated in-block entries per row in each pass (one-warp sweeps).
bool gs_multi_ok(const amg_hier *h) {
    if (h->gs_nu <= 0) return true;
    for (size_t l = 0; l + 1 < h->lev.size(); l++) {
        const Level &lv = h->lev[l];
        int nb = gs_rows(lv.A.n, h->gs_blocks);
        if (nb > 32 || 32 % nb) return false;
        for (int d = 0; d < 2; d++)
            if (lv.gs_w[d] < 0 || lv.gs_w[d] > kGsPartM) return false;
    }
    return true;
}

// Allocates a K-column workspace; which: 1 float32 V-cycle vectors,
// 2 float64 V-cycle vectors, 3 both.
int mws_alloc(amg_hier *h, Mem &M, MultiWS &W, int K, int hist_cap, int which) {
    int L = (int)h->lev.size() - 1;
    int n0 = h->lev[0].A.n;
    int64_t nk = (int64_t)n0 * K;
    W.K = K;
    W.hist_cap = hist_cap;
    PCG_TRY(alloc(M, &W.b, nk));
    PCG_TRY(alloc(M, &W.x, nk));
    PCG_TRY(alloc(M, &W.r, nk));
    PCG_TRY(alloc(M, &W.z, nk));
    PCG_TRY(alloc(M, &W.p, nk));
    PCG_TRY(alloc(M, &W.q, nk));
    PCG_TRY(alloc(M, &W.r32, nk));
    W.lev.assign(L + 1, MultiLevel{});
    for (int l = 0; l <= L; l++) {
        int64_t m = (int64_t)h->lev[l].A.n * K;
        MultiLevel &v = W.lev[l];
        if (which & 1) {
            PCG_TRY(alloc(M, &v.b32, m));
            PCG_TRY(alloc(M, &v.x32, m));
            PCG_TRY(alloc(M, &v.t32, m));
            PCG_TRY(alloc(M, &v.xpre32, m));
            PCG_TRY(alloc(M, &v.xp32, m));
        }
        if (which & 2) {
            PCG_TRY(alloc(M, &v.b64, m));
            PCG_TRY(alloc(M, &v.x64, m));
            PCG_TRY(alloc(M, &v.t64, m));
            PCG_TRY(alloc(M, &v.xpre64, m));
            PCG_TRY(alloc(M, &v.xp64, m));
        }
    }
    PCG_TRY(alloc(M, &W.bL, (int64_t)h->nL * K));
    W.flex = h->coarse_iter;
    if (h->coarse_iter) PCG_TRY(cws_alloc(h, M, W.cws, K));
    int sms = 0;
    PCG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    int64_t want = (nk + kMB - 1) / kMB;
    int64_t cap = (int64_t)sms * 8;
    W.grid = (int)(want < cap ? want : cap);
    if (W.grid < 1) W.grid = 1;
    PCG_TRY(alloc(M, &W.partials, (size_t)2 * K * W.grid));
    PCG_TRY(alloc(M, &W.ctl, 1));
    PCG_TRY(alloc(M, &W.hist, (size_t)K * W.hist_cap));
    if (M.dry) return AMG_OK;
    PCG_CK(cudaMemsetAsync(W.ctl, 0, sizeof(CtlM), M.stream));
    PCG_CK(cudaMallocHost(&W.ctl_host, sizeof(CtlM)));
    return AMG_OK;
}

// Device bytes that mws_alloc takes for this workspace shape (exact: the
// same requests, counted by a dry-run pool).
size_t mws_bytes(amg_hier *h, int K, int hist_cap, int which) {
    Mem M;
    M.dry = true;
    MultiWS W;
    if (mws_alloc(h, M, W, K, hist_cap, which)) return (size_t)-1;
    return M.bytes;
}

void mws_free(Mem &M, MultiWS &W) {
    for (auto &g : W.gexec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    if (W.step_exec) cudaGraphExecDestroy(W.step_exec);
    if (W.step_graph) cudaGraphDestroy(W.step_graph);
    W.step_exec = nullptr;
    W.step_graph = nullptr;
    W.step_iters = 0;
    W.step_mode = -1;
    release(M, W.b);
    release(M, W.x);
    release(M, W.r);
    release(M, W.z);
    release(M, W.p);
    release(M, W.q);
    release(M, W.r32);
    for (auto &v : W.lev) {
        release(M, v.b32); release(M, v.x32); release(M, v.t32); release(M, v.xpre32); release(M, v.xp32);
        release(M, v.b64); release(M, v.x64); release(M, v.t64); release(M, v.xpre64); release(M, v.xp64);
    }
    W.lev.clear();
    release(M, W.bL);
    cws_free(M, W.cws);
    release(M, W.partials);
    release(M, W.ctl);
    release(M, W.hist);
    if (W.ctl_host) cudaFreeHost(W.ctl_host);
    W.ctl_host = nullptr;
    W.K = 0;
    W.hist_cap = 0;
}

void free_multi(amg_hier *h) { mws_free(h->mem, h->multi); }

namespace {

// Column c of a new request: b and x0 in, and p = q = 0 (the first
// iteration's p = z + 0 p and FCG's z.q_old must not see an earlier
// occupant's values).
__global__ void k_col_put(const double *__restrict__ b, const double *__restrict__ x0, double *__restrict__ B,
                          double *__restrict__ X, double *__restrict__ P, double *__restrict__ Q, int K, int c,
                          int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t e = (int64_t)i * K + c;
    B[e] = b[i];
    X[e] = x0[i];
    P[e] = 0.0;
    Q[e] = 0.0;
}

// Marks new columns for initialisation and wakes the solve up.
__global__ void k_admit(CtlM *ctl, unsigned mask) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int c = 0; c < ctl->K; c++)
        if (mask & (1u << c)) {
            ctl->pending[c] = 1;
            ctl->active[c] = 0;
            ctl->status[c] = AMG_OK;
        }
    ctl->done = 0;
}

// Only the new columns' p and q were cleared (by their put): the running
// columns keep their search directions.
template <int K>
int mws_init_pending(amg_hier *h, MultiWS &W, int mode, cudaStream_t s) {
    return launch_init_residual_m<K>(h, W, mode, s);
}

}  // namespace

// Resets a workspace's state: no column in use, solve idle.
int mws_reset(MultiWS &W, int mode, double rtol, int maxit, cudaStream_t s) {
    CtlM c0;
    memset(&c0, 0, sizeof(c0));
    c0.rtol = rtol;
    c0.maxit = maxit;
    c0.mode = mode;
    c0.flex = W.flex;
    c0.k = W.K;
    c0.K = W.K;
    c0.done = 1;
    *W.ctl_host = c0;
    PCG_CK(cudaMemcpyAsync(W.ctl, W.ctl_host, sizeof(CtlM), cudaMemcpyHostToDevice, s));
    PCG_CK(cudaStreamSynchronize(s));
    return AMG_OK;
}

int mws_put_column(MultiWS &W, int c, const double *b_dev, const double *x_dev, int n, cudaStream_t s) {
    k_col_put<<<(n + kMB - 1) / kMB, kMB, 0, s>>>(b_dev, x_dev, W.b, W.x, W.p, W.q, W.K, c, n);
    PCG_LAUNCH_CK();
    return AMG_OK;
}

// Starts the columns in mask: residual, ||b|| and state of each, while the
// other columns keep their place in their own iterations.
int mws_admit(amg_hier *h, MultiWS &W, int mode, unsigned mask, cudaStream_t s) {
    k_admit<<<1, 32, 0, s>>>(W.ctl, mask);
    PCG_LAUNCH_CK();
    switch (W.K) {
        case 4: return mws_init_pending<4>(h, W, mode, s);
        case 8: return mws_init_pending<8>(h, W, mode, s);
        case 16: return mws_init_pending<16>(h, W, mode, s);
        default: return mws_init_pending<32>(h, W, mode, s);
    }
}

// `iterations` iterations of every active column (kernels of finished
// columns do no work), then the state is copied to the pinned host mirror.
// The chunk is captured once as a graph (kept in W) that every later call
// replays; launch = 0 only captures it.
int mws_iterate(amg_hier *h, MultiWS &W, int mode, int iterations, cudaStream_t s, int launch) {
    if (!W.step_exec || W.step_iters != iterations || W.step_mode != mode) {
        if (W.step_exec) cudaGraphExecDestroy(W.step_exec);
        if (W.step_graph) cudaGraphDestroy(W.step_graph);
        W.step_exec = nullptr;
        W.step_graph = nullptr;
        if (!h->cap_stream) PCG_CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        cudaStream_t cs = h->cap_stream;
        PCG_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int st = AMG_OK;
        for (int k = 0; k < iterations && !st; k++) {
            switch (W.K) {
                case 4: st = launch_iteration_m<4>(h, W, mode, cs); break;
                case 8: st = launch_iteration_m<8>(h, W, mode, cs); break;
                case 16: st = launch_iteration_m<16>(h, W, mode, cs); break;
                default: st = launch_iteration_m<32>(h, W, mode, cs); break;
            }
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&W.step_exec, g, 0);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            W.step_exec = nullptr;
            return cuda_fail(e, "serving step graph", __FILE__, __LINE__);
        }
        W.step_graph = g;
        W.step_iters = iterations;
        W.step_mode = mode;
    }
    if (!launch) return AMG_OK;
    PCG_CK(cudaGraphLaunch(W.step_exec, s));
    PCG_CK(cudaMemcpyAsync(W.ctl_host, W.ctl, sizeof(CtlM), cudaMemcpyDeviceToHost, s));
    return AMG_OK;
}

int solve_multi_impl(amg_hier *h, int k, const double *B, double *X, double rtol, int maxit, int *iters,
                     double *res_hist, cudaStream_t s) {
    if (k < 1 || k > kMaxK || !B || !X || !(rtol >= 0.0) || maxit < 0) {
        set_error("pcg_solve_multi: bad arguments (1 <= k <= 32, rtol >= 0, maxit >= 0)");
        return AMG_ERR_ARG;
    }
    if (h->lev.size() < 2) {
        set_error("pcg_solve_multi: the hierarchy has a single level; use pcg_solve per column");
        return AMG_ERR_ARG;
    }
    int K = 4;
    while (K < k) K <<= 1;
    switch (K) {
        case 4: return solve_multi_k<4>(h, k, B, X, rtol, maxit, iters, res_hist, s);
        case 8: return solve_multi_k<8>(h, k, B, X, rtol, maxit, iters, res_hist, s);
        case 16: return solve_multi_k<16>(h, k, B, X, rtol, maxit, iters, res_hist, s);
        default: return solve_multi_k<32>(h, k, B, X, rtol, maxit, iters, res_hist, s);
    }
}

}  // namespace pcgamg
