// Iterative coarsest solve (arxiv 2210.16660, Sec. 3.1, coarsest solver):
// flexible CG preconditioned by block-Jacobi whose blocks are solved by an
// incomplete LU factorization with one level of fill-in, ILU(1); the
// iteration stops once ||r|| <= tol ||b|| (tol = 1e-3: three orders of
// magnitude) or after maxit (30) iterations, starting from x = 0.
//
// Blocks are 32 consecutive rows of the coarsest matrix, one sliced-ELL
// slice: a warp owns a block, a lane a row. Setup factors each block with
// the level-of-fill ILU(1) in row (IKJ) order, with the rounding of each
// operation spelled out so the factors equal a sequential CPU factorization
// bit for bit, then forms the block's dense inverse M_b^{-1} = (L_b U_b)^{-1}.
// Applying the preconditioner is then a 32 x 32 matrix-vector product per
// block done with warp shuffles: 32 independent FMAs per lane instead of two
// chains of dependent substitutions (GB300 has ~2 float64 FMAs per clock per
// SM, so the count of float64 warp instructions is what the apply costs).
//
// One inner iteration is two launches (no grid-wide waits):
//   k_cq : p = z + beta p_old (into the other p buffer) and q = A p, formed
//          as A z + beta q_old (A p_old = q_old: one gathered vector and one
//          FMA per stored entry), p.q; the last block forms alpha = rho / p.q
//   k_cx : x += alpha p, r -= alpha q, z = M^{-1} r (block-local), and the
//          partial sums r.r, r.z, z.q; the last block applies the stop test
//          and forms rho and beta = -(z.q) / (p.q)_old of the next iteration
// The maxit iterations are launched unconditionally; a kernel whose solve
// has stopped in every column returns at once. Reductions are two-stage and
// deterministic (block partials, summed in block order by the last block).
// K columns (multi right-hand-side solves) run side by side, each with its
// own scalars and stop; a thread owns KC = 1 or 2 adjacent columns of a row.
#include <cmath>
#include <cstdio>

#include "internal.cuh"

namespace pcgamg {

namespace {

constexpr int kB = kCoarseBlock;  // 32 rows per block
constexpr int kCT = 256;          // threads per block of the solve kernels
constexpr int kCW = kCT / 32;     // warps per block
constexpr int kNoLev = 1 << 20;   // "no entry" level of fill
constexpr int kQU = 4;            // matrix entries a lane loads ahead of their gathers

// ------------------------------------------------------------------ setup
// ILU(1) of block b, one thread per block. Row il of the block: the stored
// entries (i, j) with j in the block start at level 0; eliminating with the
// earlier rows k (increasing, entries of level <= 1 only): l_ik = a_ik / u_kk,
// then a_ij -= l_ik u_kj for every kept upper entry of row k, lev_ij =
// min(lev_ij, lev_ik + lev_kj + 1); the row keeps its entries of level <= 1.
// Operations round one at a time (no contraction), as the CPU oracle's. F
// receives the factors (row-major per block); flag bit 0 is set when a
// pivot is not a positive finite number.
__global__ void k_ilu1(int n, int nb, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const double *__restrict__ v, double *__restrict__ F, int *flag) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int s = b * kB, m = min(kB, n - s);
    double *Fb = F + (int64_t)b * kB * kB;
    unsigned char lv[kB][kB];  // level of each kept entry of the rows done so far
    double w[kB];
    int wl[kB];
    for (int il = 0; il < kB; il++) {
        for (int j = 0; j < kB; j++) Fb[il * kB + j] = 0.0;
    }
    for (int il = 0; il < m; il++) {
        int i = s + il;
        for (int j = 0; j < kB; j++) { w[j] = 0.0; wl[j] = kNoLev; }
        for (int32_t q = rp[i]; q < rp[i + 1]; q++) {
            int j = ci[q] - s;
            if (j >= 0 && j < m) { w[j] = v[q]; wl[j] = 0; }
        }
        for (int k = 0; k < il; k++) {
            if (wl[k] > 1) continue;
            double lik = __ddiv_rn(w[k], Fb[k * kB + k]);
            w[k] = lik;
            for (int j = k + 1; j < m; j++) {
                if (lv[k][j] > 1) continue;
                w[j] = __dsub_rn(w[j], __dmul_rn(lik, Fb[k * kB + j]));
                int nl = wl[k] + (int)lv[k][j] + 1;
                if (nl < wl[j]) wl[j] = nl;
            }
        }
        for (int j = 0; j < kB; j++) {
            bool keep = j < m && wl[j] <= 1;
            lv[il][j] = keep ? (unsigned char)wl[j] : (unsigned char)255;
            Fb[il * kB + j] = keep ? w[j] : 0.0;
        }
        double piv = w[il];
        if (!(piv > 0.0) || !isfinite(piv)) atomicOr(flag, 1);
    }
}

// Column j of (L_b U_b)^{-1}, one thread per (block, column): L y = e_j
// (unit lower), U x = y; rows past the block's end are the identity.
__global__ void k_block_inverse(int n, int nb, const double *__restrict__ F, double *__restrict__ Minv) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * kB) return;
    int b = t / kB, j = t % kB;
    int m = min(kB, n - b * kB);
    const double *Fb = F + (int64_t)b * kB * kB;
    double *out = Minv + (int64_t)b * kB * kB + (int64_t)j * kB;
    double y[kB];
    for (int i = 0; i < kB; i++) y[i] = i == j ? 1.0 : 0.0;
    if (j < m) {
        for (int i = 0; i < m; i++) {
            double acc = y[i];
            for (int k = 0; k < i; k++) acc -= Fb[i * kB + k] * y[k];
            y[i] = acc;
        }
        for (int i = m - 1; i >= 0; i--) {
            double acc = y[i];
            for (int k = m - 1; k > i; k--) acc -= Fb[i * kB + k] * y[k];
            y[i] = acc / Fb[i * kB + i];
        }
    }
    for (int i = 0; i < kB; i++) out[i] = y[i];
}

// ------------------------------------------------------------ solve kernels
template <int KC>
__device__ __forceinline__ void ld_cols(const double *p, double (&o)[KC]) {
    if constexpr (KC == 2) {
        double2 u = __ldg(reinterpret_cast<const double2 *>(p));
        o[0] = u.x;
        o[1] = u.y;
    } else {
        o[0] = __ldg(p);
    }
}

template <int KC>
__device__ __forceinline__ void st_cols(double *p, const double (&o)[KC]) {
    if constexpr (KC == 2) *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
    else p[0] = o[0];
}

// z_b = M_b^{-1} r_b for this warp's block: lane i sums (M^{-1})_{ik} r_k over
// k = 0..31 in order, r_k taken from lane k.
// All 32 entries of the lane's row are loaded before the first FMA (one
// round trip to L2 instead of a chain of them).
__device__ __forceinline__ void block_row(const double *__restrict__ Mb, int lane, double (&m)[kB]) {
#pragma unroll
    for (int k = 0; k < kB; k++) m[k] = __ldg(Mb + k * kB + lane);
}

template <int KC>
__device__ __forceinline__ void block_apply_m(const double (&m)[kB], const double (&r)[KC], double (&z)[KC]) {
#pragma unroll
    for (int v = 0; v < KC; v++) z[v] = 0.0;
#pragma unroll
    for (int k = 0; k < kB; k++) {
#pragma unroll
        for (int v = 0; v < KC; v++) z[v] = fma(m[k], __shfl_sync(0xffffffffu, r[v], k), z[v]);
    }
}

template <int KC>
__device__ __forceinline__ void block_apply(const double *__restrict__ Mb, const double (&r)[KC], double (&z)[KC],
                                            int lane) {
    double m[kB];
    block_row(Mb, lane, m);
#pragma unroll
    for (int v = 0; v < KC; v++) z[v] = 0.0;
#pragma unroll
    for (int k = 0; k < kB; k++) {
#pragma unroll
        for (int v = 0; v < KC; v++) z[v] = fma(m[k], __shfl_sync(0xffffffffu, r[v], k), z[v]);
    }
}

// Block partials of NQ quantities per column. a[q][v]: this thread's sums
// for column g*KC + v (g = the warp's column group, fixed over its items).
// Layout [q][column][block]; returns true in every thread of the last block.
template <int KC, int NQ>
__device__ __forceinline__ bool publish(double (&a)[NQ][KC], int g, bool valid, int K, double *partials,
                                        unsigned *counter) {
    __shared__ double sh[kCW][NQ][KC];
    __shared__ int sg[kCW];
    __shared__ bool last;
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NQ; q++)
#pragma unroll
        for (int v = 0; v < KC; v++) {
            double x = a[q][v];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            a[q][v] = x;
        }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; q++)
#pragma unroll
            for (int v = 0; v < KC; v++) sh[w][q][v] = a[q][v];
        sg[w] = valid ? g : -1;
    }
    __syncthreads();
    int G = gridDim.x;
    for (int t = threadIdx.x; t < NQ * K; t += blockDim.x) {
        int q = t / K, c = t % K;
        double s = 0.0;
        for (int ww = 0; ww < kCW; ww++)
            if (sg[ww] == c / KC) s += sh[ww][q][c % KC];
        partials[(int64_t)t * G + blockIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        last = (t == (unsigned)G - 1);
    }
    __syncthreads();
    return last;
}

// Last block: res[t] = sum over blocks (in block order) of partials[t][.],
// t < NQ K; res is shared memory.
template <int NQ>
__device__ __forceinline__ void final_sums(const double *partials, int K, double *res) {
    __threadfence();
    int G = gridDim.x;
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = w; t < NQ * K; t += kCW) {
        const double *src = partials + (int64_t)t * G;
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
        if (lane == 0) res[t] = s;
    }
    __syncthreads();
}

// A thread's items: warp index wg over nb * G (block, group) pairs; the
// total warp count is a multiple of G, so a warp's group is fixed.
struct Items {
    int wg, nw, g;
};
__device__ __forceinline__ Items items(int G) {
    Items it;
    it.wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    it.nw = (gridDim.x * blockDim.x) >> 5;
    it.g = it.wg % G;
    return it;
}

// Start: x = 0, r = b, z = M^{-1} b, ||b||^2 and r.z; the last block sets
// each column's state (a column whose ||b|| or r.z is not a positive finite
// number, or whose outer solve has stopped, does not iterate: x = 0).
template <int KC, typename TO>
__global__ void __launch_bounds__(kCT) k_cinit(int n, int nb, int K, const double *__restrict__ bL,
                                               TO *__restrict__ xo, double *__restrict__ x, double *__restrict__ r,
                                               double *__restrict__ z, const double *__restrict__ Minv,
                                               double *partials, CCtl *ctl, const int *outer_done,
                                               const int *outer_live) {
    pdl_enter();
    if (*outer_done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->any = 0;
        return;
    }
    int G = K / KC;
    Items it = items(G);
    int lane = threadIdx.x & 31;
    int c0 = it.g * KC;
    double acc[2][KC] = {};
    for (int wi = it.wg; wi < nb * G; wi += it.nw) {
        int b = wi / G, i = b * kB + lane;
        double bv[KC], zv[KC], zero[KC];
#pragma unroll
        for (int v = 0; v < KC; v++) zero[v] = 0.0;
        if (i < n) ld_cols<KC>(bL + (int64_t)i * K + c0, bv);
        else
#pragma unroll
            for (int v = 0; v < KC; v++) bv[v] = 0.0;
        block_apply<KC>(Minv + (int64_t)b * kB * kB, bv, zv, lane);
        int64_t o = (int64_t)i * K + c0;
        st_cols<KC>(x + o, zero);
        st_cols<KC>(r + o, bv);
        st_cols<KC>(z + o, zv);
        if (i < n)
#pragma unroll
            for (int v = 0; v < KC; v++) xo[o + v] = (TO)0;
#pragma unroll
        for (int v = 0; v < KC; v++) {
            acc[0][v] += bv[v] * bv[v];
            acc[1][v] += bv[v] * zv[v];
        }
    }
    if (publish<KC, 2>(acc, it.g, it.wg < nb * G, K, partials, &ctl->counter[0])) {
        __shared__ double res[2 * 32];
        final_sums<2>(partials, K, res);
        if (threadIdx.x == 0) {
            int any = 0;
            for (int c = 0; c < K; c++) {
                double bn = sqrt(res[c]), rz = res[K + c];
                int live = outer_live ? outer_live[c] : 1;
                int a = live && bn > 0.0 && isfinite(bn) && rz > 0.0 && isfinite(rz);
                ctl->bn[c] = bn;
                ctl->rho[c] = rz;
                ctl->beta[c] = 0.0;
                ctl->its[c] = 0;
                ctl->active[c] = a;
                any |= a;
            }
            ctl->any = any;
            ctl->counter[0] = 0;
        }
    }
}

// p_new = z + beta p_old and q = A p_new = A z + beta q_old over the
// sliced-ELL slices (q_old = A p_old from the previous iteration), p.q; the
// last block forms alpha = rho / p.q (a p.q that is not a positive finite
// number stops the column with its current x). Four lanes share a row: lane
// quarter s takes the row's entries s, s+4, s+8, ... in chunks whose columns
// and values are all loaded before their gathers, and the four partial sums
// meet in a shuffle tree ((s0 + s1) + (s2 + s3)), so a warp covers 8 rows of
// a slice and the longest row's chain is a quarter of its length. The first
// chunk's columns and values (written at setup only) are loaded before the
// wait for the preceding kernel.
template <int KC, typename IDX>
__global__ void __launch_bounds__(kCT) k_cq(int n, int nb, int K, const int32_t *__restrict__ sptr,
                                            const IDX *__restrict__ col, const double *__restrict__ val,
                                            const double *__restrict__ z, const double *__restrict__ pold,
                                            double *__restrict__ pnew, double *__restrict__ q, double *partials,
                                            CCtl *ctl) {
    int G = K / KC;
    Items it = items(G);
    int lane = threadIdx.x & 31, s = lane & 3;
    // the warp's first item: its matrix chunk does not depend on earlier kernels
    int j0[kQU];
    double a0[kQU];
    int wdt0 = 0;
    int32_t base0 = 0;
    {
        int wi = it.wg;
        int b = wi / (4 * G), quarter = (wi / G) & 3;
        int rl = 8 * quarter + (lane >> 2), i = b * kB + rl;
#pragma unroll
        for (int u = 0; u < kQU; u++) { j0[u] = 0; a0[u] = 0.0; }
        if (wi < nb * 4 * G && i < n) {
            base0 = __ldg(sptr + b);
            wdt0 = (__ldg(sptr + b + 1) - base0) >> 5;
            if (s < wdt0) {
#pragma unroll
                for (int u = 0; u < kQU; u++) {
                    int k = s + 4 * u;
                    int kk = k < wdt0 ? k : s;
                    if constexpr (sizeof(IDX) == 2) j0[u] = i + (int)__ldg(col + base0 + rl + kk * kB);
                    else j0[u] = __ldg(col + base0 + rl + kk * kB);
                    double av = __ldg(val + base0 + rl + kk * kB);
                    a0[u] = k < wdt0 ? av : 0.0;
                }
            }
        }
    }
    pdl_enter();
    z = after_wait(z);
    pold = after_wait(pold);
    pnew = after_wait(pnew);
    q = after_wait(q);
    if (!ctl->any) return;
    int c0 = it.g * KC;
    double beta[KC];
    bool live = false, first = true;
#pragma unroll
    for (int v = 0; v < KC; v++) {
        beta[v] = ctl->beta[c0 + v];
        live |= ctl->active[c0 + v] != 0;
    }
    double acc[1][KC] = {};
    if (live) {
        for (int wi = it.wg; wi < nb * 4 * G; wi += it.nw, first = false) {
            int b = wi / (4 * G), quarter = (wi / G) & 3;
            int rl = 8 * quarter + (lane >> 2);  // row within the slice
            int i = b * kB + rl;
            double qi[KC];
#pragma unroll
            for (int v = 0; v < KC; v++) qi[v] = 0.0;
            if (i < n) {
                int32_t base = first ? base0 : __ldg(sptr + b);
                int wdt = first ? wdt0 : (__ldg(sptr + b + 1) - base) >> 5;
                const IDX *cp = col + base + rl;
                const double *ap = val + base + rl;
                for (int k0 = s; k0 < wdt; k0 += 4 * kQU) {
                    int j[kQU];
                    double a[kQU];
                    if (first && k0 == s) {
#pragma unroll
                        for (int u = 0; u < kQU; u++) { j[u] = j0[u]; a[u] = a0[u]; }
                    } else {
#pragma unroll
                        for (int u = 0; u < kQU; u++) {
                            int k = k0 + 4 * u;
                            int kk = k < wdt ? k : k0;  // a valid entry of the row
                            if constexpr (sizeof(IDX) == 2) j[u] = i + (int)__ldg(cp + kk * kB);
                            else j[u] = __ldg(cp + kk * kB);
                            double av = __ldg(ap + kk * kB);
                            a[u] = k < wdt ? av : 0.0;
                        }
                    }
                    double zj[kQU][KC];
#pragma unroll
                    for (int u = 0; u < kQU; u++) ld_cols<KC>(z + (int64_t)j[u] * K + c0, zj[u]);
#pragma unroll
                    for (int u = 0; u < kQU; u++)
#pragma unroll
                        for (int v = 0; v < KC; v++) qi[v] = fma(a[u], zj[u][v], qi[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < KC; v++) {
                qi[v] += __shfl_xor_sync(0xffffffffu, qi[v], 1);
                qi[v] += __shfl_xor_sync(0xffffffffu, qi[v], 2);
            }
            if (s == 0) {
                int64_t o = (int64_t)i * K + c0;
                double zi[KC], pi[KC], qo[KC];
                ld_cols<KC>(z + o, zi);
                ld_cols<KC>(pold + o, pi);
                ld_cols<KC>(q + o, qo);
#pragma unroll
                for (int v = 0; v < KC; v++) {
                    if (beta[v] != 0.0) {
                        pi[v] = zi[v] + beta[v] * pi[v];
                        qi[v] = qi[v] + beta[v] * qo[v];
                    } else {
                        pi[v] = zi[v];
                    }
                }
                st_cols<KC>(pnew + o, pi);
                st_cols<KC>(q + o, qi);
#pragma unroll
                for (int v = 0; v < KC; v++) acc[0][v] += pi[v] * qi[v];
            }
        }
    }
    if (publish<KC, 1>(acc, it.g, it.wg < nb * 4 * G, K, partials, &ctl->counter[1])) {
        __shared__ double res[32];
        final_sums<1>(partials, K, res);
        if (threadIdx.x == 0) {
            int any = 0;
            for (int c = 0; c < K; c++) {
                if (ctl->active[c]) {
                    double pq = res[c];
                    if (pq > 0.0 && isfinite(pq)) {
                        ctl->pq[c] = pq;
                        ctl->alpha[c] = ctl->rho[c] / pq;
                    } else {
                        ctl->active[c] = 0;
                    }
                }
                any |= ctl->active[c];
            }
            ctl->any = any;
            ctl->counter[1] = 0;
        }
    }
}

// x += alpha p, r -= alpha q, z = M^{-1} r, partials r.r, r.z, z.q; the last
// block applies the stop test of iteration `iter` (||r|| <= tol ||b|| or
// iter = maxit) and otherwise forms rho = r.z and beta = -(z.q) / p.q (an
// r.z that is not a positive finite number stops the column).
template <int KC, typename TO>
__global__ void __launch_bounds__(kCT) k_cx(int n, int nb, int K, const double *__restrict__ Minv,
                                            const double *__restrict__ pnew, const double *__restrict__ q,
                                            double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
                                            TO *__restrict__ xo, double *partials, CCtl *ctl, int iter, int maxit,
                                            double tol) {
    int G = K / KC;
    Items it = items(G);
    int lane = threadIdx.x & 31;
    // the first block's inverse row (written at setup only) before the wait
    double m0[kB];
    if (it.wg < nb * G) block_row(Minv + (int64_t)(it.wg / G) * kB * kB, lane, m0);
    pdl_enter();
    pnew = after_wait(pnew);
    q = after_wait(q);
    x = after_wait(x);
    r = after_wait(r);
    z = after_wait(z);
    xo = after_wait(xo);
    if (!ctl->any) return;
    int c0 = it.g * KC;
    double alpha[KC];
    bool act[KC];
    bool live = false;
#pragma unroll
    for (int v = 0; v < KC; v++) {
        act[v] = ctl->active[c0 + v] != 0;
        alpha[v] = act[v] ? ctl->alpha[c0 + v] : 0.0;
        live |= act[v];
    }
    double acc[3][KC] = {};
    if (live) {
        for (int wi = it.wg; wi < nb * G; wi += it.nw) {
            int b = wi / G, i = b * kB + lane;
            int64_t o = (int64_t)i * K + c0;
            double pi[KC], qi[KC], xi[KC], ri[KC], zi[KC];
            ld_cols<KC>(pnew + o, pi);
            ld_cols<KC>(q + o, qi);
            ld_cols<KC>(x + o, xi);
            ld_cols<KC>(r + o, ri);
#pragma unroll
            for (int v = 0; v < KC; v++) {
                if (act[v]) {
                    xi[v] = fma(alpha[v], pi[v], xi[v]);
                    ri[v] = fma(-alpha[v], qi[v], ri[v]);
                }
            }
            if (wi == it.wg) block_apply_m<KC>(m0, ri, zi);
            else block_apply<KC>(Minv + (int64_t)b * kB * kB, ri, zi, lane);
            st_cols<KC>(x + o, xi);
            st_cols<KC>(r + o, ri);
            st_cols<KC>(z + o, zi);
            if (i < n)
#pragma unroll
                for (int v = 0; v < KC; v++)
                    if (act[v]) xo[o + v] = (TO)xi[v];
#pragma unroll
            for (int v = 0; v < KC; v++) {
                acc[0][v] += ri[v] * ri[v];
                acc[1][v] += ri[v] * zi[v];
                acc[2][v] += zi[v] * qi[v];
            }
        }
    }
    if (publish<KC, 3>(acc, it.g, it.wg < nb * G, K, partials, &ctl->counter[0])) {
        __shared__ double res[3 * 32];
        final_sums<3>(partials, K, res);
        if (threadIdx.x == 0) {
            int any = 0;
            for (int c = 0; c < K; c++) {
                if (ctl->active[c]) {
                    ctl->its[c] = iter;
                    double rn = sqrt(res[c]), rz = res[K + c], zq = res[2 * K + c];
                    if (rn <= tol * ctl->bn[c] || iter >= maxit || !(rz > 0.0) || !isfinite(rz)) {
                        ctl->active[c] = 0;
                    } else {
                        ctl->beta[c] = -zq / ctl->pq[c];
                        ctl->rho[c] = rz;
                    }
                }
                any |= ctl->active[c];
            }
            ctl->any = any;
            ctl->counter[0] = 0;
        }
    }
}

int grid_for_items(amg_hier *h, int items, int G) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms < 1) sms = 152;
    int want = (items + kCW - 1) / kCW;
    int cap = sms * 4;
    int g = want < cap ? want : cap;
    if (g < 1) g = 1;
    // the warp count must be a multiple of G (a warp's column group is fixed)
    while (((int64_t)g * kCW) % G) g++;
    return g;
}

#define WITH_COARSE_COLS(S, BODY)         \
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

template <int KC, typename TO>
int launch_ci(amg_hier *h, CoarseWS &W, const double *bL, TO *xL, const int *outer_done, const int *outer_live,
              cudaStream_t s) {
    Level &lc = h->lev.back();
    const CoarseIter &C = h->cit;
    int n = lc.A.n, nb = C.nb, K = W.K, g = W.grid;
    const bool pdl = h->pdl;
    PCG_CK(launch_k(pdl, k_cinit<KC, TO>, g, kCT, s, n, nb, K, bL, xL, W.x, W.r, W.z, (const double *)C.Minv,
                    W.partials, W.ctl, outer_done, outer_live));
    int maxit = h->prm.coarse_maxit;
    double tol = h->prm.coarse_tol;
    for (int it = 1; it <= maxit; it++) {
        double *pold = (it & 1) ? W.p1 : W.p0;
        double *pnew = (it & 1) ? W.p0 : W.p1;
        cudaError_t e = cudaSuccess;
        WITH_COARSE_COLS(lc.S, (e = launch_k(pdl, k_cq<KC, IDX>, W.grid_q, kCT, s, n, nb, K, (const int32_t *)lc.S.sptr,
                                             cols, (const double *)lc.S.v64, (const double *)W.z,
                                             (const double *)pold, pnew, W.q, W.partials, W.ctl)));
        PCG_CK(e);
        PCG_CK(launch_k(pdl, k_cx<KC, TO>, g, kCT, s, n, nb, K, (const double *)C.Minv, (const double *)pnew,
                        (const double *)W.q, W.x, W.r, W.z, xL, W.partials, W.ctl, it, maxit, tol));
    }
    return AMG_OK;
}

}  // namespace

// Factors of the iterative coarsest solve from the coarsest level's CSR
// (setup and refresh). Keeps the arrays' addresses when they exist.
int coarse_iter_build(amg_hier *h, cudaStream_t s) {
    Mem &M = h->mem;
    Level &lc = h->lev.back();
    int n = lc.A.n;
    CoarseIter &C = h->cit;
    int nb = (n + kB - 1) / kB;
    if (!C.F) {
        C.nb = nb;
        PCG_TRY(alloc(M, &C.F, (size_t)nb * kB * kB));
        PCG_TRY(alloc(M, &C.Minv, (size_t)nb * kB * kB));
        PCG_TRY(alloc(M, &C.zero, 1));
        PCG_CK(cudaMemsetAsync(C.zero, 0, sizeof(int), s));
    }
    int *dflag = nullptr;
    PCG_TRY(alloc(M, &dflag, 1));
    PCG_CK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
    k_ilu1<<<(nb + 63) / 64, 64, 0, s>>>(n, nb, lc.A.rp, lc.A.ci, lc.A.v, C.F, dflag);
    PCG_LAUNCH_CK();
    k_block_inverse<<<(nb * kB + 127) / 128, 128, 0, s>>>(n, nb, C.F, C.Minv);
    PCG_LAUNCH_CK();
    int flag = 0;
    PCG_CK(cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    PCG_CK(cudaStreamSynchronize(s));
    release(M, dflag);
    if (flag) {
        set_error("coarsest solver: an ILU(1) pivot of a block is not positive");
        return AMG_ERR_BREAKDOWN;
    }
    return AMG_OK;
}

int cws_alloc(amg_hier *h, Mem &M, CoarseWS &W, int K) {
    int nb = h->cit.nb;
    int64_t m = (int64_t)nb * kB * K;
    W.K = K;
    int KC = K == 1 ? 1 : 2;
    W.grid = grid_for_items(h, nb * (K / KC), K / KC);
    W.grid_q = grid_for_items(h, nb * 4 * (K / KC), K / KC);
    PCG_TRY(alloc(M, &W.x, m));
    PCG_TRY(alloc(M, &W.r, m));
    PCG_TRY(alloc(M, &W.z, m));
    PCG_TRY(alloc(M, &W.p0, m));
    PCG_TRY(alloc(M, &W.p1, m));
    PCG_TRY(alloc(M, &W.q, m));
    PCG_TRY(alloc(M, &W.partials, (size_t)3 * K * (W.grid > W.grid_q ? W.grid : W.grid_q)));
    PCG_TRY(alloc(M, &W.ctl, 1));
    if (M.dry) return AMG_OK;
    PCG_CK(cudaMemsetAsync(W.ctl, 0, sizeof(CCtl), M.stream));
    // p buffers are read (times beta = 0 on the first iteration) before they
    // are written: keep them finite
    PCG_CK(cudaMemsetAsync(W.p0, 0, sizeof(double) * m, M.stream));
    PCG_CK(cudaMemsetAsync(W.p1, 0, sizeof(double) * m, M.stream));
    return AMG_OK;
}

void cws_free(Mem &M, CoarseWS &W) {
    release(M, W.x);
    release(M, W.r);
    release(M, W.z);
    release(M, W.p0);
    release(M, W.p1);
    release(M, W.q);
    release(M, W.partials);
    release(M, W.ctl);
    W.K = 0;
    W.grid = 0;
    W.grid_q = 0;
}

// Kernels launched by one iterative coarsest solve.
int coarse_iter_launches(const amg_hier *h) { return 1 + 2 * h->prm.coarse_maxit; }

// x_L ~ A_L^{-1} b_L for the W.K columns of bL (n_L x K row-major, float64);
// xL receives the result in the V-cycle precision. outer_done: the outer
// solve's stop flag (every kernel returns at once when it is set);
// outer_live: K flags of columns still iterating outside (NULL: all).
template <typename TO>
int launch_coarse_iter(amg_hier *h, CoarseWS &W, const double *bL, TO *xL, const int *outer_done,
                       const int *outer_live, cudaStream_t s) {
    if (W.K == 1) return launch_ci<1, TO>(h, W, bL, xL, outer_done, outer_live, s);
    return launch_ci<2, TO>(h, W, bL, xL, outer_done, outer_live, s);
}

}  // namespace pcgamg

using namespace pcgamg;

extern "C" {

int amg_coarse_info(amg_handle h, int *kind, int *rows, int *blocks) {
    if (!h) {
        set_error("amg_coarse_info: NULL handle");
        return AMG_ERR_ARG;
    }
    if (kind) *kind = h->coarse_iter ? AMG_COARSE_ITER : AMG_COARSE_DENSE;
    if (rows) *rows = h->nL;
    if (blocks) *blocks = h->coarse_iter ? h->cit.nb : 0;
    return AMG_OK;
}

int amg_coarse_factors(amg_handle h, double *F) {
    if (!h || !F || !h->coarse_iter) {
        set_error("amg_coarse_factors: NULL argument, or the handle uses the dense coarsest solve");
        return AMG_ERR_ARG;
    }
    PCG_CK(cudaMemcpy(F, h->cit.F, sizeof(double) * (size_t)h->cit.nb * kCoarseBlock * kCoarseBlock,
                      cudaMemcpyDeviceToHost));
    return AMG_OK;
}

int amg_coarse_solve(amg_handle h, const double *b, double *x, int *iters, void *stream) {
    if (!h || !b || !x || !h->coarse_iter || h->invalid) {
        set_error("amg_coarse_solve: NULL argument, a handle with the dense coarsest solve, or an invalid handle");
        return AMG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int n = h->nL;
    Level &lc = h->lev.back();
    PCG_CK(cudaMemcpyAsync(h->bL, b, sizeof(double) * n, cudaMemcpyDefault, s));
    PCG_TRY(launch_coarse_iter<double>(h, h->cws, h->bL, lc.x64, h->cit.zero, nullptr, s));
    PCG_CK(cudaMemcpyAsync(x, lc.x64, sizeof(double) * n, cudaMemcpyDefault, s));
    int its = 0;
    PCG_CK(cudaMemcpyAsync(&its, &h->cws.ctl->its[0], sizeof(int), cudaMemcpyDeviceToHost, s));
    PCG_CK(cudaStreamSynchronize(s));
    if (iters) *iters = its;
    return AMG_OK;
}

}  // extern "C"

namespace pcgamg {

template int launch_coarse_iter<float>(amg_hier *, CoarseWS &, const double *, float *, const int *, const int *,
                                       cudaStream_t);
template int launch_coarse_iter<double>(amg_hier *, CoarseWS &, const double *, double *, const int *, const int *,
                                        cudaStream_t);

}  // namespace pcgamg
