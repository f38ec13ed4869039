// Device-side construction of the AMG hierarchy (arxiv 2210.16660, Sec. 3.1).
//
// Per level: n_pass pairwise passes of {edge weights of Eq. (weights) ->
// matching (Eq. approximatematch) -> pair/singleton aggregates and the
// tentative prolongator of Eq. (prolongator) -> Galerkin product P^T A P};
// the composed map and weight of the passes define the level's transfer.
// Then l1 diagonals, sliced-ELL copies in float64/float32, and the dense
// inverse of the coarsest matrix.
//
// Floating-point steps whose results decide integers (the edge weights that
// order the matching) and the values feeding them (Galerkin products,
// prolongator weights) use explicitly rounded operations (__dmul_rn etc.),
// never a fused multiply-add, in the order stated at each kernel, so the
// aggregates are reproducible bit for bit by any IEEE implementation that
// follows the same order.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>

#include "internal.cuh"

namespace pcgamg {

namespace {

inline int grid_for(int64_t n, int block = kBlock) {
    int64_t g = (n + block - 1) / block;
    return (int)(g > 0 ? g : 1);
}

// ------------------------------------------------------------ prefix sums
// Exclusive scan of n values into out[0..n], out[n] = total.
constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename Tin, typename T>
__global__ void k_scan_tiles(const Tin *__restrict__ in, T *__restrict__ out, T *__restrict__ tsum,
                             int64_t n) {
    __shared__ T sh[kScanThreads];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T loc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k;
        v[k] = i < n ? (T)in[i] : (T)0;
        loc += v[k];
    }
    sh[threadIdx.x] = loc;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        T a = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : (T)0;
        __syncthreads();
        sh[threadIdx.x] += a;
        __syncthreads();
    }
    T ex = sh[threadIdx.x] - loc;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
    if (threadIdx.x == kScanThreads - 1) tsum[blockIdx.x] = sh[kScanThreads - 1];
}

template <typename T>
__global__ void k_scan_tile_sums(T *tsum, int64_t nt, T *total) {
    __shared__ T sh[1024];
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c = 0; c < nt; c += 1024) {
        int64_t i = c + threadIdx.x;
        T v = i < nt ? tsum[i] : (T)0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            T a = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : (T)0;
            __syncthreads();
            sh[threadIdx.x] += a;
            __syncthreads();
        }
        if (i < nt) tsum[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += sh[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

template <typename T>
__global__ void k_scan_add(T *__restrict__ out, const T *__restrict__ tsum, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tsum[i / kScanTile];
}

// out must hold n + 1 values. *total_host receives out[n] (synchronises).
template <typename Tin, typename T>
int scan_exclusive(Mem &M, const Tin *in, T *out, int64_t n, T *total_host, cudaStream_t s) {
    int64_t nt = (n + kScanTile - 1) / kScanTile;
    if (nt < 1) nt = 1;
    T *tsum = nullptr;
    PCG_TRY(alloc(M, &tsum, (size_t)nt));
    k_scan_tiles<Tin, T><<<(unsigned)nt, kScanThreads, 0, s>>>(in, out, tsum, n);
    k_scan_tile_sums<T><<<1, 1024, 0, s>>>(tsum, nt, out + n);
    if (n > 0) k_scan_add<T><<<grid_for(n), kBlock, 0, s>>>(out, tsum, n);
    PCG_LAUNCH_CK();
    if (total_host) {
        PCG_CK(cudaMemcpyAsync(total_host, out + n, sizeof(T), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaStreamSynchronize(s));
    }
    release(M, tsum);
    return AMG_OK;
}

__global__ void k_narrow(const int64_t *__restrict__ in, int32_t *__restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)in[i];
}

// ------------------------------------------------------------ validation
// flag bits: 1 column out of range or unsorted, 2 diagonal missing or <= 0,
// 4 row pointer decreasing or wrong bounds, 8 not exactly symmetric.
__global__ void k_check_csr(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, int64_t nnz, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t s = rp[i], e = rp[i + 1];
    if (e < s || s < 0 || (int64_t)e > nnz || (i == 0 && s != 0) || (i == n - 1 && (int64_t)e != nnz)) {
        atomicOr(flag, 4);
        return;
    }
    int has = 0;
    for (int32_t k = s; k < e; k++) {
        int32_t j = ci[k];
        if (j < 0 || j >= n || (k > s && j <= ci[k - 1])) atomicOr(flag, 1);
        if (j == i) has = v[k] > 0.0 ? 1 : -1;
    }
    if (has != 1) atomicOr(flag, 2);
}

__global__ void k_check_sym(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
        int32_t j = ci[k];
        if (j <= i) continue;
        int32_t lo = rp[j], hi = rp[j + 1] - 1, hit = -1;
        while (lo <= hi) {
            int32_t mid = (lo + hi) >> 1;
            int32_t c = ci[mid];
            if (c == i) { hit = mid; break; }
            if (c < i) lo = mid + 1; else hi = mid - 1;
        }
        if (hit < 0 || __double_as_longlong(v[hit]) != __double_as_longlong(v[k])) {
            atomicOr(flag, 8);
            return;
        }
    }
}

// ------------------------------------------------------------ small fills
template <typename T>
__global__ void k_fill(T *a, int64_t n, T val) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = val;
}

__global__ void k_iota(int32_t *a, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}

__global__ void k_diag(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const double *__restrict__ v, double *__restrict__ dg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; k++)
        if (ci[k] == i) { d = v[k]; break; }
    dg[i] = d;
}

// ------------------------------------------------------------ matching
// Eq. (weights) for edge {a, b}, a < b, evaluated as
// 1 - ((2 a_ab) w_a) w_b / ((a_aa w_a) w_a + (a_bb w_b) w_b), every step rounded.
__device__ __forceinline__ double edge_weight(double aab, double aaa, double abb, double wa, double wb) {
    double num = __dmul_rn(__dmul_rn(__dmul_rn(2.0, aab), wa), wb);
    double den = __dadd_rn(__dmul_rn(__dmul_rn(aaa, wa), wa), __dmul_rn(__dmul_rn(abb, wb), wb));
    return __dsub_rn(1.0, __ddiv_rn(num, den));
}

// Strict total order on candidate edges: larger weight first, then smaller
// (min, max) endpoint pair.
__device__ __forceinline__ bool edge_before(double c1, int a1, int b1, double c2, int a2, int b2) {
    if (c1 != c2) return c1 > c2;
    if (a1 != a2) return a1 < a2;
    return b1 < b2;
}

// Candidate list of each row for one matching pass: the neighbours j with
// c_ij > 1, in the strict total order of edge_before (largest weight first,
// ties by the smaller (min, max) pair). Weights do not change while the pass
// runs, so they are formed once here (same rounding as the oracle's) and
// sorted in the row's own slots [rp[i], rp[i] + len[i]) by insertion.
__global__ void k_match_prep(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ v, const double *__restrict__ dg,
                             const double *__restrict__ w, int32_t *__restrict__ lst, double *__restrict__ lc,
                             int32_t *__restrict__ len, int32_t *__restrict__ ptr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t r0 = rp[i];
    int m = 0;
    for (int32_t k = r0; k < rp[i + 1]; k++) {
        int j = ci[k];
        if (j == i) continue;
        int a = min(i, j), b = max(i, j);
        double c = edge_weight(v[k], dg[a], dg[b], w[a], w[b]);
        if (!(c > 1.0)) continue;
        // insert (c, j) into the sorted prefix
        int t = m;
        while (t > 0) {
            int jp = lst[r0 + t - 1];
            double cp = lc[r0 + t - 1];
            if (!edge_before(c, a, b, cp, min(i, jp), max(i, jp))) break;
            lst[r0 + t] = jp;
            lc[r0 + t] = cp;
            t--;
        }
        lst[r0 + t] = j;
        lc[r0 + t] = c;
        m++;
    }
    len[i] = m;
    ptr[i] = 0;
}

// One round of the locally-dominant matching, part 1: every free vertex
// points at its best candidate that is still free (its list pointer moves
// past matched neighbours: vertices only ever become matched, so the first
// free entry of the sorted list is the best free candidate). any is set when
// some vertex points somewhere.
__global__ void k_match_round(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ lst,
                              const int32_t *__restrict__ len, int32_t *__restrict__ ptr,
                              const int32_t *__restrict__ mate, int32_t *__restrict__ cand, int *any) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (mate[i] >= 0) { cand[i] = -1; return; }
    int32_t r0 = rp[i];
    int p = ptr[i], e = len[i];
    while (p < e && mate[lst[r0 + p]] >= 0) p++;
    ptr[i] = p;
    int j = p < e ? lst[r0 + p] : -1;
    cand[i] = j;
    if (j >= 0) *any = 1;
}

// Part 2: mutual pointers are locally dominant edges; take them.
__global__ void k_match_commit(int n, const int32_t *__restrict__ cand, int32_t *__restrict__ mate) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (mate[i] >= 0) return;
    int j = cand[i];
    if (j >= 0 && cand[j] == i) mate[i] = j;
}

// ------------------------------------------------------------ aggregates
// lead[i] = 1 when i opens an aggregate: a singleton that has a nonzero
// off-diagonal entry, or the smaller end of a matched pair. Unmatched rows
// without nonzero couplings are left out of the coarse space.
__global__ void k_leaders(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ v, const int32_t *__restrict__ mate,
                          int32_t *__restrict__ lead) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int m = mate[i];
    if (m >= 0) { lead[i] = i < m ? 1 : 0; return; }
    int iso = 1;
    for (int32_t k = rp[i]; k < rp[i + 1]; k++)
        if (ci[k] != i && v[k] != 0.0) { iso = 0; break; }
    lead[i] = iso ? 0 : 1;
}

// Eq. (prolongator): pair weights w_e = (w_i, w_j) / ||(w_i, w_j)||, singleton
// weight w_s / |w_s|; coarse w_c = ||w restricted to the aggregate||.
__global__ void k_assign(int n, const int32_t *__restrict__ mate, const int32_t *__restrict__ lead,
                         const int32_t *__restrict__ idx, const double *__restrict__ w,
                         int32_t *__restrict__ agg, double *__restrict__ p, double *__restrict__ wc,
                         int32_t *__restrict__ mem0, int32_t *__restrict__ mem1) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = mate[i];
    if (!lead[i]) {
        if (j < 0) { agg[i] = -1; p[i] = 0.0; }
        return;
    }
    int I = idx[i];
    double wi = w[i];
    if (j >= 0) {
        double wj = w[j];
        double nrm = __dsqrt_rn(__dadd_rn(__dmul_rn(wi, wi), __dmul_rn(wj, wj)));
        agg[i] = I; agg[j] = I;
        p[i] = __ddiv_rn(wi, nrm);
        p[j] = __ddiv_rn(wj, nrm);
        wc[I] = nrm;
        mem0[I] = i; mem1[I] = j;
    } else {
        double a = fabs(wi);
        agg[i] = I;
        p[i] = __ddiv_rn(wi, a);
        wc[I] = a;
        mem0[I] = i; mem1[I] = -1;
    }
}

// ------------------------------------------------------------ Galerkin product
__global__ void k_rap_count(int nc, const int32_t *__restrict__ mem0, const int32_t *__restrict__ mem1,
                            const int32_t *__restrict__ rp, int32_t *__restrict__ cnt) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int i0 = mem0[I], i1 = mem1[I];
    int c = rp[i0 + 1] - rp[i0];
    if (i1 >= 0) c += rp[i1 + 1] - rp[i1];
    cnt[I] = c;
}

// Coarse row I of P^T A P for a pairwise aggregation: every stored a_ij with
// i in G_I and agg(j) >= 0 contributes t = a_ij * (p_i * p_j) to entry
// (I, agg(j)); contributions to one entry are added in increasing order of
// (min(i,j), max(i,j)). Terms are kept sorted by (J, min, max) in the row's
// scratch segment (insertion sort, stable), then runs are summed in place.
__global__ void k_rap_terms(int nc, const int32_t *__restrict__ mem0, const int32_t *__restrict__ mem1,
                            const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, const int32_t *__restrict__ agg,
                            const double *__restrict__ p, const int32_t *__restrict__ off,
                            int32_t *__restrict__ tJ, unsigned long long *__restrict__ tK,
                            double *__restrict__ tT, int32_t *__restrict__ ucnt) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int32_t base = off[I];
    int m = 0;
    int mem[2] = {mem0[I], mem1[I]};
    for (int q = 0; q < 2; q++) {
        int i = mem[q];
        if (i < 0) break;
        double pi = p[i];
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            int j = ci[k];
            int J = agg[j];
            if (J < 0) continue;
            unsigned long long key = ((unsigned long long)(unsigned)min(i, j) << 32) |
                                     (unsigned long long)(unsigned)max(i, j);
            double t = __dmul_rn(v[k], __dmul_rn(pi, p[j]));
            int32_t pos = base + m;
            while (pos > base && (tJ[pos - 1] > J || (tJ[pos - 1] == J && tK[pos - 1] > key))) {
                tJ[pos] = tJ[pos - 1];
                tK[pos] = tK[pos - 1];
                tT[pos] = tT[pos - 1];
                pos--;
            }
            tJ[pos] = J; tK[pos] = key; tT[pos] = t;
            m++;
        }
    }
    int u = 0;
    for (int q = 0; q < m; q++) {
        int32_t J = tJ[base + q];
        double t = tT[base + q];
        if (u == 0 || J != tJ[base + u - 1]) {
            tJ[base + u] = J;
            tT[base + u] = t;
            u++;
        } else {
            tT[base + u - 1] = __dadd_rn(tT[base + u - 1], t);
        }
    }
    ucnt[I] = u;
}

__global__ void k_rap_copy(int nc, const int32_t *__restrict__ off, const int32_t *__restrict__ rpc,
                           const int32_t *__restrict__ tJ, const double *__restrict__ tT,
                           int32_t *__restrict__ cic, double *__restrict__ vc) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int32_t o = off[I], s = rpc[I], e = rpc[I + 1];
    for (int32_t q = 0; q < e - s; q++) {
        cic[s + q] = tJ[o + q];
        vc[s + q] = tT[o + q];
    }
}

// Product of the pass maps and weights, in pass order.
__global__ void k_compose(int n, int32_t *__restrict__ cagg, double *__restrict__ cp,
                          const int32_t *__restrict__ agg, const double *__restrict__ p) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = cagg[i];
    double c = cp[i];
    if (a >= 0) {
        c = __dmul_rn(c, p[a]);
        a = agg[a];
    }
    if (a < 0) c = 0.0;
    cagg[i] = a;
    cp[i] = c;
}

// ------------------------------------------------------------ level data
// l1 smoother diagonal d_i = sum_j |a_ij| (row order), stored inverted.
__global__ void k_l1diag(int n, const int32_t *__restrict__ rp, const double *__restrict__ v,
                         double *__restrict__ dinv, float *__restrict__ dinv32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; k++) s = __dadd_rn(s, fabs(v[k]));
    double d = __ddiv_rn(1.0, s);
    dinv[i] = d;
    dinv32[i] = __double2float_rn(d);
}

// l1 diagonal of the hybrid Gauss-Seidel smoother, blocks of nb rows:
// d_i = a_ii + sum of |a_ij| over j outside i's block (row order; in-block
// off-diagonal entries skipped), stored inverted. nb = 1 is k_l1diag.
__global__ void k_hybrid_l1(int n, int nb, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, double *__restrict__ dinv, float *__restrict__ dinv32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = (i / nb) * nb, hi = lo + nb;
    double s = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
        int j = ci[k];
        if (j == i || j < lo || j >= hi) s = __dadd_rn(s, fabs(v[k]));
    }
    double d = __ddiv_rn(1.0, s);
    dinv[i] = d;
    dinv32[i] = __double2float_rn(d);
}

// In-block entries a pass has already updated when it reaches row i (LOWER:
// j in [lo, i), the forward pass; else j in (i, hi), the backward pass):
// count, then fill a width-w table in storage order (column -1, value 0 pad).
template <bool LOWER>
__global__ void k_part_count(int n, int nb, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             int32_t *__restrict__ cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = (i / nb) * nb, hi = min(n, lo + nb);
    int c = 0;
    for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
        int j = ci[k];
        if (LOWER ? (j >= lo && j < i) : (j > i && j < hi)) c++;
    }
    cnt[i] = c;
}

template <bool LOWER>
__global__ void k_part_fill(int n, int nb, int w, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, int32_t *__restrict__ pci, double *__restrict__ pv64,
                            float *__restrict__ pv32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = (i / nb) * nb, hi = min(n, lo + nb);
    int64_t base = (int64_t)i * w;
    int c = 0;
    for (int32_t k = rp[i]; k < rp[i + 1] && c < w; k++) {
        int j = ci[k];
        if (LOWER ? (j >= lo && j < i) : (j > i && j < hi)) {
            pci[base + c] = j;
            pv64[base + c] = v[k];
            pv32[base + c] = __double2float_rn(v[k]);
            c++;
        }
    }
    for (; c < w; c++) {
        pci[base + c] = -1;
        pv64[base + c] = 0.0;
        pv32[base + c] = 0.0f;
    }
}

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __double2float_rn(a[i]);
}

__global__ void k_sell_width(int n, int nsl, const int32_t *__restrict__ rp, int32_t *__restrict__ sw) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsl) return;
    int r0 = s * kSlice, r1 = min(r0 + kSlice, n);
    int mx = 0;
    for (int r = r0; r < r1; r++) mx = max(mx, rp[r + 1] - rp[r]);
    sw[s] = mx * kSlice;
}

__global__ void k_sell_fill(int n, int nsl, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, const int32_t *__restrict__ sptr,
                            int32_t *__restrict__ col, double *__restrict__ v64, float *__restrict__ v32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsl * kSlice) return;
    int s = i / kSlice, lane = i % kSlice;
    int32_t base = sptr[s];
    int w = (sptr[s + 1] - base) / kSlice;
    int len = i < n ? rp[i + 1] - rp[i] : 0;
    int32_t r0 = i < n ? rp[i] : 0;
    int pad = i < n ? i : 0;
    for (int k = 0; k < w; k++) {
        int32_t e = base + k * kSlice + lane;
        if (k < len) {
            double a = v[r0 + k];
            col[e] = ci[r0 + k];
            v64[e] = a;
            v32[e] = __double2float_rn(a);
        } else {
            col[e] = pad;
            v64[e] = 0.0;
            v32[e] = 0.0f;
        }
    }
}

// flag = 1 when some stored |col - row| does not fit in int16.
__global__ void k_col16_check(int n, int nsl, const int32_t *__restrict__ sptr, const int32_t *__restrict__ col,
                              int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsl * kSlice) return;
    int s = i / kSlice, lane = i % kSlice;
    int row = i < n ? i : 0;
    int32_t base = sptr[s];
    int w = (sptr[s + 1] - base) / kSlice;
    for (int k = 0; k < w; k++) {
        int d = col[base + k * kSlice + lane] - row;
        if (d < -32768 || d > 32767) { atomicOr(flag, 1); return; }
    }
}

__global__ void k_col16_fill(int n, int nsl, const int32_t *__restrict__ sptr, const int32_t *__restrict__ col,
                             int16_t *__restrict__ col16) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsl * kSlice) return;
    int s = i / kSlice, lane = i % kSlice;
    int row = i < n ? i : 0;
    int32_t base = sptr[s];
    int w = (sptr[s + 1] - base) / kSlice;
    for (int k = 0; k < w; k++) {
        int32_t e = base + k * kSlice + lane;
        col16[e] = (int16_t)(col[e] - row);
    }
}

__global__ void k_count_members(int n, const int32_t *__restrict__ agg, int32_t *__restrict__ cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (agg[i] >= 0) atomicAdd(&cnt[agg[i]], 1);
}

__global__ void k_fill_members(int n, const int32_t *__restrict__ agg, const int32_t *__restrict__ rptr,
                               int32_t *__restrict__ cur, int32_t *__restrict__ ridx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = agg[i];
    if (a < 0) return;
    int pos = atomicAdd(&cur[a], 1);
    ridx[rptr[a] + pos] = i;
}

__global__ void k_sort_members(int nc, const int32_t *__restrict__ rptr, int32_t *__restrict__ ridx) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int32_t s = rptr[I], e = rptr[I + 1];
    for (int32_t a = s + 1; a < e; a++) {
        int32_t x = ridx[a];
        int32_t b = a;
        while (b > s && ridx[b - 1] > x) { ridx[b] = ridx[b - 1]; b--; }
        ridx[b] = x;
    }
}

// ------------------------------------------------------------ coarsest level
__global__ void k_dense(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                        const double *__restrict__ v, double *__restrict__ ad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t k = rp[i]; k < rp[i + 1]; k++) ad[(int64_t)i * n + ci[k]] = v[k];
}

// In-place Cholesky (lower triangle, row-major) by one block; flag = 1 when
// a pivot is not positive.
__global__ void k_chol(int n, double *a, int *flag) {
    __shared__ double red[1024];
    __shared__ double piv;
    for (int j = 0; j < n; j++) {
        double s = 0.0;
        for (int k = threadIdx.x; k < j; k += blockDim.x) s += a[(int64_t)j * n + k] * a[(int64_t)j * n + k];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < (unsigned)o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double d = a[(int64_t)j * n + j] - red[0];
            if (!(d > 0.0)) { *flag = 1; d = 1.0; }
            piv = sqrt(d);
            a[(int64_t)j * n + j] = piv;
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double t = a[(int64_t)i * n + j];
            for (int k = 0; k < j; k++) t -= a[(int64_t)i * n + k] * a[(int64_t)j * n + k];
            a[(int64_t)i * n + j] = t / piv;
        }
        __syncthreads();
    }
}

// Column c of A^{-1} = L^{-T} L^{-1} e_c by one block per column.
__global__ void k_chol_inverse(int n, const double *__restrict__ L, double *__restrict__ ainv) {
    extern __shared__ double y[];
    int c = blockIdx.x;
    for (int k = threadIdx.x; k < n; k += blockDim.x) y[k] = k == c ? 1.0 : 0.0;
    __syncthreads();
    for (int i = 0; i < n; i++) {           // L y = e_c
        double yi = y[i] / L[(int64_t)i * n + i];
        __syncthreads();
        if (threadIdx.x == 0) y[i] = yi;
        for (int k = i + 1 + threadIdx.x; k < n; k += blockDim.x) y[k] -= L[(int64_t)k * n + i] * yi;
        __syncthreads();
    }
    for (int i = n - 1; i >= 0; i--) {      // L^T x = y
        double xi = y[i] / L[(int64_t)i * n + i];
        __syncthreads();
        if (threadIdx.x == 0) y[i] = xi;
        for (int k = threadIdx.x; k < i; k += blockDim.x) y[k] -= L[(int64_t)i * n + k] * xi;
        __syncthreads();
    }
    for (int k = threadIdx.x; k < n; k += blockDim.x) ainv[(int64_t)k * n + c] = y[k];
}

// ------------------------------------------------------------ partial reuse
// flag 16 where (rp, ci) differs from the pattern the hierarchy was built on.
__global__ void k_same_pattern(int n, int64_t nnz, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const int32_t *__restrict__ rp0, const int32_t *__restrict__ ci0, int *flag) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= n && rp[k] != rp0[k]) atomicOr(flag, 16);
    if (k < nnz && ci[k] != ci0[k]) atomicOr(flag, 16);
}

// Members of each aggregate of one kept pass map: smallest in first, largest
// in second (equal for a singleton; a pass aggregate has one or two members).
__global__ void k_pass_members(int m, const int32_t *__restrict__ agg, int32_t *__restrict__ first,
                               int32_t *__restrict__ second) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int I = agg[i];
    if (I < 0) return;
    atomicMin(first + I, i);
    atomicMax(second + I, i);
}

// Eq. (prolongator) weights of a kept pass from its map and w, with the
// arithmetic of k_assign: pair w_e / ||w_e||, singleton w_s / |w_s|, 0 for a
// row left out; the coarse w_c; members as mem0 < mem1 (-1 for a singleton).
__global__ void k_pass_weights(int m, int nc, const int32_t *__restrict__ first, const int32_t *__restrict__ second,
                               const double *__restrict__ w, double *__restrict__ p, double *__restrict__ wc,
                               int32_t *__restrict__ mem0, int32_t *__restrict__ mem1, int *flag) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int i = first[I], j = second[I];
    if (i < 0 || i >= m || j < 0 || j >= m) {  // an aggregate without members: not a kept map
        atomicOr(flag, 1);
        return;
    }
    double wi = w[i];
    if (j != i) {
        double wj = w[j];
        double nrm = __dsqrt_rn(__dadd_rn(__dmul_rn(wi, wi), __dmul_rn(wj, wj)));
        p[i] = __ddiv_rn(wi, nrm);
        p[j] = __ddiv_rn(wj, nrm);
        wc[I] = nrm;
        mem0[I] = i;
        mem1[I] = j;
    } else {
        double a = fabs(wi);
        p[i] = __ddiv_rn(wi, a);
        wc[I] = a;
        mem0[I] = i;
        mem1[I] = -1;
    }
}

// Values only of the sliced-ELL copies (the layout and columns are those of
// the same pattern, already in place). A slice with a shared offset pattern
// (upat) takes row i's value for offset o_k from its CSR entry of column
// i + o_k, or 0 where the row has none.
__global__ void k_sell_vals(int n, int nsl, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, const int32_t *__restrict__ sptr,
                            const int32_t *__restrict__ upat, double *__restrict__ v64, float *__restrict__ v32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsl * kSlice) return;
    int s = i / kSlice, lane = i % kSlice;
    int32_t base = sptr[s];
    int w = (sptr[s + 1] - base) / kSlice;
    int len = i < n ? rp[i + 1] - rp[i] : 0;
    int32_t r0 = i < n ? rp[i] : 0;
    const bool uni = upat && upat[base / kSlice] != kNoPattern<int32_t>;
    int q = 0;
    for (int k = 0; k < w; k++) {
        int32_t e = base + k * kSlice + lane;
        double a = 0.0;
        if (uni) {
            if (q < len && ci[r0 + q] - i == upat[base / kSlice + k]) a = v[r0 + q++];
        } else if (k < len) {
            a = v[r0 + k];
        }
        v64[e] = a;
        v32[e] = __double2float_rn(a);
    }
}

// 16-bit copy of the offset patterns (beside 16-bit column offsets).
__global__ void k_pattern16(const int32_t *__restrict__ up, int16_t *__restrict__ up16, int64_t m) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < m) up16[q] = up[q] == kNoPattern<int32_t> ? kNoPattern<int16_t> : (int16_t)up[q];
}

// Shared offset patterns of level 0, one warp per slice. The candidate is
// the offsets j - i of the slice's longest row (the lowest lane among those
// of the slice's width); the slice takes it when every row's offsets are a
// subset of it and every i + o_k is a row index. It is then rewritten in
// pattern order: entry k of row i gets column i + o_k and the row's value
// there, or 0 where the row has no entry of that offset (a row's entries
// keep their increasing column order, the zeros fall between them), and
// upat receives the pattern; otherwise upat marks the slice kNoPattern.
__global__ void k_sell_uniform(int n, int nsl, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const double *__restrict__ v, const int32_t *__restrict__ sptr,
                               int32_t *__restrict__ col, int16_t *__restrict__ col16, double *__restrict__ v64,
                               float *__restrict__ v32, int32_t *__restrict__ upat, unsigned long long *count) {
    const int lane = threadIdx.x & 31;
    const int s = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (s >= nsl) return;  // the whole warp leaves together
    const int32_t base = sptr[s];
    const int w = (sptr[s + 1] - base) / kSlice;
    const int i = s * kSlice + lane;
    const bool real = i < n;
    const int32_t r0 = real ? rp[i] : 0;
    const int len = real ? rp[i + 1] - r0 : 0;
    const unsigned longest = __ballot_sync(0xffffffffu, real && len == w);
    const int isrc = s * kSlice + __ffs(longest) - 1;
    const int32_t rs = rp[isrc];
    bool ok = true;
    if (real) {
        int q = 0;
        for (int k = 0; k < w; k++) {
            const int o = ci[rs + k] - isrc;
            const int64_t j = (int64_t)i + o;
            if (j < 0 || j >= n) ok = false;
            if (q < len && ci[r0 + q] - i == o) q++;
        }
        if (q != len) ok = false;
    }
    if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) upat[base / kSlice] = kNoPattern<int32_t>;
        return;
    }
    int q = 0;
    for (int k = 0; k < w; k++) {
        const int o = ci[rs + k] - isrc;
        if (lane == 0) upat[base / kSlice + k] = o;
        if (!real) continue;  // lanes past the last row are never swept
        const int32_t e = base + k * kSlice + lane;
        double a = 0.0;
        if (q < len && ci[r0 + q] - i == o) a = v[r0 + q++];
        col[e] = i + o;
        if (col16) col16[e] = (int16_t)o;
        v64[e] = a;
        v32[e] = __double2float_rn(a);
    }
    if (lane == 0) atomicAdd(count, 1ull);
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr int kMatchBatch = 8;      // matching rounds launched per host check
constexpr int kMatchRounds = 20000; // rounds allowed per pass

int read_flag(int *dflag, cudaStream_t s, int *out) {
    PCG_CK(cudaMemcpyAsync(out, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    PCG_CK(cudaStreamSynchronize(s));
    return AMG_OK;
}

void free_csr(Mem &M, DevCSR &a) {
    release(M, a.rp);
    release(M, a.ci);
    release(M, a.v);
}

// Galerkin product P^T cur P of one pairwise pass (aggregate members mem0 <
// mem1, -1 = singleton; map agg; weights p) into a new CSR matrix c.
int galerkin(amg_hier *h, const DevCSR &cur, const int32_t *agg, const double *p, const int32_t *mem0,
             const int32_t *mem1, int nc, DevCSR *out, cudaStream_t s) {
    Mem &M = h->mem;
    int32_t *cnt = nullptr, *off = nullptr, *ucnt = nullptr, *tJ = nullptr;
    unsigned long long *tK = nullptr;
    double *tT = nullptr;
    PCG_TRY(alloc(M, &cnt, nc));
    PCG_TRY(alloc(M, &off, (size_t)nc + 1));
    k_rap_count<<<grid_for(nc), kBlock, 0, s>>>(nc, mem0, mem1, cur.rp, cnt);
    PCG_LAUNCH_CK();
    int32_t nterm = 0;
    PCG_TRY(scan_exclusive(M, cnt, off, nc, &nterm, s));
    release(M, cnt);
    PCG_TRY(alloc(M, &tJ, nterm));
    PCG_TRY(alloc(M, &tK, nterm));
    PCG_TRY(alloc(M, &tT, nterm));
    PCG_TRY(alloc(M, &ucnt, nc));
    k_rap_terms<<<grid_for(nc, 128), 128, 0, s>>>(nc, mem0, mem1, cur.rp, cur.ci, cur.v, agg, p, off, tJ,
                                                   tK, tT, ucnt);
    PCG_LAUNCH_CK();
    DevCSR c;
    c.n = nc;
    PCG_TRY(alloc(M, &c.rp, (size_t)nc + 1));
    int32_t nzc = 0;
    PCG_TRY(scan_exclusive(M, ucnt, c.rp, nc, &nzc, s));
    c.nnz = nzc;
    PCG_TRY(alloc(M, &c.ci, nzc));
    PCG_TRY(alloc(M, &c.v, nzc));
    k_rap_copy<<<grid_for(nc), kBlock, 0, s>>>(nc, off, c.rp, tJ, tT, c.ci, c.v);
    PCG_LAUNCH_CK();
    PCG_CK(cudaStreamSynchronize(s));
    release(M, tJ);
    release(M, tK);
    release(M, tT);
    release(M, ucnt);
    release(M, off);
    *out = c;
    return AMG_OK;
}

// One pairwise pass on cur (weights w): fills agg/p of the pass, the coarse
// matrix nxt and its w. Returns AMG_OK or an error.
int pairwise_pass(amg_hier *h, const DevCSR &cur, const double *w, int32_t **agg_out, double **p_out,
                  DevCSR *nxt, double **wc_out, double *t_match, double *t_rap, cudaStream_t s) {
    Mem &M = h->mem;
    int m = cur.n;
    double *dg = nullptr, *p = nullptr, *wc = nullptr;
    int32_t *mate = nullptr, *cand = nullptr, *lead = nullptr, *idx = nullptr, *agg = nullptr;
    int32_t *mem0 = nullptr, *mem1 = nullptr;
    int *dflag = nullptr;
    int32_t *lst = nullptr, *len = nullptr, *ptr = nullptr;
    double *lc = nullptr;
    PCG_TRY(alloc(M, &dg, m));
    PCG_TRY(alloc(M, &mate, m));
    PCG_TRY(alloc(M, &cand, m));
    PCG_TRY(alloc(M, &lst, cur.nnz));
    PCG_TRY(alloc(M, &lc, cur.nnz));
    PCG_TRY(alloc(M, &len, m));
    PCG_TRY(alloc(M, &ptr, m));
    PCG_TRY(alloc(M, &dflag, kMatchBatch));
    double t0 = now_ms();
    k_diag<<<grid_for(m), kBlock, 0, s>>>(m, cur.rp, cur.ci, cur.v, dg);
    k_fill<int32_t><<<grid_for(m), kBlock, 0, s>>>(mate, m, -1);
    k_match_prep<<<grid_for(m, 128), 128, 0, s>>>(m, cur.rp, cur.ci, cur.v, dg, w, lst, lc, len, ptr);
    PCG_LAUNCH_CK();
    release(M, lc);
    // rounds in batches of kMatchBatch, one host check per batch: a round
    // after the last productive one finds no candidate and changes nothing
    int rounds = 0;
    for (;;) {
        PCG_CK(cudaMemsetAsync(dflag, 0, sizeof(int) * kMatchBatch, s));
        for (int r = 0; r < kMatchBatch; r++) {
            k_match_round<<<grid_for(m), kBlock, 0, s>>>(m, cur.rp, lst, len, ptr, mate, cand, dflag + r);
            k_match_commit<<<grid_for(m), kBlock, 0, s>>>(m, cand, mate);
        }
        PCG_LAUNCH_CK();
        int any[kMatchBatch];
        PCG_CK(cudaMemcpyAsync(any, dflag, sizeof(int) * kMatchBatch, cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaStreamSynchronize(s));
        rounds += kMatchBatch;
        if (!any[kMatchBatch - 1]) break;
        if (rounds >= kMatchRounds) {
            set_error("amg_setup: the matching did not finish in %d rounds", kMatchRounds);
            return AMG_ERR_MATCH;
        }
    }
    release(M, lst);
    release(M, len);
    release(M, ptr);
    release(M, cand);
    release(M, dg);
    *t_match += now_ms() - t0;
    t0 = now_ms();
    PCG_TRY(alloc(M, &lead, m));
    PCG_TRY(alloc(M, &idx, (size_t)m + 1));
    k_leaders<<<grid_for(m), kBlock, 0, s>>>(m, cur.rp, cur.ci, cur.v, mate, lead);
    PCG_LAUNCH_CK();
    int32_t nc = 0;
    PCG_TRY(scan_exclusive(M, lead, idx, m, &nc, s));
    PCG_TRY(alloc(M, &agg, m));
    PCG_TRY(alloc(M, &p, m));
    PCG_TRY(alloc(M, &wc, nc));
    PCG_TRY(alloc(M, &mem0, nc));
    PCG_TRY(alloc(M, &mem1, nc));
    k_assign<<<grid_for(m), kBlock, 0, s>>>(m, mate, lead, idx, w, agg, p, wc, mem0, mem1);
    PCG_LAUNCH_CK();
    release(M, lead);
    release(M, idx);
    release(M, mate);

    DevCSR c;
    PCG_TRY(galerkin(h, cur, agg, p, mem0, mem1, nc, &c, s));
    release(M, mem0);
    release(M, mem1);
    release(M, dflag);
    *t_rap += now_ms() - t0;
    *agg_out = agg;
    *p_out = p;
    *nxt = c;
    *wc_out = wc;
    return AMG_OK;
}

int finish_level(amg_hier *h, Level &lv, bool coarsest, cudaStream_t s) {
    Mem &M = h->mem;
    int n = lv.A.n;
    PCG_TRY(alloc(M, &lv.dinv, n));
    PCG_TRY(alloc(M, &lv.dinv32, n));
    k_l1diag<<<grid_for(n), kBlock, 0, s>>>(n, lv.A.rp, lv.A.v, lv.dinv, lv.dinv32);
    PCG_LAUNCH_CK();
    // sliced ELL
    Sell &S = lv.S;
    S.n = n;
    S.nslices = (n + kSlice - 1) / kSlice;
    int32_t *sw = nullptr;
    PCG_TRY(alloc(M, &sw, S.nslices));
    PCG_TRY(alloc(M, &S.sptr, (size_t)S.nslices + 1));
    k_sell_width<<<grid_for(S.nslices), kBlock, 0, s>>>(n, S.nslices, lv.A.rp, sw);
    PCG_LAUNCH_CK();
    // slice offsets are int32: scan in int64 and refuse a level whose padded
    // entries do not fit, instead of letting the offsets wrap
    int64_t *sp64 = nullptr;
    PCG_TRY(alloc(M, &sp64, (size_t)S.nslices + 1));
    int64_t tot64 = 0;
    PCG_TRY(scan_exclusive(M, sw, sp64, S.nslices, &tot64, s));
    release(M, sw);
    if (tot64 > (int64_t)INT32_MAX) {
        release(M, sp64);
        set_error("amg_setup: level with %d rows needs %lld sliced-ELL entries (int32 offsets allow %d)", n,
                  (long long)tot64, INT32_MAX);
        return AMG_ERR_ARG;
    }
    k_narrow<<<grid_for((int64_t)S.nslices + 1), kBlock, 0, s>>>(sp64, S.sptr, (int64_t)S.nslices + 1);
    PCG_LAUNCH_CK();
    release(M, sp64);
    int32_t tot = (int32_t)tot64;
    S.nnz_pad = tot;
    PCG_TRY(alloc(M, &S.col, tot));
    PCG_TRY(alloc(M, &S.v64, tot));
    PCG_TRY(alloc(M, &S.v32, tot));
    k_sell_fill<<<grid_for((int64_t)S.nslices * kSlice), kBlock, 0, s>>>(n, S.nslices, lv.A.rp, lv.A.ci,
                                                                         lv.A.v, S.sptr, S.col, S.v64, S.v32);
    PCG_LAUNCH_CK();
    // 16-bit column offsets where they fit (2 bytes per entry instead of 4)
    {
        int *dflag = nullptr;
        PCG_TRY(alloc(M, &dflag, 1));
        PCG_CK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
        k_col16_check<<<grid_for((int64_t)S.nslices * kSlice), kBlock, 0, s>>>(n, S.nslices, S.sptr, S.col, dflag);
        PCG_LAUNCH_CK();
        int wide = 0;
        PCG_TRY(read_flag(dflag, s, &wide));
        release(M, dflag);
        if (!wide && !h->no_col16) {
            PCG_TRY(alloc(M, &S.col16, tot));
            k_col16_fill<<<grid_for((int64_t)S.nslices * kSlice), kBlock, 0, s>>>(n, S.nslices, S.sptr, S.col,
                                                                                  S.col16);
            PCG_LAUNCH_CK();
        }
    }
    // shared offset patterns (every level: level 0 of a structured mesh
    // takes them almost everywhere, level 1 mostly)
    if (!h->no_uniform) {
        PCG_TRY(alloc(M, &S.upat, (size_t)tot / kSlice));
        unsigned long long *dcount = nullptr;
        PCG_TRY(alloc(M, &dcount, 1));
        PCG_CK(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), s));
        k_sell_uniform<<<grid_for((int64_t)S.nslices * kSlice), kBlock, 0, s>>>(
            n, S.nslices, lv.A.rp, lv.A.ci, lv.A.v, S.sptr, S.col, S.col16, S.v64, S.v32, S.upat, dcount);
        PCG_LAUNCH_CK();
        unsigned long long cnt = 0;
        PCG_CK(cudaMemcpyAsync(&cnt, dcount, sizeof(cnt), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaStreamSynchronize(s));
        release(M, dcount);
        S.uniform_slices = (int64_t)cnt;
        if (cnt == 0) {
            release(M, S.upat);
            S.upat = nullptr;
        } else {
            // entries of the uniform slices: sum of their widths x 32
            std::vector<int32_t> sp((size_t)S.nslices + 1), up((size_t)tot / kSlice);
            PCG_CK(cudaMemcpy(sp.data(), S.sptr, sizeof(int32_t) * sp.size(), cudaMemcpyDeviceToHost));
            PCG_CK(cudaMemcpy(up.data(), S.upat, sizeof(int32_t) * up.size(), cudaMemcpyDeviceToHost));
            int64_t e = 0;
            for (int q = 0; q < S.nslices; q++)
                if (up[sp[q] / kSlice] != kNoPattern<int32_t>) e += sp[q + 1] - sp[q];
            S.uniform_entries = e;
            if (S.col16) {
                PCG_TRY(alloc(M, &S.upat16, (size_t)tot / kSlice));
                k_pattern16<<<grid_for((int64_t)tot / kSlice), kBlock, 0, s>>>(S.upat, S.upat16,
                                                                               (int64_t)tot / kSlice);
                PCG_LAUNCH_CK();
            }
        }
    }
    // work vectors
    PCG_TRY(alloc(M, &lv.b64, n));
    PCG_TRY(alloc(M, &lv.x64, n));
    PCG_TRY(alloc(M, &lv.t64, n));
    PCG_TRY(alloc(M, &lv.xpre64, n));
    PCG_TRY(alloc(M, &lv.xp64, n));
    PCG_TRY(alloc(M, &lv.b32, n));
    PCG_TRY(alloc(M, &lv.x32, n));
    PCG_TRY(alloc(M, &lv.t32, n));
    PCG_TRY(alloc(M, &lv.xpre32, n));
    PCG_TRY(alloc(M, &lv.xp32, n));
    if (!coarsest) {
        PCG_TRY(alloc(M, &lv.p32, n));
        k_to_f32<<<grid_for(n), kBlock, 0, s>>>(lv.p, lv.p32, n);
        if (h->smoothed) {
            PCG_TRY(alloc(M, &lv.ones64, n));
            PCG_TRY(alloc(M, &lv.ones32, n));
            k_fill<double><<<grid_for(n), kBlock, 0, s>>>(lv.ones64, n, 1.0);
            k_fill<float><<<grid_for(n), kBlock, 0, s>>>(lv.ones32, n, 1.0f);
        }
        // members of each coarse row, increasing fine index
        int32_t *cnt = nullptr, *cur = nullptr;
        PCG_TRY(alloc(M, &cnt, lv.nc));
        PCG_TRY(alloc(M, &cur, lv.nc));
        PCG_TRY(alloc(M, &lv.rptr, (size_t)lv.nc + 1));
        PCG_CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * lv.nc, s));
        PCG_CK(cudaMemsetAsync(cur, 0, sizeof(int32_t) * lv.nc, s));
        k_count_members<<<grid_for(n), kBlock, 0, s>>>(n, lv.agg, cnt);
        PCG_LAUNCH_CK();
        int32_t nm = 0;
        PCG_TRY(scan_exclusive(M, cnt, lv.rptr, lv.nc, &nm, s));
        PCG_TRY(alloc(M, &lv.ridx, nm));
        k_fill_members<<<grid_for(n), kBlock, 0, s>>>(n, lv.agg, lv.rptr, cur, lv.ridx);
        k_sort_members<<<grid_for(lv.nc), kBlock, 0, s>>>(lv.nc, lv.rptr, lv.ridx);
        PCG_LAUNCH_CK();
        PCG_CK(cudaStreamSynchronize(s));
        release(M, cnt);
        release(M, cur);
    }
    return AMG_OK;
}

}  // namespace

// Exclusive prefix sum of n int32 counts into out[0..n], total to the host.
int scan_counts(Mem &M, const int32_t *in, int32_t *out, int64_t n, int32_t *total_host, cudaStream_t s) {
    return scan_exclusive(M, in, out, n, total_host, s);
}

int setup_impl(amg_hier *h, const amg_csr *A, const amg_params *prm, cudaStream_t s) {
    double t_begin = now_ms(), t_match = 0, t_rap = 0;
    Mem &M = h->mem;
    M.stream = s;
    M.budget = prm->hbm_budget;
    h->prm = *prm;
    h->mode = prm->mode;
    h->smoothed = prm->smoothed ? 1 : 0;
    // PCGAMG_GRAPH=0 launches each solve kernel on the stream instead of
    // replaying the whole-solve graph (same kernels; for profilers).
    const char *g = getenv("PCGAMG_GRAPH");
    if (g && g[0] == '0') h->use_graph = 0;
    // PCGAMG_COL16=0 keeps int32 columns on every level.
    const char *c16 = getenv("PCGAMG_COL16");
    if (c16 && c16[0] == '0') h->no_col16 = 1;
    // PCGAMG_UNIFORM=0 stores level 0 without shared offset patterns.
    const char *un = getenv("PCGAMG_UNIFORM");
    if (un && un[0] == '0') h->no_uniform = 1;
    const char *pd = getenv("PCGAMG_PDL");
    if (pd && pd[0] == '0') h->pdl = 0;
    // PCGAMG_GS_FUSED=0 keeps the two-launch Gauss-Seidel sweeps everywhere.
    const char *gf = getenv("PCGAMG_GS_FUSED");
    if (gf && gf[0] == '0') h->gs_fused = 0;
    if (!A || A->n <= 0 || A->n >= (int64_t)1 << 31 || A->nnz < A->n || A->nnz >= (int64_t)1 << 31 ||
        !A->row_ptr || !A->col || !A->val) {
        set_error("amg_setup: bad CSR sizes or NULL arrays");
        return AMG_ERR_ARG;
    }
    if (prm->n_pass < 1 || prm->n_pass > kMaxPass || prm->coarse_max < 1 || prm->max_levels < 1 ||
        (prm->mode != AMG_MODE_PCG64 && prm->mode != AMG_MODE_FCG32) || prm->coarse_solver < AMG_COARSE_AUTO ||
        prm->coarse_solver > AMG_COARSE_ITER || prm->coarse_maxit < 0 || prm->coarse_maxit > 1000 ||
        prm->smoothed < 0 || prm->smoothed > 1 ||
        !(prm->coarse_tol >= 0.0 && prm->coarse_tol < 1.0)) {
        set_error("amg_setup: bad parameters");
        return AMG_ERR_ARG;
    }
    // 0 selects the defaults of the iterative coarsest solve
    if (h->prm.coarse_maxit == 0) h->prm.coarse_maxit = 30;
    if (h->prm.coarse_tol == 0.0) h->prm.coarse_tol = 1e-3;
    int n = (int)A->n;
    int64_t nnz = A->nnz;
    h->lev.reserve((size_t)prm->max_levels + 1);
    h->lev.emplace_back();
    Level &l0 = h->lev[0];
    l0.A.n = n;
    l0.A.nnz = nnz;
    PCG_TRY(alloc(M, &l0.A.rp, (size_t)n + 1));
    PCG_TRY(alloc(M, &l0.A.ci, nnz));
    PCG_TRY(alloc(M, &l0.A.v, nnz));
    cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    PCG_CK(cudaMemcpyAsync(l0.A.rp, A->row_ptr, sizeof(int32_t) * ((size_t)n + 1), kind, s));
    PCG_CK(cudaMemcpyAsync(l0.A.ci, A->col, sizeof(int32_t) * nnz, kind, s));
    PCG_CK(cudaMemcpyAsync(l0.A.v, A->val, sizeof(double) * nnz, kind, s));
    int *dflag = nullptr;
    PCG_TRY(alloc(M, &dflag, 1));
    PCG_CK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
    k_check_csr<<<grid_for(n), kBlock, 0, s>>>(n, l0.A.rp, l0.A.ci, l0.A.v, nnz, dflag);
    PCG_LAUNCH_CK();
    int flag = 0;
    PCG_TRY(read_flag(dflag, s, &flag));
    if (flag == 0) {
        k_check_sym<<<grid_for(n), kBlock, 0, s>>>(n, l0.A.rp, l0.A.ci, l0.A.v, dflag);
        PCG_LAUNCH_CK();
        PCG_TRY(read_flag(dflag, s, &flag));
    }
    release(M, dflag);
    if (flag) {
        set_error("amg_setup: invalid CSR (flags 0x%x: 1 column order/range, 2 diagonal, 4 row "
                  "pointers, 8 not exactly symmetric)", flag);
        return AMG_ERR_ARG;
    }
    PCG_TRY(alloc(M, &l0.w, n));
    k_fill<double><<<grid_for(n), kBlock, 0, s>>>(l0.w, n, 1.0);
    PCG_LAUNCH_CK();

    for (int l = 0;; l++) {
        Level &lv = h->lev[l];
        int nl = lv.A.n;
        if (nl <= prm->coarse_max || l == prm->max_levels - 1) break;
        DevCSR cur = lv.A;
        double *curw = lv.w;
        bool own = false;
        int32_t *cagg = nullptr;
        double *cp = nullptr;
        PCG_TRY(alloc(M, &cagg, nl));
        PCG_TRY(alloc(M, &cp, nl));
        k_iota<<<grid_for(nl), kBlock, 0, s>>>(cagg, nl);
        k_fill<double><<<grid_for(nl), kBlock, 0, s>>>(cp, nl, 1.0);
        PCG_LAUNCH_CK();
        lv.pass_n.push_back(nl);
        for (int ps = 0; ps < prm->n_pass; ps++) {
            int32_t *agg = nullptr;
            double *p = nullptr, *wc = nullptr;
            DevCSR nxt;
            PCG_TRY(pairwise_pass(h, cur, curw, &agg, &p, &nxt, &wc, &t_match, &t_rap, s));
            k_compose<<<grid_for(nl), kBlock, 0, s>>>(nl, cagg, cp, agg, p);
            PCG_LAUNCH_CK();
            PCG_CK(cudaStreamSynchronize(s));
            release(M, p);
            lv.pass_agg.push_back(agg);
            lv.pass_n.push_back(nxt.n);
            if (own) {
                free_csr(M, cur);
                release(M, curw);
            }
            cur = nxt;
            curw = wc;
            own = true;
        }
        int nc = cur.n;
        if (nc == 0 || (double)nc > 0.9 * (double)nl) {
            free_csr(M, cur);
            release(M, curw);
            release(M, cagg);
            release(M, cp);
            for (auto *a : lv.pass_agg) M.release(a);
            lv.pass_agg.clear();
            lv.pass_n.clear();
            break;
        }
        lv.agg = cagg;
        lv.p = cp;
        lv.nc = nc;
        if (h->smoothed) {
            // P = (I - omega D^-1 A) P_hat and A_{l+1} = P^T A P replace the
            // passes' tentative product (which only fed their matchings)
            double t0 = now_ms();
            DevCSR ac;
            PCG_TRY(build_smoothed(h, lv, nc, &ac, s));
            free_csr(M, cur);
            cur = ac;
            t_rap += now_ms() - t0;
        }
        h->lev.emplace_back();
        Level &nx = h->lev[l + 1];
        nx.A = cur;
        nx.w = curw;
    }
    int L = (int)h->lev.size() - 1;
    for (int l = 0; l <= L; l++) PCG_TRY(finish_level(h, h->lev[l], l == L, s));

    // coarsest solver: dense inverse up to kDenseMax rows (AUTO), else the
    // iterative FCG + block-Jacobi ILU(1) solve of Sec. 3.1
    Level &lc = h->lev[L];
    int nL = lc.A.n;
    int cs = prm->coarse_solver;
    h->coarse_iter = cs == AMG_COARSE_ITER || (cs == AMG_COARSE_AUTO && nL > kDenseMax) ? 1 : 0;
    if (h->coarse_iter && L == 0) {
        if (cs == AMG_COARSE_ITER) {
            set_error("amg_setup: the iterative coarsest solve needs at least two levels (lower coarse_max)");
            return AMG_ERR_ARG;
        }
        set_error("amg_setup: single level of %d rows above the dense limit %d (lower coarse_max)", nL, kDenseMax);
        return AMG_ERR_COARSE;
    }
    if (!h->coarse_iter && nL > kDenseMax) {
        set_error("amg_setup: coarsening stalled at %d rows (dense limit %d)", nL, kDenseMax);
        return AMG_ERR_COARSE;
    }
    h->nL = nL;
    PCG_TRY(alloc(M, &h->bL, nL));
    if (h->coarse_iter) {
        PCG_TRY(coarse_iter_build(h, s));
        PCG_TRY(alloc_solve_workspace(h));
        PCG_CK(cudaStreamSynchronize(s));
        h->setup_ms[0] = now_ms() - t_begin;
        h->setup_ms[1] = t_match;
        h->setup_ms[2] = t_rap;
        h->setup_ms[3] = h->setup_ms[0] - t_match - t_rap;
        return AMG_OK;
    }
    double *ad = nullptr;
    PCG_TRY(alloc(M, &ad, (size_t)nL * nL));
    PCG_TRY(alloc(M, &h->Ainv, (size_t)nL * nL));
    PCG_TRY(alloc(M, &dflag, 1));
    PCG_CK(cudaMemsetAsync(ad, 0, sizeof(double) * (size_t)nL * nL, s));
    PCG_CK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
    k_dense<<<grid_for(nL), kBlock, 0, s>>>(nL, lc.A.rp, lc.A.ci, lc.A.v, ad);
    k_chol<<<1, 256, 0, s>>>(nL, ad, dflag);
    PCG_LAUNCH_CK();
    PCG_TRY(read_flag(dflag, s, &flag));
    release(M, dflag);
    if (flag) {
        release(M, ad);
        set_error("amg_setup: coarsest matrix is not SPD (Cholesky pivot <= 0)");
        return AMG_ERR_BREAKDOWN;
    }
    k_chol_inverse<<<nL, 256, sizeof(double) * nL, s>>>(nL, ad, h->Ainv);
    PCG_LAUNCH_CK();
    PCG_CK(cudaStreamSynchronize(s));
    release(M, ad);
    PCG_TRY(alloc_solve_workspace(h));
    PCG_CK(cudaStreamSynchronize(s));
    h->setup_ms[0] = now_ms() - t_begin;
    h->setup_ms[1] = t_match;
    h->setup_ms[2] = t_rap;
    h->setup_ms[3] = h->setup_ms[0] - t_match - t_rap;
    return AMG_OK;
}

// Partial reuse (Sec. 4): new values of the finest matrix on the pattern the
// hierarchy was built on. Every pass keeps its aggregates; its weights are
// formed again from the map and w (they do not depend on the values), then
// the Galerkin products pass by pass, the l1 diagonals, the sliced-ELL values
// and the coarsest inverse. Every array keeps its address, so captured solve
// graphs, batch graphs and serving engines stay valid. Nothing is changed
// when the input is rejected (AMG_ERR_ARG).
int refresh_impl(amg_hier *h, const amg_csr *A, cudaStream_t s) {
    double t_begin = now_ms();
    Mem &M = h->mem;
    M.stream = s;
    Level &l0 = h->lev[0];
    int n = l0.A.n;
    int64_t nnz = l0.A.nnz;
    if (!A || A->n != n || A->nnz != nnz || !A->row_ptr || !A->col || !A->val) {
        set_error("amg_refresh: sizes differ from the hierarchy's matrix, or NULL arrays");
        return AMG_ERR_ARG;
    }
    int32_t *rp = nullptr, *ci = nullptr;
    double *v = nullptr;
    int *dflag = nullptr;
    PCG_TRY(alloc(M, &rp, (size_t)n + 1));
    PCG_TRY(alloc(M, &ci, nnz));
    PCG_TRY(alloc(M, &v, nnz));
    PCG_TRY(alloc(M, &dflag, 1));
    cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    PCG_CK(cudaMemcpyAsync(rp, A->row_ptr, sizeof(int32_t) * ((size_t)n + 1), kind, s));
    PCG_CK(cudaMemcpyAsync(ci, A->col, sizeof(int32_t) * nnz, kind, s));
    PCG_CK(cudaMemcpyAsync(v, A->val, sizeof(double) * nnz, kind, s));
    PCG_CK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
    k_same_pattern<<<grid_for(nnz > n ? nnz : (int64_t)n + 1), kBlock, 0, s>>>(n, nnz, rp, ci, l0.A.rp, l0.A.ci,
                                                                               dflag);
    PCG_LAUNCH_CK();
    int flag = 0;
    PCG_TRY(read_flag(dflag, s, &flag));
    if (!flag) {
        k_check_csr<<<grid_for(n), kBlock, 0, s>>>(n, rp, ci, v, nnz, dflag);
        PCG_LAUNCH_CK();
        PCG_TRY(read_flag(dflag, s, &flag));
    }
    if (!flag) {
        k_check_sym<<<grid_for(n), kBlock, 0, s>>>(n, rp, ci, v, dflag);
        PCG_LAUNCH_CK();
        PCG_TRY(read_flag(dflag, s, &flag));
    }
    release(M, rp);
    release(M, ci);
    if (flag) {
        release(M, v);
        release(M, dflag);
        set_error("amg_refresh: rejected (flags 0x%x: 16 another sparsity pattern, 1 column order/range, "
                  "2 diagonal, 4 row pointers, 8 not exactly symmetric)", flag);
        return AMG_ERR_ARG;
    }
    PCG_CK(cudaMemcpyAsync(l0.A.v, v, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, s));
    PCG_CK(cudaStreamSynchronize(s));
    release(M, v);
    h->invalid = 1;  // until every level and the coarsest inverse are rebuilt
    int L = (int)h->lev.size() - 1;
    for (int l = 0; l < L; l++) {
        Level &lv = h->lev[l];
        if (h->smoothed) {
            // P and A_{l+1} = P^T A P formed again on their kept patterns
            // from the kept map and weight (which do not depend on values)
            int st = build_smoothed(h, lv, h->lev[l + 1].A.n, &h->lev[l + 1].A, s);
            if (st) {
                release(M, dflag);
                return st;
            }
            continue;
        }
        DevCSR cur = lv.A;
        double *curw = lv.w;
        bool own = false;
        int npass = (int)lv.pass_agg.size();
        for (int ps = 0; ps < npass; ps++) {
            int m = lv.pass_n[ps], nc = lv.pass_n[ps + 1];
            const int32_t *agg = lv.pass_agg[ps];
            int32_t *first = nullptr, *second = nullptr, *mem0 = nullptr, *mem1 = nullptr;
            double *p = nullptr, *wc = nullptr;
            PCG_TRY(alloc(M, &first, nc));
            PCG_TRY(alloc(M, &second, nc));
            PCG_TRY(alloc(M, &mem0, nc));
            PCG_TRY(alloc(M, &mem1, nc));
            PCG_TRY(alloc(M, &p, m));
            PCG_TRY(alloc(M, &wc, nc));
            k_fill<int32_t><<<grid_for(nc), kBlock, 0, s>>>(first, nc, INT32_MAX);
            k_fill<int32_t><<<grid_for(nc), kBlock, 0, s>>>(second, nc, -1);
            k_fill<double><<<grid_for(m), kBlock, 0, s>>>(p, m, 0.0);
            k_pass_members<<<grid_for(m), kBlock, 0, s>>>(m, agg, first, second);
            PCG_CK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
            k_pass_weights<<<grid_for(nc), kBlock, 0, s>>>(m, nc, first, second, curw, p, wc, mem0, mem1, dflag);
            PCG_LAUNCH_CK();
            PCG_TRY(read_flag(dflag, s, &flag));
            if (flag) {
                set_error("amg_refresh: level %d pass %d has an aggregate without members", l, ps);
                return AMG_ERR_CUDA;
            }
            DevCSR nxt;
            PCG_TRY(galerkin(h, cur, agg, p, mem0, mem1, nc, &nxt, s));
            release(M, first);
            release(M, second);
            release(M, mem0);
            release(M, mem1);
            release(M, p);
            if (own) {
                free_csr(M, cur);
                release(M, curw);
            }
            cur = nxt;
            curw = wc;
            own = true;
        }
        // the last pass gives A_{l+1} on its kept pattern
        Level &nx = h->lev[l + 1];
        flag = cur.n != nx.A.n || cur.nnz != nx.A.nnz;
        if (!flag) {
            PCG_CK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
            k_same_pattern<<<grid_for(cur.nnz > cur.n ? cur.nnz : (int64_t)cur.n + 1), kBlock, 0, s>>>(
                cur.n, cur.nnz, cur.rp, cur.ci, nx.A.rp, nx.A.ci, dflag);
            PCG_LAUNCH_CK();
            PCG_TRY(read_flag(dflag, s, &flag));
        }
        if (!flag)
            PCG_CK(cudaMemcpyAsync(nx.A.v, cur.v, sizeof(double) * cur.nnz, cudaMemcpyDeviceToDevice, s));
        PCG_CK(cudaStreamSynchronize(s));
        if (own) {
            free_csr(M, cur);
            release(M, curw);
        }
        if (flag) {
            release(M, dflag);
            set_error("amg_refresh: level %d came out with another pattern", l + 1);
            return AMG_ERR_CUDA;
        }
    }
    for (int l = 0; l <= L; l++) {
        Level &lv = h->lev[l];
        Sell &S = lv.S;
        int nl = lv.A.n;
        if (h->gs_nu > 0)
            k_hybrid_l1<<<grid_for(nl), kBlock, 0, s>>>(nl, gs_rows(nl, h->gs_blocks), lv.A.rp, lv.A.ci, lv.A.v,
                                                        lv.dinv, lv.dinv32);
        else
            k_l1diag<<<grid_for(nl), kBlock, 0, s>>>(nl, lv.A.rp, lv.A.v, lv.dinv, lv.dinv32);
        k_sell_vals<<<grid_for((int64_t)S.nslices * kSlice), kBlock, 0, s>>>(nl, S.nslices, lv.A.rp, lv.A.ci,
                                                                             lv.A.v, S.sptr, S.upat, S.v64, S.v32);
        if (lv.v32csr) k_to_f32<<<grid_for(lv.A.nnz), kBlock, 0, s>>>(lv.A.v, lv.v32csr, lv.A.nnz);
        PCG_LAUNCH_CK();
        if (h->gs_nu) PCG_TRY(fill_gs_parts(lv, h->gs_blocks, s));
    }
    // coarsest solver's data, in place
    Level &lc = h->lev[L];
    int nL = lc.A.n;
    if (h->coarse_iter) {
        release(M, dflag);
        int st = coarse_iter_build(h, s);
        if (st) {
            set_error("amg_refresh: an ILU(1) pivot of the coarsest level is not positive; the handle refuses "
                      "solves until a refresh succeeds");
            return st;
        }
        h->invalid = 0;
        h->refresh_ms = now_ms() - t_begin;
        return AMG_OK;
    }
    double *ad = nullptr;
    PCG_TRY(alloc(M, &ad, (size_t)nL * nL));
    PCG_CK(cudaMemsetAsync(ad, 0, sizeof(double) * (size_t)nL * nL, s));
    PCG_CK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
    k_dense<<<grid_for(nL), kBlock, 0, s>>>(nL, lc.A.rp, lc.A.ci, lc.A.v, ad);
    k_chol<<<1, 256, 0, s>>>(nL, ad, dflag);
    PCG_LAUNCH_CK();
    PCG_TRY(read_flag(dflag, s, &flag));
    release(M, dflag);
    if (flag) {
        release(M, ad);
        set_error("amg_refresh: coarsest matrix is not SPD (Cholesky pivot <= 0); the handle refuses "
                  "solves until a refresh succeeds");
        return AMG_ERR_BREAKDOWN;
    }
    k_chol_inverse<<<nL, 256, sizeof(double) * nL, s>>>(nL, ad, h->Ainv);
    PCG_LAUNCH_CK();
    PCG_CK(cudaStreamSynchronize(s));
    release(M, ad);
    PCG_TRY(refresh_smem_tail(h));
    h->invalid = 0;
    h->refresh_ms = now_ms() - t_begin;
    return AMG_OK;
}

// Rows per Gauss-Seidel block of a level with n rows: nblocks contiguous
// blocks per level ("processes", Sec. 3.1), so blocks shrink on coarser
// levels; nblocks = 0 gives one row per block.
int gs_rows(int n, int nblocks) {
    if (nblocks <= 0) return 1;
    int64_t nb = ((int64_t)n + nblocks - 1) / nblocks;
    return nb < 1 ? 1 : (int)nb;
}

// The two-phase sweep tables of a level (values of its current matrix): for
// blocks of at most 32 rows whose rows have at most kGsPart already-updated
// in-block entries; other levels keep gs_w = -1 (one thread per block).
constexpr int kGsPart = 8;
int build_gs_parts(amg_hier *h, Level &lv, int nblocks, cudaStream_t s) {
    Mem &M = h->mem;
    int n = lv.A.n, nb = gs_rows(n, nblocks);
    for (int d = 0; d < 2; d++) {
        release(M, lv.gs_ci[d]);
        release(M, lv.gs_v64[d]);
        release(M, lv.gs_v32[d]);
        lv.gs_w[d] = -1;
    }
    if (nb > 32) return AMG_OK;
    int32_t *cnt = nullptr;
    PCG_TRY(alloc(M, &cnt, n));
    std::vector<int32_t> hc(n);
    for (int d = 0; d < 2; d++) {
        if (d == 0) k_part_count<true><<<grid_for(n), kBlock, 0, s>>>(n, nb, lv.A.rp, lv.A.ci, cnt);
        else k_part_count<false><<<grid_for(n), kBlock, 0, s>>>(n, nb, lv.A.rp, lv.A.ci, cnt);
        PCG_LAUNCH_CK();
        PCG_CK(cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaStreamSynchronize(s));
        int w = 0;
        for (int i = 0; i < n; i++) w = std::max(w, (int)hc[i]);
        if (w > kGsPart) continue;
        lv.gs_w[d] = w;
        if (w > 0) {
            PCG_TRY(alloc(M, &lv.gs_ci[d], (size_t)n * w));
            PCG_TRY(alloc(M, &lv.gs_v64[d], (size_t)n * w));
            PCG_TRY(alloc(M, &lv.gs_v32[d], (size_t)n * w));
        }
    }
    release(M, cnt);
    if (!lv.gs_acc) PCG_TRY(alloc(M, &lv.gs_acc, n));
    return fill_gs_parts(lv, nblocks, s);
}

// Values of the tables (after a setup of the smoother or a refresh).
int fill_gs_parts(Level &lv, int nblocks, cudaStream_t s) {
    int n = lv.A.n, nb = gs_rows(n, nblocks);
    for (int d = 0; d < 2; d++) {
        int w = lv.gs_w[d];
        if (w <= 0) continue;
        if (d == 0)
            k_part_fill<true><<<grid_for(n), kBlock, 0, s>>>(n, nb, w, lv.A.rp, lv.A.ci, lv.A.v, lv.gs_ci[d],
                                                             lv.gs_v64[d], lv.gs_v32[d]);
        else
            k_part_fill<false><<<grid_for(n), kBlock, 0, s>>>(n, nb, w, lv.A.rp, lv.A.ci, lv.A.v, lv.gs_ci[d],
                                                              lv.gs_v64[d], lv.gs_v32[d]);
        PCG_LAUNCH_CK();
    }
    return AMG_OK;
}

// Smoother of the V-cycle: nu = 0 restores the setup's one-sweep l1-Jacobi;
// nu >= 1 selects nu sweeps of l1 hybrid Gauss-Seidel over nblocks row blocks
// per level (Sec. 3.1 with the l1 reading). Forms D^-1 by the block rule and
// the float32 CSR values the sweeps read; captured graphs are dropped.
int set_smoother_impl(amg_hier *h, int nu, int nblocks, cudaStream_t s) {
    Mem &M = h->mem;
    M.stream = s;
    PCG_CK(cudaStreamSynchronize(s));
    drop_graphs(h);
    h->gs_nu = 0;  // the Jacobi diagonals until the new ones are in place
    for (Level &lv : h->lev) {
        int nl = lv.A.n;
        if (nu > 0) {
            if (!lv.v32csr) {
                PCG_TRY(alloc(M, &lv.v32csr, lv.A.nnz));
                k_to_f32<<<grid_for(lv.A.nnz), kBlock, 0, s>>>(lv.A.v, lv.v32csr, lv.A.nnz);
            }
            k_hybrid_l1<<<grid_for(nl), kBlock, 0, s>>>(nl, gs_rows(nl, nblocks), lv.A.rp, lv.A.ci, lv.A.v, lv.dinv,
                                                        lv.dinv32);
            PCG_TRY(build_gs_parts(h, lv, nblocks, s));
        } else {
            k_l1diag<<<grid_for(nl), kBlock, 0, s>>>(nl, lv.A.rp, lv.A.v, lv.dinv, lv.dinv32);
        }
        PCG_LAUNCH_CK();
    }
    PCG_CK(cudaStreamSynchronize(s));
    // the cluster tail's shared-memory image holds the small levels' D^-1:
    // form it again from the diagonals now in place (used while nu = 0)
    PCG_TRY(refresh_smem_tail(h));
    h->gs_nu = nu;
    h->gs_blocks = nu > 0 ? nblocks : 0;
    return AMG_OK;
}

}  // namespace pcgamg
