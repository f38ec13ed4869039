// Smoothed aggregation (arxiv 2210.16660, Sec. 3.1): the prolongator actually
// used is P = (I - omega D^-1 A) P_hat, D = diag(A), omega = 1 / ||D^-1 A||_inf,
// with P_hat the level's composed tentative prolongator (its pass maps and
// weights multiplied), and the next level's matrix is the Galerkin product
// P^T A P formed with that explicit P.
//
// Every value is formed with the summation order the CPU oracle states, each
// operation rounded on its own, so P and every coarse matrix equal the
// oracle's bit for bit (the next level's matching reads them):
//   * row i of P: the tentative entry p_i at column agg(i), then for each
//     stored a_ij (storage order) with agg(j) >= 0 the term
//     -((omega / a_ii) a_ij) p_j for column agg(j); one column's terms are
//     added in increasing j, the tentative one first;
//   * (A P)_iJ: the sum over row i's entries a_ik in storage order of
//     a_ik P_kJ, formed by a merge over the sorted rows P_k. of the row's
//     neighbours, so each column's terms arrive in storage order;
//   * A_c = P^T A P: row I, columns J >= I, the sum over the rows i of P's
//     column I (increasing i) of P_iI (A P)_iJ, again by a merge; the entries
//     below the diagonal are mirrored from above (bitwise symmetric).
// One thread per row; count passes size the outputs before fill passes.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "internal.cuh"

namespace pcgamg {

namespace {

__device__ __forceinline__ double diag_of(const int32_t *rp, const int32_t *ci, const double *v, int i) {
    for (int32_t k = rp[i]; k < rp[i + 1]; k++)
        if (ci[k] == i) return v[k];
    return 0.0;
}

// ||D^-1 A||_inf: the largest row sum of |a_ij| / a_ii (storage order);
// the sums are non-negative, so their IEEE bit patterns order like them.
__global__ void k_sa_rowsum(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, unsigned long long *mx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = diag_of(rp, ci, v, i), s = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; k++) s = __dadd_rn(s, __ddiv_rn(fabs(v[k]), d));
    atomicMax(mx, (unsigned long long)__double_as_longlong(s));
}

// Terms of P's row i: one for the tentative entry, one per stored neighbour
// inside the coarse space.
__global__ void k_sa_tcount(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const int32_t *__restrict__ agg, int32_t *__restrict__ cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = agg[i] >= 0 ? 1 : 0;
    for (int32_t k = rp[i]; k < rp[i + 1]; k++) c += agg[ci[k]] >= 0 ? 1 : 0;
    cnt[i] = c;
}

// The terms (J, j, t) of row i in its slots [toff[i], toff[i+1]), sorted by
// (J, j) with the tentative term (j = -1) first; pcnt[i] = distinct columns.
__global__ void k_sa_terms(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ v, const int32_t *__restrict__ agg,
                           const double *__restrict__ p, double omega, const int32_t *__restrict__ toff,
                           int32_t *__restrict__ tJ, int32_t *__restrict__ tj, double *__restrict__ tt,
                           int32_t *__restrict__ pcnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t o = toff[i];
    int m = 0;
    double s = __ddiv_rn(omega, diag_of(rp, ci, v, i));
    auto put = [&](int J, int j, double t) {
        // insertion into the sorted prefix [o, o + m)
        int x = m;
        while (x > 0) {
            int Jp = tJ[o + x - 1], jp = tj[o + x - 1];
            if (Jp < J || (Jp == J && jp < j)) break;
            tJ[o + x] = Jp;
            tj[o + x] = jp;
            tt[o + x] = tt[o + x - 1];
            x--;
        }
        tJ[o + x] = J;
        tj[o + x] = j;
        tt[o + x] = t;
        m++;
    };
    if (agg[i] >= 0) put(agg[i], -1, p[i]);
    for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
        int j = ci[k];
        if (agg[j] < 0) continue;
        put(agg[j], j, __dmul_rn(-__dmul_rn(s, v[k]), p[j]));
    }
    int d = 0;
    for (int x = 0; x < m; x++) d += (x == 0 || tJ[o + x] != tJ[o + x - 1]) ? 1 : 0;
    pcnt[i] = d;
}

// Merges each row's sorted terms into P (values added in term order).
__global__ void k_sa_pfill(int n, const int32_t *__restrict__ toff, const int32_t *__restrict__ tJ,
                           const double *__restrict__ tt, const int32_t *__restrict__ prp, int32_t *__restrict__ pci,
                           double *__restrict__ pv, float *__restrict__ pv32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t q = prp[i] - 1;
    for (int32_t x = toff[i]; x < toff[i + 1]; x++) {
        if (x == toff[i] || tJ[x] != tJ[x - 1]) {
            q++;
            pci[q] = tJ[x];
            pv[q] = tt[x];
        } else {
            pv[q] = __dadd_rn(pv[q], tt[x]);
        }
    }
    for (int32_t r = prp[i]; r < prp[i + 1]; r++) pv32[r] = __double2float_rn(pv[r]);
}

// Row i of A P by a merge over the P rows of i's neighbours: the smallest
// remaining column J, then every neighbour whose row holds J (storage order)
// adds a_ik P_kJ. FILL = false counts the columns; FILL = true writes them.
// ptr: scratch of one cursor per stored entry of A.
template <bool FILL>
__global__ void k_sa_ap(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                        const double *__restrict__ v, const int32_t *__restrict__ prp,
                        const int32_t *__restrict__ pci, const double *__restrict__ pv, int32_t *__restrict__ ptr,
                        int32_t *__restrict__ cnt, const int32_t *__restrict__ orp, int32_t *__restrict__ oci,
                        double *__restrict__ ov) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t k0 = rp[i], k1 = rp[i + 1];
    for (int32_t k = k0; k < k1; k++) ptr[k] = prp[ci[k]];
    int32_t out = FILL ? orp[i] : 0;
    int d = 0;
    for (;;) {
        int J = INT32_MAX;
        for (int32_t k = k0; k < k1; k++) {
            int32_t q = ptr[k];
            if (q < prp[ci[k] + 1]) J = min(J, pci[q]);
        }
        if (J == INT32_MAX) break;
        double acc = 0.0;
        for (int32_t k = k0; k < k1; k++) {
            int32_t q = ptr[k];
            if (q < prp[ci[k] + 1] && pci[q] == J) {
                if (FILL) acc = __dadd_rn(acc, __dmul_rn(v[k], pv[q]));
                ptr[k] = q + 1;
            }
        }
        if (FILL) {
            oci[out] = J;
            ov[out] = acc;
            out++;
        }
        d++;
    }
    if (!FILL) cnt[i] = d;
}

// P^T: entries counted per column, placed, then each column sorted by row.
__global__ void k_sa_tcnt(int n, const int32_t *__restrict__ prp, const int32_t *__restrict__ pci,
                          int32_t *__restrict__ cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t q = prp[i]; q < prp[i + 1]; q++) atomicAdd(&cnt[pci[q]], 1);
}

__global__ void k_sa_tplace(int n, const int32_t *__restrict__ prp, const int32_t *__restrict__ pci,
                            const double *__restrict__ pv, int32_t *__restrict__ fill, int32_t *__restrict__ tri,
                            double *__restrict__ trv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t q = prp[i]; q < prp[i + 1]; q++) {
        int32_t pos = atomicAdd(&fill[pci[q]], 1);
        tri[pos] = i;
        trv[pos] = pv[q];
    }
}

// Sorts each segment [off[r], off[r+1]) of (key, val) by key (insertion).
__global__ void k_sa_segsort(int rows, const int32_t *__restrict__ off, int32_t *__restrict__ key,
                             double *__restrict__ val) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int32_t a = off[r], b = off[r + 1];
    for (int32_t x = a + 1; x < b; x++) {
        int32_t kx = key[x];
        double vx = val[x];
        int32_t y = x;
        while (y > a && key[y - 1] > kx) {
            key[y] = key[y - 1];
            val[y] = val[y - 1];
            y--;
        }
        key[y] = kx;
        val[y] = vx;
    }
}

__global__ void k_sa_to_f32(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __double2float_rn(a[i]);
}

// Upper part of row I of P^T A P (columns J >= I) by a merge over the AP
// rows of the rows i in P's column I (increasing i). ptr: one cursor per
// entry of P^T. FILL = false counts (and the mirrored entries per column
// J > I into lcnt); FILL = true writes the upper part after the row's lower
// part and places the mirrored entries.
template <bool FILL>
__global__ void k_sa_rap(int nc, const int32_t *__restrict__ trp, const int32_t *__restrict__ tri,
                         const double *__restrict__ trv, const int32_t *__restrict__ arp,
                         const int32_t *__restrict__ aci, const double *__restrict__ av, int32_t *__restrict__ ptr,
                         int32_t *__restrict__ ucnt, int32_t *__restrict__ lcnt, const int32_t *__restrict__ crp,
                         int32_t *__restrict__ lfill, int32_t *__restrict__ cci, double *__restrict__ cv) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int32_t q0 = trp[I], q1 = trp[I + 1];
    for (int32_t q = q0; q < q1; q++) {
        int i = tri[q];
        int32_t r = arp[i];
        while (r < arp[i + 1] && aci[r] < I) r++;
        ptr[q] = r;
    }
    int32_t out = 0;
    if (FILL) out = crp[I] + lcnt[I];
    int d = 0;
    for (;;) {
        int J = INT32_MAX;
        for (int32_t q = q0; q < q1; q++) {
            int i = tri[q];
            int32_t r = ptr[q];
            if (r < arp[i + 1]) J = min(J, aci[r]);
        }
        if (J == INT32_MAX) break;
        double acc = 0.0;
        for (int32_t q = q0; q < q1; q++) {
            int i = tri[q];
            int32_t r = ptr[q];
            if (r < arp[i + 1] && aci[r] == J) {
                if (FILL) acc = __dadd_rn(acc, __dmul_rn(trv[q], av[r]));
                ptr[q] = r + 1;
            }
        }
        if (FILL) {
            cci[out] = J;
            cv[out] = acc;
            out++;
            if (J != I) {
                int32_t pos = atomicAdd(&lfill[J], 1);
                cci[pos] = I;
                cv[pos] = acc;
            }
        } else if (J != I) {
            atomicAdd(&lcnt[J], 1);
        }
        d++;
    }
    if (!FILL) ucnt[I] = d;
}

__global__ void k_sa_rowlen(int nc, const int32_t *__restrict__ ucnt, const int32_t *__restrict__ lcnt,
                            int32_t *__restrict__ len) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I < nc) len[I] = ucnt[I] + lcnt[I];
}

// The mirrored part of each row, [crp[I], crp[I] + lcnt[I]), sorted by column.
__global__ void k_sa_lowsort(int nc, const int32_t *__restrict__ crp, const int32_t *__restrict__ lcnt,
                             int32_t *__restrict__ cci, double *__restrict__ cv) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    int32_t a = crp[I], b = crp[I] + lcnt[I];
    for (int32_t x = a + 1; x < b; x++) {
        int32_t kx = cci[x];
        double vx = cv[x];
        int32_t y = x;
        while (y > a && cci[y - 1] > kx) {
            cci[y] = cci[y - 1];
            cv[y] = cv[y - 1];
            y--;
        }
        cci[y] = kx;
        cv[y] = vx;
    }
}

inline int grid_n(int64_t n, int b = kBlock) { return (int)((n + b - 1) / b); }

}  // namespace

// Smoothed prolongator P of level lv (its matrix, composed map and weight,
// nc coarse rows), its transpose, and the coarse matrix P^T A P into *out.
// When lv.P already exists (a refresh) the patterns are kept and only the
// values are formed again; AMG_ERR_ARG if a pattern came out different.
int build_smoothed(amg_hier *h, Level &lv, int nc, DevCSR *out, cudaStream_t s) {
    Mem &M = h->mem;
    const DevCSR &A = lv.A;
    int n = A.n;
    // omega = 1 / ||D^-1 A||_inf
    unsigned long long *dmx = nullptr;
    PCG_TRY(alloc(M, &dmx, 1));
    PCG_CK(cudaMemsetAsync(dmx, 0, sizeof(unsigned long long), s));
    k_sa_rowsum<<<grid_n(n), kBlock, 0, s>>>(n, A.rp, A.ci, A.v, dmx);
    PCG_LAUNCH_CK();
    unsigned long long bits = 0;
    PCG_CK(cudaMemcpyAsync(&bits, dmx, sizeof(bits), cudaMemcpyDeviceToHost, s));
    PCG_CK(cudaStreamSynchronize(s));
    release(M, dmx);
    double mx;
    memcpy(&mx, &bits, sizeof(mx));
    double omega = 1.0 / mx;
    // terms of P
    int32_t *tcnt = nullptr, *toff = nullptr, *tJ = nullptr, *tj = nullptr, *pcnt = nullptr;
    double *tt = nullptr;
    PCG_TRY(alloc(M, &tcnt, n));
    PCG_TRY(alloc(M, &toff, (size_t)n + 1));
    k_sa_tcount<<<grid_n(n), kBlock, 0, s>>>(n, A.rp, A.ci, lv.agg, tcnt);
    PCG_LAUNCH_CK();
    int32_t nterm = 0;
    PCG_TRY(scan_counts(M, tcnt, toff, n, &nterm, s));
    release(M, tcnt);
    PCG_TRY(alloc(M, &tJ, nterm));
    PCG_TRY(alloc(M, &tj, nterm));
    PCG_TRY(alloc(M, &tt, nterm));
    PCG_TRY(alloc(M, &pcnt, n));
    k_sa_terms<<<grid_n(n, 128), 128, 0, s>>>(n, A.rp, A.ci, A.v, lv.agg, lv.p, omega, toff, tJ, tj, tt, pcnt);
    PCG_LAUNCH_CK();
    release(M, tj);
    const bool fresh = lv.P.rp == nullptr;
    DevCSR P;
    P.n = n;
    PCG_TRY(alloc(M, &P.rp, (size_t)n + 1));
    int32_t pnz = 0;
    PCG_TRY(scan_counts(M, pcnt, P.rp, n, &pnz, s));
    release(M, pcnt);
    P.nnz = pnz;
    PCG_TRY(alloc(M, &P.ci, pnz));
    PCG_TRY(alloc(M, &P.v, pnz));
    float *p32 = nullptr;
    PCG_TRY(alloc(M, &p32, pnz));
    k_sa_pfill<<<grid_n(n), kBlock, 0, s>>>(n, toff, tJ, tt, P.rp, P.ci, P.v, p32);
    PCG_LAUNCH_CK();
    release(M, toff);
    release(M, tJ);
    release(M, tt);
    // A P
    DevCSR AP;
    AP.n = n;
    int32_t *cur = nullptr, *cnt = nullptr;
    PCG_TRY(alloc(M, &cur, A.nnz));
    PCG_TRY(alloc(M, &cnt, n));
    PCG_TRY(alloc(M, &AP.rp, (size_t)n + 1));
    k_sa_ap<false><<<grid_n(n, 128), 128, 0, s>>>(n, A.rp, A.ci, A.v, P.rp, P.ci, P.v, cur, cnt, nullptr, nullptr,
                                                  nullptr);
    PCG_LAUNCH_CK();
    int32_t apnz = 0;
    PCG_TRY(scan_counts(M, cnt, AP.rp, n, &apnz, s));
    AP.nnz = apnz;
    PCG_TRY(alloc(M, &AP.ci, apnz));
    PCG_TRY(alloc(M, &AP.v, apnz));
    k_sa_ap<true><<<grid_n(n, 128), 128, 0, s>>>(n, A.rp, A.ci, A.v, P.rp, P.ci, P.v, cur, nullptr, AP.rp, AP.ci,
                                                 AP.v);
    PCG_LAUNCH_CK();
    release(M, cur);
    release(M, cnt);
    // P^T (rows of each column in increasing order)
    DevCSR Pt;
    Pt.n = nc;
    Pt.nnz = pnz;
    int32_t *ccnt = nullptr, *cfill = nullptr;
    PCG_TRY(alloc(M, &ccnt, nc));
    PCG_TRY(alloc(M, &Pt.rp, (size_t)nc + 1));
    PCG_CK(cudaMemsetAsync(ccnt, 0, sizeof(int32_t) * nc, s));
    k_sa_tcnt<<<grid_n(n), kBlock, 0, s>>>(n, P.rp, P.ci, ccnt);
    PCG_LAUNCH_CK();
    int32_t tnz = 0;
    PCG_TRY(scan_counts(M, ccnt, Pt.rp, nc, &tnz, s));
    release(M, ccnt);
    PCG_TRY(alloc(M, &Pt.ci, pnz));
    PCG_TRY(alloc(M, &Pt.v, pnz));
    PCG_TRY(alloc(M, &cfill, nc));
    PCG_CK(cudaMemcpyAsync(cfill, Pt.rp, sizeof(int32_t) * nc, cudaMemcpyDeviceToDevice, s));
    k_sa_tplace<<<grid_n(n), kBlock, 0, s>>>(n, P.rp, P.ci, P.v, cfill, Pt.ci, Pt.v);
    k_sa_segsort<<<grid_n(nc), kBlock, 0, s>>>(nc, Pt.rp, Pt.ci, Pt.v);
    PCG_LAUNCH_CK();
    release(M, cfill);
    float *pt32 = nullptr;
    PCG_TRY(alloc(M, &pt32, pnz));
    k_sa_to_f32<<<grid_n(pnz), kBlock, 0, s>>>(Pt.v, pt32, pnz);
    PCG_LAUNCH_CK();
    // P^T A P: upper part by merge, lower part mirrored
    DevCSR C;
    C.n = nc;
    int32_t *uc = nullptr, *lc = nullptr, *len = nullptr, *lfill = nullptr, *tcur = nullptr;
    PCG_TRY(alloc(M, &uc, nc));
    PCG_TRY(alloc(M, &lc, nc));
    PCG_TRY(alloc(M, &tcur, pnz));
    PCG_CK(cudaMemsetAsync(lc, 0, sizeof(int32_t) * nc, s));
    k_sa_rap<false><<<grid_n(nc, 128), 128, 0, s>>>(nc, Pt.rp, Pt.ci, Pt.v, AP.rp, AP.ci, AP.v, tcur, uc, lc,
                                                    nullptr, nullptr, nullptr, nullptr);
    PCG_LAUNCH_CK();
    PCG_TRY(alloc(M, &len, nc));
    k_sa_rowlen<<<grid_n(nc), kBlock, 0, s>>>(nc, uc, lc, len);
    PCG_LAUNCH_CK();
    PCG_TRY(alloc(M, &C.rp, (size_t)nc + 1));
    int32_t cnz = 0;
    PCG_TRY(scan_counts(M, len, C.rp, nc, &cnz, s));
    C.nnz = cnz;
    PCG_TRY(alloc(M, &C.ci, cnz));
    PCG_TRY(alloc(M, &C.v, cnz));
    PCG_TRY(alloc(M, &lfill, nc));
    PCG_CK(cudaMemcpyAsync(lfill, C.rp, sizeof(int32_t) * nc, cudaMemcpyDeviceToDevice, s));
    k_sa_rap<true><<<grid_n(nc, 128), 128, 0, s>>>(nc, Pt.rp, Pt.ci, Pt.v, AP.rp, AP.ci, AP.v, tcur, uc, lc, C.rp,
                                                   lfill, C.ci, C.v);
    k_sa_lowsort<<<grid_n(nc), kBlock, 0, s>>>(nc, C.rp, lc, C.ci, C.v);
    PCG_LAUNCH_CK();
    PCG_CK(cudaStreamSynchronize(s));
    release(M, uc);
    release(M, lc);
    release(M, len);
    release(M, lfill);
    release(M, tcur);
    release(M, AP.rp);
    release(M, AP.ci);
    release(M, AP.v);
    if (fresh) {
        lv.P = P;
        lv.P32 = p32;
        lv.Pt = Pt;
        lv.Pt32 = pt32;
        *out = C;
        return AMG_OK;
    }
    // refresh: same patterns, new values in place (addresses kept)
    int st = AMG_OK;
    if (P.nnz != lv.P.nnz || Pt.nnz != lv.Pt.nnz || C.nnz != out->nnz) st = AMG_ERR_ARG;
    if (!st) {
        PCG_CK(cudaMemcpyAsync(lv.P.v, P.v, sizeof(double) * P.nnz, cudaMemcpyDeviceToDevice, s));
        PCG_CK(cudaMemcpyAsync(lv.P32, p32, sizeof(float) * P.nnz, cudaMemcpyDeviceToDevice, s));
        PCG_CK(cudaMemcpyAsync(lv.Pt.v, Pt.v, sizeof(double) * Pt.nnz, cudaMemcpyDeviceToDevice, s));
        PCG_CK(cudaMemcpyAsync(lv.Pt32, pt32, sizeof(float) * Pt.nnz, cudaMemcpyDeviceToDevice, s));
        PCG_CK(cudaMemcpyAsync(out->v, C.v, sizeof(double) * C.nnz, cudaMemcpyDeviceToDevice, s));
        PCG_CK(cudaStreamSynchronize(s));
    }
    release(M, P.rp); release(M, P.ci); release(M, P.v); release(M, p32);
    release(M, Pt.rp); release(M, Pt.ci); release(M, Pt.v); release(M, pt32);
    release(M, C.rp); release(M, C.ci); release(M, C.v);
    if (st) set_error("amg_refresh: the smoothed prolongator or coarse matrix changed pattern");
    return st;
}

}  // namespace pcgamg
