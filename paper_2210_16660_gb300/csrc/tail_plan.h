// Host-side planning of the shared-memory cluster tail (tail.cu): the
// shared-memory layout every CTA uses and each CTA's static data. Plain C++
// (no CUDA), so the layout and the index arithmetic can be checked on the
// host.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <vector>

namespace pcgamg {

constexpr int kMaxTailLevels = 12;
constexpr int kSmemTailRows = 12000;
constexpr uint32_t kNone = 0xffffffffu;

// Per tail level: the rows each CTA owns and the byte offsets of that
// level's arrays in every CTA's shared memory (the same offsets in every
// CTA, so a row another CTA owns is found at the same offset in the owner's
// shared memory).
struct SmemTailLevel {
    int n, rpc;  // rows; rows per CTA (CTA r owns rows r*rpc ..)
    int off_rp, off_col, off_val, off_dinv, off_p, off_agg, off_mp, off_mem;  // static data
    int off_b, off_x, off_t, off_xpre, off_xp;                                // vectors
};
struct SmemTailPlan {
    int nt, ctas, static_bytes, off_ainv, off_bl;
    SmemTailLevel lev[kMaxTailLevels];
};

// A packed reference to a row of a tail level: owning CTA in the top 8 bits,
// row within the owner's block in the low 24.
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t pack(int owner, int local) { return ((uint32_t)owner << 24) | (uint32_t)local; }

// Host-side copies of what one tail level needs.
struct HostLevel {
    int n = 0;
    std::vector<int32_t> rp, ci, agg, rptr, ridx;
    std::vector<double> v, dinv, p;
    std::vector<float> dinv32, p32;
};

inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Shared-memory layout and per-CTA static blob of one precision. Returns
// the per-CTA shared bytes (static + vectors), or 0 if the levels don't fit.
template <typename T>
size_t build_plan(const std::vector<HostLevel> &hl, const std::vector<double> &ainv, int ctas, SmemTailPlan &plan,
                  std::vector<unsigned char> &blob) {
    int nt = (int)hl.size();
    plan.nt = nt;
    plan.ctas = ctas;
    std::vector<int> rpc(nt);
    for (int k = 0; k < nt; k++) {
        int n = hl[k].n;
        rpc[k] = std::max(1, (n + ctas - 1) / ctas);
        plan.lev[k].n = n;
        plan.lev[k].rpc = rpc[k];
    }
    auto owner = [&](int k, int j) { return pack(j / rpc[k], j % rpc[k]); };
    // sizes (max over CTAs) of the per-CTA arrays
    size_t off = 0;
    std::vector<size_t> maxnnz(nt, 0), maxmem(nt, 0);
    for (int k = 0; k + 1 < nt; k++) {  // the coarsest level has no sweeps
        const HostLevel &L = hl[k];
        for (int r = 0; r < ctas; r++) {
            int r0 = std::min(L.n, r * rpc[k]), r1 = std::min(L.n, r0 + rpc[k]);
            maxnnz[k] = std::max(maxnnz[k], (size_t)(L.rp[r1] - L.rp[r0]));
            int c0 = std::min(hl[k + 1].n, r * rpc[k + 1]), c1 = std::min(hl[k + 1].n, c0 + rpc[k + 1]);
            maxmem[k] = std::max(maxmem[k], (size_t)(L.rptr[c1] - L.rptr[c0]));
        }
    }
    for (int k = 0; k < nt; k++) {
        SmemTailLevel &S = plan.lev[k];
        size_t R = (size_t)rpc[k];
        bool sweeps = k + 1 < nt;
        S.off_rp = (int)off; off = align16(off + (sweeps ? (R + 1) * 4 : 0));
        S.off_col = (int)off; off = align16(off + (sweeps ? maxnnz[k] * 4 : 0));
        S.off_val = (int)off; off = align16(off + (sweeps ? maxnnz[k] * sizeof(T) : 0));
        S.off_dinv = (int)off; off = align16(off + R * sizeof(T));
        S.off_p = (int)off; off = align16(off + (sweeps ? R * sizeof(T) : 0));
        S.off_agg = (int)off; off = align16(off + (sweeps ? R * 4 : 0));
        size_t CR = sweeps ? (size_t)rpc[k + 1] : 0;
        S.off_mp = (int)off; off = align16(off + (sweeps ? (CR + 1) * 4 : 0));
        S.off_mem = (int)off; off = align16(off + (sweeps ? maxmem[k] * 4 : 0));
    }
    int nL = hl[nt - 1].n;
    plan.off_ainv = (int)off;
    off = align16(off + (size_t)rpc[nt - 1] * nL * sizeof(double));
    plan.static_bytes = (int)off;
    for (int k = 0; k < nt; k++) {
        SmemTailLevel &S = plan.lev[k];
        size_t R = (size_t)rpc[k];
        S.off_b = (int)off; off = align16(off + R * sizeof(T));
        S.off_x = (int)off; off = align16(off + R * sizeof(T));
        S.off_t = (int)off; off = align16(off + R * sizeof(T));
        S.off_xpre = (int)off; off = align16(off + R * sizeof(T));
        S.off_xp = (int)off; off = align16(off + R * sizeof(T));
    }
    plan.off_bl = (int)off;
    off = align16(off + (size_t)rpc[nt - 1] * sizeof(double));
    size_t total = off;
    // static blob per CTA
    blob.assign((size_t)ctas * plan.static_bytes, 0);
    for (int r = 0; r < ctas; r++) {
        unsigned char *B = blob.data() + (size_t)r * plan.static_bytes;
        for (int k = 0; k < nt; k++) {
            const HostLevel &L = hl[k];
            const SmemTailLevel &S = plan.lev[k];
            int r0 = std::min(L.n, r * rpc[k]), r1 = std::min(L.n, r0 + rpc[k]);
            bool sweeps = k + 1 < nt;
            T *dinv = reinterpret_cast<T *>(B + S.off_dinv);
            for (int i = r0; i < r1; i++) dinv[i - r0] = sizeof(T) == 4 ? (T)L.dinv32[i] : (T)L.dinv[i];
            if (!sweeps) continue;
            int32_t *rp = reinterpret_cast<int32_t *>(B + S.off_rp);
            uint32_t *col = reinterpret_cast<uint32_t *>(B + S.off_col);
            T *val = reinterpret_cast<T *>(B + S.off_val);
            T *p = reinterpret_cast<T *>(B + S.off_p);
            uint32_t *agg = reinterpret_cast<uint32_t *>(B + S.off_agg);
            int base = L.rp[r0];
            for (int i = r0; i <= r1; i++) rp[i - r0] = L.rp[i] - base;
            for (int q = L.rp[r0]; q < L.rp[r1]; q++) {
                col[q - base] = owner(k, L.ci[q]);
                val[q - base] = (T)L.v[q];
            }
            for (int i = r0; i < r1; i++) {
                p[i - r0] = sizeof(T) == 4 ? (T)L.p32[i] : (T)L.p[i];
                agg[i - r0] = L.agg[i] >= 0 ? owner(k + 1, L.agg[i]) : kNone;
            }
            int nc = hl[k + 1].n;
            int c0 = std::min(nc, r * rpc[k + 1]), c1 = std::min(nc, c0 + rpc[k + 1]);
            int32_t *mp = reinterpret_cast<int32_t *>(B + S.off_mp);
            uint32_t *mem = reinterpret_cast<uint32_t *>(B + S.off_mem);
            int mb = L.rptr[c0];
            for (int I = c0; I <= c1; I++) mp[I - c0] = L.rptr[I] - mb;
            for (int q = L.rptr[c0]; q < L.rptr[c1]; q++) mem[q - mb] = owner(k, L.ridx[q]);
        }
        double *a = reinterpret_cast<double *>(B + plan.off_ainv);
        int c0 = std::min(nL, r * rpc[nt - 1]), c1 = std::min(nL, c0 + rpc[nt - 1]);
        for (int i = c0; i < c1; i++)
            for (int j = 0; j < nL; j++) a[(size_t)(i - c0) * nL + j] = ainv[(size_t)i * nL + j];
    }
    return total;
}


}  // namespace pcgamg
