// Host check of the shared-memory cluster tail's plan (tail_plan.h) and of
// the index arithmetic of its kernel: build_plan lays out every CTA's shared
// memory and static blob; this program emulates each phase of the tail on
// per-CTA byte arrays (a read of a row another CTA owns goes to the owner's
// array through the packed reference) and compares the entry level's x with
// the same V-cycle computed level by level on plain arrays. Built by
// tests/test_tail_plan.py (with AddressSanitizer where the compiler has it).
//
// Input file (written by the test): F, L; per tail level n, its CSR, values
// and D^-1, and for all but the coarsest the aggregate map, weights and the
// member lists of its coarse rows; then the dense coarsest inverse.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

#include "../paper_2210_16660_gb300/csrc/tail_plan.h"

using namespace pcgamg;

template <class X>
static std::vector<X> read_vec(FILE *f) {
    long long n = 0;
    if (fread(&n, 8, 1, f) != 1 || n < 0) { fprintf(stderr, "bad input\n"); exit(2); }
    std::vector<X> v((size_t)n);
    if (n && fread(v.data(), sizeof(X), (size_t)n, f) != (size_t)n) { fprintf(stderr, "short input\n"); exit(2); }
    return v;
}

template <typename T>
static T *arr(std::vector<unsigned char> &cta, int off) { return reinterpret_cast<T *>(cta.data() + off); }

template <typename T>
static int check(const std::vector<HostLevel> &hl, const std::vector<double> &ainv, int ctas) {
    SmemTailPlan plan = {};
    std::vector<unsigned char> blob;
    const size_t bytes = build_plan<T>(hl, ainv, ctas, plan, blob);
    const int nt = plan.nt, nL = hl[nt - 1].n;
    if (blob.size() != (size_t)ctas * plan.static_bytes || bytes < (size_t)plan.static_bytes) {
        printf("layout sizes inconsistent\n");
        return 1;
    }
    std::mt19937_64 rng(7);
    std::uniform_real_distribution<double> U(-1, 1);
    std::vector<T> bF(hl[0].n), xpreF(hl[0].n);
    for (auto &v : bF) v = (T)U(rng);
    for (auto &v : xpreF) v = (T)U(rng);

    // shared memory of every CTA: its static blob, then the entry rows
    std::vector<std::vector<unsigned char>> sm(ctas, std::vector<unsigned char>(bytes, 0xCD));
    for (int r = 0; r < ctas; r++) {
        memcpy(sm[r].data(), blob.data() + (size_t)r * plan.static_bytes, plan.static_bytes);
        const SmemTailLevel &F = plan.lev[0];
        int r0 = r * F.rpc, r1 = std::min(F.n, r0 + F.rpc);
        for (int i = r0; i < r1; i++) {
            arr<T>(sm[r], F.off_b)[i - r0] = bF[i];
            arr<T>(sm[r], F.off_xpre)[i - r0] = xpreF[i];
        }
    }
    int bad_ref = 0;
    auto remote = [&](int off, uint32_t ref) -> T & {
        int o = (int)(ref >> 24), l = (int)(ref & 0xffffffu);
        if (o >= ctas) { bad_ref++; o = 0; l = 0; }
        return arr<T>(sm[o], off)[l];
    };
    auto remote_d = [&](int off, uint32_t ref) -> double & {
        int o = (int)(ref >> 24), l = (int)(ref & 0xffffffu);
        if (o >= ctas) { bad_ref++; o = 0; l = 0; }
        return arr<double>(sm[o], off)[l];
    };
    // down: pre-smoothed residual, restriction
    for (int k = 0; k + 1 < nt; k++) {
        const SmemTailLevel &Lv = plan.lev[k], &Cv = plan.lev[k + 1];
        for (int r = 0; r < ctas; r++) {
            int rows = std::min(Lv.rpc, Lv.n - r * Lv.rpc);
            const int32_t *rp = arr<int32_t>(sm[r], Lv.off_rp);
            const uint32_t *cp = arr<uint32_t>(sm[r], Lv.off_col);
            const T *val = arr<T>(sm[r], Lv.off_val), *p = arr<T>(sm[r], Lv.off_p);
            T *b = arr<T>(sm[r], Lv.off_b), *t = arr<T>(sm[r], Lv.off_t);
            for (int i = 0; i < rows; i++) {
                T acc = 0;
                for (int q = rp[i]; q < rp[i + 1]; q++) acc += val[q] * remote(Lv.off_xpre, cp[q]);
                t[i] = p[i] * (b[i] - acc);
            }
        }
        const bool last = k + 2 == nt;
        for (int r = 0; r < ctas; r++) {
            int crows = std::min(Cv.rpc, Cv.n - r * Cv.rpc);
            const int32_t *mp = arr<int32_t>(sm[r], Lv.off_mp);
            const uint32_t *mem = arr<uint32_t>(sm[r], Lv.off_mem);
            for (int I = 0; I < crows; I++) {
                T s = 0;
                for (int q = mp[I]; q < mp[I + 1]; q++) s += remote(Lv.off_t, mem[q]);
                if (last) {
                    arr<double>(sm[r], plan.off_bl)[I] = (double)s;
                } else {
                    arr<T>(sm[r], Cv.off_b)[I] = s;
                    arr<T>(sm[r], Cv.off_xpre)[I] = arr<T>(sm[r], Cv.off_dinv)[I] * s;
                }
            }
        }
    }
    // coarsest: lane-strided partial sums and the shuffle tree of the kernel
    {
        const SmemTailLevel &C = plan.lev[nt - 1];
        for (int r = 0; r < ctas; r++) {
            int rows = std::min(C.rpc, C.n - r * C.rpc);
            const double *ai = arr<double>(sm[r], plan.off_ainv);
            for (int row = 0; row < rows; row++) {
                double part[32];
                for (int lane = 0; lane < 32; lane++) {
                    double s = 0;
                    for (int j = lane; j < C.n; j += 32)
                        s += ai[(size_t)row * C.n + j] * remote_d(plan.off_bl, pack(j / C.rpc, j % C.rpc));
                    part[lane] = s;
                }
                for (int o = 16; o > 0; o >>= 1)
                    for (int lane = 0; lane < o; lane++) part[lane] += part[lane + o];
                arr<T>(sm[r], C.off_x)[row] = (T)part[0];
            }
        }
    }
    // up: prolongation, post-smoothing
    for (int k = nt - 2; k >= 0; k--) {
        const SmemTailLevel &Lv = plan.lev[k], &Cv = plan.lev[k + 1];
        for (int r = 0; r < ctas; r++) {
            int rows = std::min(Lv.rpc, Lv.n - r * Lv.rpc);
            const uint32_t *agg = arr<uint32_t>(sm[r], Lv.off_agg);
            const T *p = arr<T>(sm[r], Lv.off_p);
            for (int i = 0; i < rows; i++) {
                T x = arr<T>(sm[r], Lv.off_xpre)[i];
                if (agg[i] != kNone) x += p[i] * remote(Cv.off_x, agg[i]);
                arr<T>(sm[r], Lv.off_xp)[i] = x;
            }
        }
        for (int r = 0; r < ctas; r++) {
            int rows = std::min(Lv.rpc, Lv.n - r * Lv.rpc);
            const int32_t *rp = arr<int32_t>(sm[r], Lv.off_rp);
            const uint32_t *cp = arr<uint32_t>(sm[r], Lv.off_col);
            const T *val = arr<T>(sm[r], Lv.off_val), *dinv = arr<T>(sm[r], Lv.off_dinv);
            for (int i = 0; i < rows; i++) {
                T acc = 0;
                for (int q = rp[i]; q < rp[i + 1]; q++) acc += val[q] * remote(Lv.off_xp, cp[q]);
                arr<T>(sm[r], Lv.off_x)[i] = arr<T>(sm[r], Lv.off_xp)[i] + dinv[i] * (arr<T>(sm[r], Lv.off_b)[i] - acc);
            }
        }
    }
    std::vector<T> xE(hl[0].n);
    {
        const SmemTailLevel &F = plan.lev[0];
        for (int r = 0; r < ctas; r++) {
            int r0 = r * F.rpc, r1 = std::min(F.n, r0 + F.rpc);
            for (int i = r0; i < r1; i++) xE[i] = arr<T>(sm[r], F.off_x)[i - r0];
        }
    }

    // the same V-cycle, level by level on plain arrays
    std::vector<std::vector<T>> b(nt), xpre(nt), t(nt), xp(nt), x(nt);
    for (int k = 0; k < nt; k++) {
        size_t n = (size_t)hl[k].n;
        b[k].assign(n, 0); xpre[k].assign(n, 0); t[k].assign(n, 0); xp[k].assign(n, 0); x[k].assign(n, 0);
    }
    b[0] = bF;
    xpre[0] = xpreF;
    std::vector<double> bL(nL);
    auto dv = [&](const HostLevel &L, int i) { return sizeof(T) == 4 ? (T)L.dinv32[i] : (T)L.dinv[i]; };
    auto pw = [&](const HostLevel &L, int i) { return sizeof(T) == 4 ? (T)L.p32[i] : (T)L.p[i]; };
    for (int k = 0; k + 1 < nt; k++) {
        const HostLevel &L = hl[k];
        for (int i = 0; i < L.n; i++) {
            T acc = 0;
            for (int q = L.rp[i]; q < L.rp[i + 1]; q++) acc += (T)L.v[q] * xpre[k][L.ci[q]];
            t[k][i] = pw(L, i) * (b[k][i] - acc);
        }
        for (int I = 0; I < hl[k + 1].n; I++) {
            T s = 0;
            for (int q = L.rptr[I]; q < L.rptr[I + 1]; q++) s += t[k][L.ridx[q]];
            if (k + 2 == nt) bL[I] = (double)s;
            else { b[k + 1][I] = s; xpre[k + 1][I] = dv(hl[k + 1], I) * s; }
        }
    }
    for (int row = 0; row < nL; row++) {
        double part[32];
        for (int lane = 0; lane < 32; lane++) {
            double s = 0;
            for (int j = lane; j < nL; j += 32) s += ainv[(size_t)row * nL + j] * bL[j];
            part[lane] = s;
        }
        for (int o = 16; o > 0; o >>= 1)
            for (int lane = 0; lane < o; lane++) part[lane] += part[lane + o];
        x[nt - 1][row] = (T)part[0];
    }
    for (int k = nt - 2; k >= 0; k--) {
        const HostLevel &L = hl[k];
        for (int i = 0; i < L.n; i++) {
            T v = xpre[k][i];
            if (L.agg[i] >= 0) v += pw(L, i) * x[k + 1][L.agg[i]];
            xp[k][i] = v;
        }
        for (int i = 0; i < L.n; i++) {
            T acc = 0;
            for (int q = L.rp[i]; q < L.rp[i + 1]; q++) acc += (T)L.v[q] * xp[k][L.ci[q]];
            x[k][i] = xp[k][i] + dv(L, i) * (b[k][i] - acc);
        }
    }
    int bad = 0;
    for (int i = 0; i < hl[0].n; i++)
        if (memcmp(&xE[i], &x[0][i], sizeof(T)) != 0) bad++;
    printf("T=%zu ctas=%d levels=%d static=%d shared=%zu mismatches=%d bad_refs=%d rows=%d\n", sizeof(T), ctas, nt,
           plan.static_bytes, bytes, bad, bad_ref, hl[0].n);
    return bad + bad_ref;
}

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int F = 0, L = 0;
    if (fread(&F, 4, 1, f) != 1 || fread(&L, 4, 1, f) != 1 || L <= F) return 2;
    std::vector<HostLevel> hl(L - F + 1);
    for (int k = 0; k <= L - F; k++) {
        HostLevel &H = hl[k];
        if (fread(&H.n, 4, 1, f) != 1) return 2;
        H.rp = read_vec<int32_t>(f);
        H.ci = read_vec<int32_t>(f);
        H.v = read_vec<double>(f);
        H.dinv = read_vec<double>(f);
        H.dinv32.resize(H.n);
        for (int i = 0; i < H.n; i++) H.dinv32[i] = (float)H.dinv[i];
        if (k < L - F) {
            H.agg = read_vec<int32_t>(f);
            H.p = read_vec<double>(f);
            H.rptr = read_vec<int32_t>(f);
            H.ridx = read_vec<int32_t>(f);
            H.p32.resize(H.n);
            for (int i = 0; i < H.n; i++) H.p32[i] = (float)H.p[i];
        } else {
            H.rp.clear(); H.ci.clear(); H.v.clear();   // the coarsest level has no sweeps
        }
    }
    const int nL = hl.back().n;
    std::vector<double> ainv((size_t)nL * nL);
    if (fread(ainv.data(), 8, ainv.size(), f) != ainv.size()) return 2;
    fclose(f);
    int bad = 0;
    for (int c : {16, 8, 5}) {
        bad += check<float>(hl, ainv, c);
        bad += check<double>(hl, ainv, c);
    }
    return bad != 0;
}
