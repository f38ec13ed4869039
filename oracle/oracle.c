/*
 * CPU oracle for PCG preconditioned by one aggregation-AMG V-cycle
 * (arxiv 2210.16660, Sec. 3.1), written in plain C99, float64 throughout
 * except the deliberately single-precision V-cycle variant.
 *
 * TEST INFRASTRUCTURE ONLY. This code exists to check the CUDA library; it is
 * not part of the product path. Only the test suite, the package smoke check
 * and the CPU-baseline leg of the benchmark load it. It shares no code, header
 * or table with the CUDA sources.
 *
 * Everything is sequential and in the order the method states it. Where the
 * paper leaves a choice open, the reading taken is stated at the function.
 * Compile with -ffp-contract=off: no multiply-add contraction, so every
 * floating-point operation rounds as written (the GPU setup kernels use the
 * same explicit roundings, which keeps the integer aggregates comparable
 * bit for bit).
 *
 * Status codes: 0 ok, 1 bad argument, 2 out of memory, 3 breakdown
 * (rho <= 0 or p'Ap <= 0: not SPD), 4 no convergence within maxit,
 * 5 NaN/Inf met, 8 coarsening stalled above the dense-solve limit (only when
 * the dense coarsest solver is requested).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_OOM 2
#define OR_ERR_BREAKDOWN 3
#define OR_ERR_NOCONV 4
#define OR_ERR_NAN 5
#define OR_ERR_COARSE 8

#define OR_MAX_LEVELS 40
#define OR_MAX_PASS 8
#define OR_DENSE_MAX 4096

typedef struct {
    int n;
    int64_t nnz;
    int32_t *rp, *ci;
    double *v;
} csr_t;

typedef struct {
    csr_t A;            /* A_l (owned, except level 0 which is a copy too) */
    double *dinv;       /* 1 / sum_j |a_ij|                                 */
    double *w;          /* the vector w of this level (w = 1 on level 0)    */
    int32_t *agg;       /* composed aggregate map level l -> l+1, -1 = none */
    double *p;          /* composed tentative-prolongator weight per row    */
    int npass;          /* passes run on this level                         */
    int32_t *pass_agg[OR_MAX_PASS];
    int pass_n[OR_MAX_PASS + 1];
    /* single-precision copies for the FP32 V-cycle */
    float *v32, *dinv32, *p32;
    /* smoothed aggregation: the explicit prolongator P (n_l x n_{l+1}) and
     * its float32 values; empty (P.rp == NULL) for the tentative one */
    csr_t P;
    float *P32;
} level_t;

typedef struct {
    int nlev;           /* levels 0..nlev-1; nlev-1 is the coarsest */
    level_t lev[OR_MAX_LEVELS];
    double *L;          /* dense Cholesky factor of the coarsest A (row-major, lower) */
    int nL;
    /* smoother: nu = 0 is the one-sweep l1-Jacobi of the setup; otherwise nu
     * sweeps of the l1 hybrid Gauss-Seidel method over nblocks row blocks per
     * level (or_set_smoother) */
    int nu, nblocks;
    int smoothed;       /* 1: P = (I - omega D^-1 A) P_hat on every level */
    /* coarsest solver: csolver = 0 dense Cholesky (L above), 1 flexible CG
     * preconditioned by block-Jacobi with ILU(1) blocks of cb rows, stopped
     * at ||r|| <= ctol ||b|| or after cmaxit iterations */
    int csolver, cb, cmaxit;
    double ctol;
    int32_t *frp, *fci, *fdg;   /* ILU(1) factors of the blocks: row i holds its
                                   in-block entries of L (unit diagonal not
                                   stored) and U, columns ascending; fdg[i] is
                                   the position of u_ii */
    double *fv;
    unsigned char *flev;        /* level of fill of each kept entry (0 or 1) */
    int64_t *cstat;             /* calls, inner iterations in total, last count */
} hier_t;

/* Options of or_setup_cfg. csolver: 0 = dense when the coarsest level has at
 * most OR_DENSE_MAX rows, else iterative; 1 = dense (OR_ERR_COARSE above the
 * limit); 2 = iterative. */
typedef struct {
    int coarse_max, n_pass, max_levels, smoothed;
    int csolver, cb, cmaxit;
    double ctol;
} or_cfg_t;

/* ---------------------------------------------------------------- helpers */

static void csr_free(csr_t *a) {
    free(a->rp); free(a->ci); free(a->v);
    a->rp = NULL; a->ci = NULL; a->v = NULL;
}

/* Structural check: sorted, in-range columns; positive diagonal present. */
static int csr_check(int n, const int32_t *rp, const int32_t *ci, const double *v) {
    if (n < 0 || rp[0] != 0) return OR_ERR_ARG;
    for (int i = 0; i < n; i++) {
        int has_diag = 0;
        if (rp[i + 1] < rp[i]) return OR_ERR_ARG;
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            if (ci[k] < 0 || ci[k] >= n) return OR_ERR_ARG;
            if (k > rp[i] && ci[k] <= ci[k - 1]) return OR_ERR_ARG;
            if (ci[k] == i) { has_diag = 1; if (!(v[k] > 0.0)) return OR_ERR_ARG; }
        }
        if (!has_diag) return OR_ERR_ARG;
    }
    return OR_OK;
}

static double diag_of(const csr_t *a, int i) {
    for (int32_t k = a->rp[i]; k < a->rp[i + 1]; k++)
        if (a->ci[k] == i) return a->v[k];
    return 0.0;
}

/* y = A x, each row summed left to right over its stored entries. */
void or_spmv(int n, const int32_t *rp, const int32_t *ci, const double *v,
             const double *x, double *y) {
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) s += v[k] * x[ci[k]];
        y[i] = s;
    }
}

static double dot(int n, const double *a, const double *b) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------ l1 diagonal (smoother)
 * The smoother replacing the paper's hybrid Gauss-Seidel (Sec. 3.1, the l1
 * smoother family it cites): M = D_l1 with d_i = sum_j |a_ij| (a_ii included).
 */
void or_l1_diag(int n, const int32_t *rp, const int32_t *ci, const double *v, double *d) {
    (void)ci;
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) s += fabs(v[k]);
        d[i] = s;
    }
}

/* ------------------------------------- hybrid Gauss-Seidel smoother (Sec. 3.1)
 * The paper smooths with nu = 4 sweeps of hybrid forward/backward
 * Gauss-Seidel: block Jacobi over the row blocks of the parallel distribution,
 * each block solved by one forward (pre-smoothing) or backward (post-
 * smoothing) Gauss-Seidel pass, M_pp = omega (L_pp + D_pp). Reading: the l1
 * form of the same method (the l1 family the paper cites), which needs no
 * damping: omega = 1 and D_pp augmented by the off-block row sums,
 * d_i = a_ii + sum_{j outside i's block} |a_ij|. The blocks are nblocks
 * contiguous row ranges per level ("processes"), ceil(n_l / nblocks) rows
 * each, so they shrink on coarser levels as a fixed distribution's do. One
 * row per block is the l1-Jacobi smoother.
 */
static int gs_rows(const hier_t *h, int n) {
    if (h->nblocks <= 0) return 1;
    int nb = (int)(((int64_t)n + h->nblocks - 1) / h->nblocks);
    return nb < 1 ? 1 : nb;
}

/* d_i summed in storage order; in-block off-diagonal entries are skipped */
static void hybrid_l1(const csr_t *a, int nb, double *dinv, float *dinv32) {
    for (int i = 0; i < a->n; i++) {
        int lo = (i / nb) * nb, hi = lo + nb;
        double s = 0.0;
        for (int32_t k = a->rp[i]; k < a->rp[i + 1]; k++) {
            int j = a->ci[k];
            if (j == i || j < lo || j >= hi) s += fabs(a->v[k]);
        }
        dinv[i] = 1.0 / s;
        dinv32[i] = (float)dinv[i];
    }
}

/* One sweep x_new = x_old + M^{-1} (b - A x_old), M = blockdiag(L_pp + D_l1)
 * (forward) or its transpose (backward), rows of a block in increasing
 * (forward) or decreasing (backward) order; within a block the updated
 * values are used, outside it the values of x_old (xo = NULL: x_old = 0). */
static void sweep64(const csr_t *a, const double *dinv, int nb, const double *b, const double *xo, double *xn,
                    int fwd) {
    int n = a->n;
    for (int lo = 0; lo < n; lo += nb) {
        int hi = lo + nb < n ? lo + nb : n;
        for (int r = lo; r < hi; r++) xn[r] = xo ? xo[r] : 0.0;
        for (int q = 0; q < hi - lo; q++) {
            int r = fwd ? lo + q : hi - 1 - q;
            double acc = 0.0;
            for (int32_t k = a->rp[r]; k < a->rp[r + 1]; k++) {
                int j = a->ci[k];
                double xj = (j >= lo && j < hi) ? xn[j] : (xo ? xo[j] : 0.0);
                acc += a->v[k] * xj;
            }
            xn[r] = xo ? xn[r] + dinv[r] * (b[r] - acc) : dinv[r] * (b[r] - acc);
        }
    }
}

static void sweep32(const csr_t *a, const float *v32, const float *dinv, int nb, const float *b, const float *xo,
                    float *xn, int fwd) {
    int n = a->n;
    for (int lo = 0; lo < n; lo += nb) {
        int hi = lo + nb < n ? lo + nb : n;
        for (int r = lo; r < hi; r++) xn[r] = xo ? xo[r] : 0.0f;
        for (int q = 0; q < hi - lo; q++) {
            int r = fwd ? lo + q : hi - 1 - q;
            float acc = 0.0f;
            for (int32_t k = a->rp[r]; k < a->rp[r + 1]; k++) {
                int j = a->ci[k];
                float xj = (j >= lo && j < hi) ? xn[j] : (xo ? xo[j] : 0.0f);
                acc += v32[k] * xj;
            }
            xn[r] = xo ? xn[r] + dinv[r] * (b[r] - acc) : dinv[r] * (b[r] - acc);
        }
    }
}

/* --------------------------------------------------------- edge weights
 * Eq. (weights): c_ij = 1 - 2 a_ij w_i w_j / (a_ii w_i^2 + a_jj w_j^2),
 * evaluated left to right with each operation rounded.
 */
double or_weight(double aij, double aii, double ajj, double wi, double wj) {
    double num = ((2.0 * aij) * wi) * wj;
    double den = (aii * wi) * wi + (ajj * wj) * wj;
    return 1.0 - num / den;
}

/* ------------------------------------------------------------- matching
 * Eq. (approximatematch): an approximate maximum-product matching on the
 * adjacency graph of A with edge weights c_ij.
 *
 * Reading: the paper computes it with a half-approximate maximum-weight
 * matching (MatchBox-P). Taken here as the greedy matching under a strict
 * total order: candidate edges are the stored pairs i < j with c_ij > 1 (an
 * edge with c_ij <= 1 can only lower or keep the product, so a maximum-product
 * matching never needs it); they are scanned by decreasing c_ij, ties broken
 * by increasing (i, j); an edge is taken when both ends are still free. Greedy
 * on log c_ij is a half-approximation of the maximum log-weight matching.
 * mate[i] = partner or -1. Returns the number of matched pairs.
 */
typedef struct { double c; int32_t i, j; } edge_t;

static int edge_cmp(const void *pa, const void *pb) {
    const edge_t *a = (const edge_t *)pa, *b = (const edge_t *)pb;
    if (a->c > b->c) return -1;
    if (a->c < b->c) return 1;
    if (a->i != b->i) return a->i < b->i ? -1 : 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    return 0;
}

int or_match(int n, const int32_t *rp, const int32_t *ci, const double *v,
             const double *w, int32_t *mate) {
    csr_t a = {n, rp[n], (int32_t *)rp, (int32_t *)ci, (double *)v};
    int64_t ne = 0;
    for (int i = 0; i < n; i++)
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) if (ci[k] > i) ne++;
    edge_t *e = (edge_t *)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(edge_t));
    double *dg = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!e || !dg) { free(e); free(dg); return -OR_ERR_OOM; }
    for (int i = 0; i < n; i++) dg[i] = diag_of(&a, i);
    int64_t m = 0;
    for (int i = 0; i < n; i++) {
        for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
            int j = ci[k];
            if (j <= i) continue;
            double c = or_weight(v[k], dg[i], dg[j], w[i], w[j]);
            if (c > 1.0) { e[m].c = c; e[m].i = i; e[m].j = j; m++; }
        }
    }
    qsort(e, (size_t)m, sizeof(edge_t), edge_cmp);
    for (int i = 0; i < n; i++) mate[i] = -1;
    int pairs = 0;
    for (int64_t t = 0; t < m; t++) {
        if (mate[e[t].i] < 0 && mate[e[t].j] < 0) {
            mate[e[t].i] = e[t].j;
            mate[e[t].j] = e[t].i;
            pairs++;
        }
    }
    free(e); free(dg);
    return pairs;
}

/* ----------------------------------------------------------- aggregates
 * Sec. 3.1 after Eq. (approximatematch), and Eq. (prolongator): aggregates are
 * the matched pairs plus a singleton for every unmatched vertex; the tentative
 * prolongator holds w restricted to each pair, normalised (w_e), and
 * w_s/|w_s| for a singleton; the coarse vector is w_c = ||w restricted to G||.
 *
 * Reading: a row with no nonzero off-diagonal entry (a Dirichlet row) is
 * decoupled from the rest; it is left out of the coarse space (agg = -1,
 * p = 0) since the smoother solves it exactly. Coarse indices are handed out
 * scanning i upward: a singleton, or the smaller end of a pair, takes the next
 * index. Returns n_c.
 */
int or_aggregate(int n, const int32_t *rp, const int32_t *ci, const double *v,
                 const int32_t *mate, const double *w,
                 int32_t *agg, double *p, double *wc) {
    int nc = 0;
    for (int i = 0; i < n; i++) agg[i] = -2;
    for (int i = 0; i < n; i++) {
        if (agg[i] != -2) continue;           /* larger end of a pair, done */
        int isolated = 1;
        for (int32_t k = rp[i]; k < rp[i + 1]; k++)
            if (ci[k] != i && v[k] != 0.0) { isolated = 0; break; }
        int j = mate[i];
        if (j >= 0) {
            /* pair (i, j), i < j: w_e = (w_i, w_j) / ||(w_i, w_j)|| */
            double nrm = sqrt(w[i] * w[i] + w[j] * w[j]);
            agg[i] = nc; agg[j] = nc;
            p[i] = w[i] / nrm; p[j] = w[j] / nrm;
            wc[nc] = nrm;
            nc++;
        } else if (isolated) {
            agg[i] = -1; p[i] = 0.0;
        } else {
            agg[i] = nc;
            p[i] = w[i] / fabs(w[i]);
            wc[nc] = fabs(w[i]);
            nc++;
        }
    }
    return nc;
}

/* --------------------------------------------------------- Galerkin RAP
 * A_c = P^T A P with P the tentative prolongator (one weight p_i per row,
 * column agg(i)), Sec. 3.1 (triple-matrix Galerkin product).
 *
 * Reading on rounding (the paper fixes none): each fine entry contributes
 * t_ij = a_ij * (p_i * p_j); the contributions to coarse entry (I, J) are
 * added in increasing order of (min(i,j), max(i,j)). Both rules are
 * symmetric in (i, j), so a bitwise-symmetric A gives a bitwise-symmetric A_c.
 * The pattern keeps every (I, J) that receives a contribution, exact zeros
 * included; columns sorted.
 */
typedef struct { int32_t J, kmin, kmax; double t; } term_t;

static int term_cmp(const void *pa, const void *pb) {
    const term_t *a = (const term_t *)pa, *b = (const term_t *)pb;
    if (a->J != b->J) return a->J < b->J ? -1 : 1;
    if (a->kmin != b->kmin) return a->kmin < b->kmin ? -1 : 1;
    if (a->kmax != b->kmax) return a->kmax < b->kmax ? -1 : 1;
    return 0;
}

static int rap(const csr_t *a, const int32_t *agg, const double *p, int nc, csr_t *out) {
    int n = a->n;
    /* members of each coarse row, increasing fine index */
    int32_t *cnt = (int32_t *)calloc((size_t)nc + 1, sizeof(int32_t));
    int32_t *mem = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!cnt || !mem) { free(cnt); free(mem); return OR_ERR_OOM; }
    for (int i = 0; i < n; i++) if (agg[i] >= 0) cnt[agg[i] + 1]++;
    for (int I = 0; I < nc; I++) cnt[I + 1] += cnt[I];
    int32_t *fill = (int32_t *)malloc(((size_t)nc + 1) * sizeof(int32_t));
    if (!fill) { free(cnt); free(mem); return OR_ERR_OOM; }
    memcpy(fill, cnt, ((size_t)nc + 1) * sizeof(int32_t));
    for (int i = 0; i < n; i++) if (agg[i] >= 0) mem[fill[agg[i]]++] = i;
    free(fill);

    int64_t cap = a->nnz > 16 ? a->nnz : 16;
    out->n = nc;
    out->rp = (int32_t *)malloc(((size_t)nc + 1) * sizeof(int32_t));
    out->ci = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    out->v = (double *)malloc((size_t)cap * sizeof(double));
    int64_t tcap = 64;
    term_t *tm = (term_t *)malloc((size_t)tcap * sizeof(term_t));
    if (!out->rp || !out->ci || !out->v || !tm) {
        free(cnt); free(mem); free(tm); csr_free(out); return OR_ERR_OOM;
    }
    int64_t nz = 0;
    out->rp[0] = 0;
    for (int I = 0; I < nc; I++) {
        int64_t nt = 0;
        for (int32_t m = cnt[I]; m < cnt[I + 1]; m++) {
            int i = mem[m];
            for (int32_t k = a->rp[i]; k < a->rp[i + 1]; k++) {
                int j = a->ci[k];
                if (agg[j] < 0) continue;
                if (nt == tcap) {
                    tcap *= 2;
                    term_t *t2 = (term_t *)realloc(tm, (size_t)tcap * sizeof(term_t));
                    if (!t2) { free(cnt); free(mem); free(tm); csr_free(out); return OR_ERR_OOM; }
                    tm = t2;
                }
                tm[nt].J = agg[j];
                tm[nt].kmin = i < j ? i : j;
                tm[nt].kmax = i < j ? j : i;
                tm[nt].t = a->v[k] * (p[i] * p[j]);
                nt++;
            }
        }
        qsort(tm, (size_t)nt, sizeof(term_t), term_cmp);
        for (int64_t t = 0; t < nt; t++) {
            if (t == 0 || tm[t].J != tm[t - 1].J) {
                if (nz == cap) {
                    cap *= 2;
                    int32_t *c2 = (int32_t *)realloc(out->ci, (size_t)cap * sizeof(int32_t));
                    if (c2) out->ci = c2;
                    double *v2 = (double *)realloc(out->v, (size_t)cap * sizeof(double));
                    if (v2) out->v = v2;
                    if (!c2 || !v2) { free(cnt); free(mem); free(tm); csr_free(out); return OR_ERR_OOM; }
                }
                out->ci[nz] = tm[t].J;
                out->v[nz] = tm[t].t;
                nz++;
            } else {
                out->v[nz - 1] = out->v[nz - 1] + tm[t].t;
            }
        }
        if (nz >= ((int64_t)1 << 31)) { free(cnt); free(mem); free(tm); csr_free(out); return OR_ERR_OOM; }
        out->rp[I + 1] = (int32_t)nz;
    }
    out->nnz = nz;
    free(cnt); free(mem); free(tm);
    return OR_OK;
}

/* Galerkin product on caller buffers: first call with ci_c == NULL to get
 * the number of coarse entries in *nnz_c, then with buffers of that size. */
int or_rap(int n, const int32_t *rp, const int32_t *ci, const double *v,
           const int32_t *agg, const double *p, int nc,
           int64_t *nnz_c, int32_t *rp_c, int32_t *ci_c, double *v_c) {
    csr_t a = {n, rp[n], (int32_t *)rp, (int32_t *)ci, (double *)v};
    csr_t c = {0, 0, NULL, NULL, NULL};
    int st = rap(&a, agg, p, nc, &c);
    if (st) return st;
    *nnz_c = c.nnz;
    if (ci_c) {
        memcpy(rp_c, c.rp, ((size_t)nc + 1) * sizeof(int32_t));
        memcpy(ci_c, c.ci, (size_t)c.nnz * sizeof(int32_t));
        memcpy(v_c, c.v, (size_t)c.nnz * sizeof(double));
    }
    csr_free(&c);
    return OR_OK;
}

/* ------------------------------------------------------- dense Cholesky
 * Direct coarsest solve B_L = A_L^{-1} (Sec. 3.1 below Eq. (multiplicative
 * composition) allows a direct solution). Plain column Cholesky A = L L^T,
 * row-major, lower triangle of L used. Returns 3 when A is not SPD.
 */
int or_chol(int n, const double *A, double *L) {
    memset(L, 0, (size_t)n * (size_t)n * sizeof(double));
    for (int j = 0; j < n; j++) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; k++) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) return OR_ERR_BREAKDOWN;
        double ljj = sqrt(s);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; i++) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; k++) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / ljj;
        }
    }
    return OR_OK;
}

void or_chol_solve(int n, const double *L, const double *b, double *x) {
    for (int i = 0; i < n; i++) {            /* L y = b */
        double s = b[i];
        for (int k = 0; k < i; k++) s -= L[(size_t)i * n + k] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {       /* L^T x = y */
        double s = x[i];
        for (int k = i + 1; k < n; k++) s -= L[(size_t)k * n + i] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
}

/* ------------------------------------------- iterative coarsest solver
 * Sec. 3.1, coarsest solver: flexible CG preconditioned by block-Jacobi,
 * each block solved approximately by an incomplete LU factorization with one
 * level of fill-in, ILU(1); the iteration stops once the residual has fallen
 * by three orders of magnitude or after 30 iterations.
 *
 * Readings: a block is a contiguous range of cb rows of the coarsest matrix
 * (the last one ragged), the rows one parallel worker owns, as the paper's
 * blocks are the rows one process owns; its matrix is A restricted to the
 * block's rows and columns. ILU(1) is the level-of-fill ILU(p) with p = 1 in
 * row (IKJ) order: stored entries have level 0; row i is eliminated with the
 * earlier rows k of its block in increasing k, using only entries (i,k) of
 * level <= 1: l_ik = a_ik / u_kk, then for every kept upper entry u_kj of
 * row k, a_ij -= l_ik u_kj and lev_ij = min(lev_ij, lev_ik + lev_kj + 1);
 * row i keeps its entries of level <= 1. A pivot u_ii that is not a positive
 * finite number is a breakdown (status 3). The solve starts from x = 0 and
 * stops when ||r_k|| <= ctol ||b|| (ctol = 1e-3) or after cmaxit (30)
 * iterations; its recurrence is the FCG(1) of the outer loop. An r.z or
 * p.Ap that is not positive ends it with the current x.
 */
static int ilu1_build(hier_t *h) {
    const csr_t *a = &h->lev[h->nlev - 1].A;
    int n = a->n, cb = h->cb;
    if (cb < 1) return OR_ERR_ARG;
    int64_t cap = (int64_t)n * (cb < n ? cb : n);
    free(h->frp); free(h->fci); free(h->fdg); free(h->fv); free(h->flev);
    h->frp = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    h->fdg = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    h->fci = (int32_t *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
    h->fv = (double *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(double));
    h->flev = (unsigned char *)malloc((size_t)(cap > 0 ? cap : 1));
    double *wv = (double *)malloc((size_t)cb * sizeof(double));
    int *wl = (int *)malloc((size_t)cb * sizeof(int));
    if (!h->frp || !h->fdg || !h->fci || !h->fv || !h->flev || !wv || !wl) {
        free(wv); free(wl);
        return OR_ERR_OOM;
    }
    const int absent = 1 << 20;
    int32_t cnt = 0;
    int st = OR_OK;
    h->frp[0] = 0;
    for (int s = 0; s < n && !st; s += cb) {
        int e = s + cb < n ? s + cb : n, m = e - s;
        for (int i = s; i < e; i++) {
            for (int j = 0; j < m; j++) { wv[j] = 0.0; wl[j] = absent; }
            for (int32_t q = a->rp[i]; q < a->rp[i + 1]; q++) {
                int j = a->ci[q];
                if (j >= s && j < e) { wv[j - s] = a->v[q]; wl[j - s] = 0; }
            }
            for (int k = s; k < i; k++) {
                if (wl[k - s] > 1) continue;
                double lik = wv[k - s] / h->fv[h->fdg[k]];
                wv[k - s] = lik;
                for (int32_t q = h->fdg[k] + 1; q < h->frp[k + 1]; q++) {
                    int j = h->fci[q] - s;
                    wv[j] = wv[j] - lik * h->fv[q];
                    int nl = wl[k - s] + (int)h->flev[q] + 1;
                    if (nl < wl[j]) wl[j] = nl;
                }
            }
            for (int j = 0; j < m; j++) {
                if (wl[j] > 1) continue;
                if (s + j == i) h->fdg[i] = cnt;
                h->fci[cnt] = s + j;
                h->fv[cnt] = wv[j];
                h->flev[cnt] = (unsigned char)wl[j];
                cnt++;
            }
            h->frp[i + 1] = cnt;
            double piv = h->fv[h->fdg[i]];
            if (!(piv > 0.0) || !isfinite(piv)) { st = OR_ERR_BREAKDOWN; break; }
        }
    }
    free(wv); free(wl);
    return st;
}

/* z = M^{-1} r, M = blockdiag(L_b U_b): per block, L y = r (forward, the
 * row's lower entries in increasing column order), then U z = y (backward,
 * rows from the last, the row's upper entries in decreasing column order,
 * then the division by u_ii). */
static void bj_apply(const hier_t *h, const double *r, double *z) {
    int n = h->lev[h->nlev - 1].A.n, cb = h->cb;
    for (int s = 0; s < n; s += cb) {
        int e = s + cb < n ? s + cb : n;
        for (int i = s; i < e; i++) {
            double acc = r[i];
            for (int32_t q = h->frp[i]; q < h->fdg[i]; q++) acc = acc - h->fv[q] * z[h->fci[q]];
            z[i] = acc;
        }
        for (int i = e - 1; i >= s; i--) {
            double acc = z[i];
            for (int32_t q = h->frp[i + 1] - 1; q > h->fdg[i]; q--) acc = acc - h->fv[q] * z[h->fci[q]];
            z[i] = acc / h->fv[h->fdg[i]];
        }
    }
}

/* x = approximate solution of A_L x = b (x0 = 0); returns the iterations
 * run. ws: 4 n_L doubles. */
static int coarse_fcg(const hier_t *h, const double *b, double *x, double *ws) {
    const csr_t *A = &h->lev[h->nlev - 1].A;
    int n = A->n;
    double *r = ws, *z = ws + n, *p = ws + 2 * (size_t)n, *q = ws + 3 * (size_t)n;
    for (int i = 0; i < n; i++) { x[i] = 0.0; r[i] = b[i]; }
    double bn = sqrt(dot(n, b, b));
    int its = 0;
    if (!(bn > 0.0) || !isfinite(bn)) goto out;
    double pq_old = 0.0;
    for (int k = 1; k <= h->cmaxit; k++) {
        bj_apply(h, r, z);
        double rho = dot(n, r, z);
        if (!(rho > 0.0) || !isfinite(rho)) break;
        if (k == 1) {
            for (int i = 0; i < n; i++) p[i] = z[i];
        } else {
            double beta = -dot(n, z, q) / pq_old;
            for (int i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        }
        or_spmv(n, A->rp, A->ci, A->v, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) break;
        double alpha = rho / pq;
        for (int i = 0; i < n; i++) x[i] = x[i] + alpha * p[i];
        for (int i = 0; i < n; i++) r[i] = r[i] - alpha * q[i];
        pq_old = pq;
        its = k;
        if (sqrt(dot(n, r, r)) <= h->ctol * bn) break;
    }
out:
    if (h->cstat) { h->cstat[0] += 1; h->cstat[1] += its; h->cstat[2] = its; }
    return its;
}

/* Factor of the coarsest level for the chosen solver: the dense Cholesky
 * factor, or the blocks' ILU(1) factors. */
static int coarse_build(hier_t *h) {
    level_t *lc = &h->lev[h->nlev - 1];
    int nL = lc->A.n;
    h->nL = nL;
    if (h->csolver == 1) return ilu1_build(h);
    if (nL > OR_DENSE_MAX) return OR_ERR_COARSE;
    double *Ad = (double *)calloc((size_t)nL * (size_t)nL, sizeof(double));
    if (!h->L) h->L = (double *)malloc((size_t)nL * (size_t)nL * sizeof(double));
    if (!Ad || !h->L) { free(Ad); return OR_ERR_OOM; }
    for (int i = 0; i < nL; i++)
        for (int32_t k = lc->A.rp[i]; k < lc->A.rp[i + 1]; k++)
            Ad[(size_t)i * nL + lc->A.ci[k]] = lc->A.v[k];
    int st = or_chol(nL, Ad, h->L);
    free(Ad);
    return st;
}

/* ------------------------------------------------------------ hierarchy
 * Sec. 3.1: A_{l+1} = P_l^T A_l P_l; aggregates larger than pairs come from
 * multiplying pairwise prolongators (the aggregate size is an input
 * parameter: n_pass pairwise passes give |G| <= 2^n_pass).
 *
 * Readings: w = 1 on level 0 and the coarse w_c of a pass is the w of the
 * next pass (and of the next level); the prolongator is the tentative one
 * (no smoothing step); the level matrix is the result of the n_pass
 * successive pairwise Galerkin products; the composed map and weight of a
 * level are the products of its passes' maps and weights, multiplied in pass
 * order. Levels stop when n_l <= coarse_max, when a level would keep more
 * than 0.9 n_l rows (or none), or at max_levels; the last level is solved by
 * dense Cholesky.
 */
void or_free(hier_t *h) {
    if (!h) return;
    for (int l = 0; l < h->nlev; l++) {
        level_t *lv = &h->lev[l];
        csr_free(&lv->A);
        free(lv->dinv); free(lv->w); free(lv->agg); free(lv->p);
        free(lv->v32); free(lv->dinv32); free(lv->p32);
        csr_free(&lv->P); free(lv->P32);
        for (int k = 0; k < OR_MAX_PASS; k++) free(lv->pass_agg[k]);
    }
    free(h->L);
    free(h->frp); free(h->fci); free(h->fdg); free(h->fv); free(h->flev); free(h->cstat);
    free(h);
}

/* ------------------------------------------------- smoothed aggregation
 * Sec. 3.1: the prolongator actually used is P = (I - omega D^-1 A) P_hat,
 * D = diag(A), omega = 1 / ||D^-1 A||_inf (~ 1 / rho(D^-1 A)). Aggregates of
 * more than two come from multiplying the pass prolongators; reading: the
 * tentative pass prolongators are multiplied into the level's P_hat (the
 * composed map and weight), which is then smoothed once with the level's A.
 *
 * Row i of P: the tentative entry p_i at column agg(i), then, for each stored
 * a_ij with agg(j) >= 0, -omega (a_ij / a_ii) p_j added to column agg(j);
 * contributions to one column are added in increasing j, starting from the
 * tentative entry. Columns sorted; every column that receives a contribution
 * is kept (exact zeros included), so the pattern depends on A's pattern only.
 */
static double smoothing_omega(const csr_t *a) {
    double mx = 0.0;
    for (int i = 0; i < a->n; i++) {
        double d = diag_of(a, i), s = 0.0;
        for (int32_t k = a->rp[i]; k < a->rp[i + 1]; k++) s += fabs(a->v[k]) / d;
        if (s > mx) mx = s;
    }
    return 1.0 / mx;
}

typedef struct { int32_t J, j; double t; } pterm_t;

static int pterm_cmp(const void *pa, const void *pb) {
    const pterm_t *a = (const pterm_t *)pa, *b = (const pterm_t *)pb;
    if (a->J != b->J) return a->J < b->J ? -1 : 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    return 0;
}

static int smooth_prolongator(const csr_t *a, const int32_t *agg, const double *p, int nc, double omega,
                              csr_t *P) {
    int n = a->n;
    P->n = n;
    P->rp = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t cap = a->nnz + n + 16;
    P->ci = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    P->v = (double *)malloc((size_t)cap * sizeof(double));
    int64_t tcap = 64;
    pterm_t *tm = (pterm_t *)malloc((size_t)tcap * sizeof(pterm_t));
    if (!P->rp || !P->ci || !P->v || !tm) { free(tm); csr_free(P); return OR_ERR_OOM; }
    (void)nc;
    int64_t nz = 0;
    P->rp[0] = 0;
    for (int i = 0; i < n; i++) {
        int64_t nt = 0;
        double s = omega / diag_of(a, i);
        /* the tentative entry sorts first within its column (j = -1) */
        if (agg[i] >= 0) { tm[nt].J = agg[i]; tm[nt].j = -1; tm[nt].t = p[i]; nt++; }
        for (int32_t k = a->rp[i]; k < a->rp[i + 1]; k++) {
            int j = a->ci[k];
            if (agg[j] < 0) continue;
            if (nt == tcap) {
                tcap *= 2;
                pterm_t *t2 = (pterm_t *)realloc(tm, (size_t)tcap * sizeof(pterm_t));
                if (!t2) { free(tm); csr_free(P); return OR_ERR_OOM; }
                tm = t2;
            }
            tm[nt].J = agg[j]; tm[nt].j = j; tm[nt].t = -(s * a->v[k]) * p[j];
            nt++;
        }
        qsort(tm, (size_t)nt, sizeof(pterm_t), pterm_cmp);
        for (int64_t t = 0; t < nt; t++) {
            if (t == 0 || tm[t].J != tm[t - 1].J) {
                P->ci[nz] = tm[t].J;
                P->v[nz] = tm[t].t;
                nz++;
            } else {
                P->v[nz - 1] = P->v[nz - 1] + tm[t].t;
            }
        }
        P->rp[i + 1] = (int32_t)nz;
    }
    P->nnz = nz;
    free(tm);
    return OR_OK;
}

/* A_c = P^T A P for an explicit P. Row I of A_c for columns J >= I:
 * acc_J = sum over the rows i of P's column I (increasing i) of
 * p_iI * (A P)_iJ, with (A P)_iJ = sum over a_ik (storage order) of
 * a_ik p_kJ; the entries below the diagonal are mirrored from above, so A_c
 * is bitwise symmetric (the next level's matching reads one copy of each
 * coupling). */
static int rap_explicit(const csr_t *a, const csr_t *P, int nc, csr_t *out) {
    int n = a->n;
    /* A P, row by row, columns sorted */
    double *acc = (double *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
    int32_t *mark = (int32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
    int32_t *list = (int32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
    csr_t AP = {n, 0, NULL, NULL, NULL};
    AP.rp = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t cap = 1024;
    AP.ci = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    AP.v = (double *)malloc((size_t)cap * sizeof(double));
    if (!acc || !mark || !list || !AP.rp || !AP.ci || !AP.v) {
        free(acc); free(mark); free(list); csr_free(&AP); return OR_ERR_OOM;
    }
    for (int J = 0; J < nc; J++) mark[J] = -1;
    int64_t nz = 0;
    AP.rp[0] = 0;
    for (int i = 0; i < n; i++) {
        int m = 0;
        for (int32_t k = a->rp[i]; k < a->rp[i + 1]; k++) {
            int c = a->ci[k];
            for (int32_t q = P->rp[c]; q < P->rp[c + 1]; q++) {
                int J = P->ci[q];
                if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; list[m++] = J; }
                acc[J] = acc[J] + a->v[k] * P->v[q];
            }
        }
        /* sort the touched columns (insertion sort: rows are short) */
        for (int x = 1; x < m; x++) {
            int y = list[x], z = x;
            while (z > 0 && list[z - 1] > y) { list[z] = list[z - 1]; z--; }
            list[z] = y;
        }
        if (nz + m > cap) {
            while (nz + m > cap) cap *= 2;
            int32_t *c2 = (int32_t *)realloc(AP.ci, (size_t)cap * sizeof(int32_t));
            if (c2) AP.ci = c2;
            double *v2 = (double *)realloc(AP.v, (size_t)cap * sizeof(double));
            if (v2) AP.v = v2;
            if (!c2 || !v2) { free(acc); free(mark); free(list); csr_free(&AP); return OR_ERR_OOM; }
        }
        for (int x = 0; x < m; x++) { AP.ci[nz] = list[x]; AP.v[nz] = acc[list[x]]; nz++; }
        AP.rp[i + 1] = (int32_t)nz;
    }
    AP.nnz = nz;
    /* P^T by columns: for each coarse I, the rows i with p_iI != stored */
    int32_t *tc = (int32_t *)calloc((size_t)nc + 1, sizeof(int32_t));
    int32_t *ti = (int32_t *)malloc((size_t)(P->nnz > 0 ? P->nnz : 1) * sizeof(int32_t));
    double *tv = (double *)malloc((size_t)(P->nnz > 0 ? P->nnz : 1) * sizeof(double));
    int32_t *fill = (int32_t *)malloc(((size_t)nc + 1) * sizeof(int32_t));
    if (!tc || !ti || !tv || !fill) {
        free(tc); free(ti); free(tv); free(fill); free(acc); free(mark); free(list); csr_free(&AP);
        return OR_ERR_OOM;
    }
    for (int64_t q = 0; q < P->nnz; q++) tc[P->ci[q] + 1]++;
    for (int I = 0; I < nc; I++) tc[I + 1] += tc[I];
    memcpy(fill, tc, ((size_t)nc + 1) * sizeof(int32_t));
    for (int i = 0; i < n; i++)
        for (int32_t q = P->rp[i]; q < P->rp[i + 1]; q++) {
            int32_t pos = fill[P->ci[q]]++;
            ti[pos] = i;
            tv[pos] = P->v[q];
        }
    free(fill);
    /* upper part of each coarse row */
    int32_t *ucnt = (int32_t *)calloc((size_t)nc + 1, sizeof(int32_t));
    int64_t ucap = 1024, unz = 0;
    int32_t *uJ = (int32_t *)malloc((size_t)ucap * sizeof(int32_t));
    double *uV = (double *)malloc((size_t)ucap * sizeof(double));
    int32_t *urp = (int32_t *)malloc(((size_t)nc + 1) * sizeof(int32_t));
    int st = OR_OK;
    if (!ucnt || !uJ || !uV || !urp) st = OR_ERR_OOM;
    for (int J = 0; J < nc; J++) mark[J] = -1;
    if (!st) urp[0] = 0;
    for (int I = 0; I < nc && !st; I++) {
        int m = 0;
        for (int32_t q = tc[I]; q < tc[I + 1]; q++) {
            int i = ti[q];
            double pv = tv[q];
            for (int32_t r = AP.rp[i]; r < AP.rp[i + 1]; r++) {
                int J = AP.ci[r];
                if (J < I) continue;
                if (mark[J] != I) { mark[J] = I; acc[J] = 0.0; list[m++] = J; }
                acc[J] = acc[J] + pv * AP.v[r];
            }
        }
        for (int x = 1; x < m; x++) {
            int y = list[x], z = x;
            while (z > 0 && list[z - 1] > y) { list[z] = list[z - 1]; z--; }
            list[z] = y;
        }
        if (unz + m > ucap) {
            while (unz + m > ucap) ucap *= 2;
            int32_t *c2 = (int32_t *)realloc(uJ, (size_t)ucap * sizeof(int32_t));
            if (c2) uJ = c2;
            double *v2 = (double *)realloc(uV, (size_t)ucap * sizeof(double));
            if (v2) uV = v2;
            if (!c2 || !v2) { st = OR_ERR_OOM; break; }
        }
        for (int x = 0; x < m; x++) {
            uJ[unz] = list[x]; uV[unz] = acc[list[x]]; unz++;
            if (list[x] != I) ucnt[list[x] + 1]++;   /* mirrored entry in row J */
        }
        urp[I + 1] = (int32_t)unz;
    }
    if (!st) {
        /* full rows: mirrored lower entries (increasing I) then the upper part */
        out->n = nc;
        out->rp = (int32_t *)malloc(((size_t)nc + 1) * sizeof(int32_t));
        int64_t tot = 0;
        for (int I = 0; I < nc; I++) tot += (urp[I + 1] - urp[I]) + ucnt[I + 1];
        out->ci = (int32_t *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
        out->v = (double *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(double));
        int32_t *lf = (int32_t *)malloc(((size_t)nc + 1) * sizeof(int32_t));
        if (!out->rp || !out->ci || !out->v || !lf) { free(lf); csr_free(out); st = OR_ERR_OOM; }
        else {
            out->rp[0] = 0;
            for (int I = 0; I < nc; I++) out->rp[I + 1] = out->rp[I] + ucnt[I + 1] + (urp[I + 1] - urp[I]);
            for (int I = 0; I < nc; I++) lf[I] = out->rp[I];
            for (int I = 0; I < nc; I++)
                for (int32_t q = urp[I]; q < urp[I + 1]; q++) {
                    int J = uJ[q];
                    if (J == I) continue;
                    out->ci[lf[J]] = I; out->v[lf[J]] = uV[q]; lf[J]++;
                }
            for (int I = 0; I < nc; I++)
                for (int32_t q = urp[I]; q < urp[I + 1]; q++) {
                    out->ci[lf[I]] = uJ[q]; out->v[lf[I]] = uV[q]; lf[I]++;
                }
            out->nnz = tot;
            free(lf);
        }
    }
    free(ucnt); free(uJ); free(uV); free(urp);
    free(tc); free(ti); free(tv); free(acc); free(mark); free(list); csr_free(&AP);
    return st;
}

static int level_finish(level_t *lv) {
    int n = lv->A.n;
    int64_t z = lv->A.nnz;
    lv->dinv = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    lv->dinv32 = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
    lv->v32 = (float *)malloc((size_t)(z > 0 ? z : 1) * sizeof(float));
    if (!lv->dinv || !lv->dinv32 || !lv->v32) return OR_ERR_OOM;
    or_l1_diag(n, lv->A.rp, lv->A.ci, lv->A.v, lv->dinv);
    for (int i = 0; i < n; i++) {
        lv->dinv[i] = 1.0 / lv->dinv[i];
        lv->dinv32[i] = (float)lv->dinv[i];
    }
    for (int64_t k = 0; k < z; k++) lv->v32[k] = (float)lv->A.v[k];
    return OR_OK;
}

int or_setup_cfg(int n, const int32_t *rp, const int32_t *ci, const double *v, const or_cfg_t *cfg,
                 hier_t **out) {
    *out = NULL;
    int coarse_max = cfg->coarse_max, n_pass = cfg->n_pass, max_levels = cfg->max_levels;
    int smoothed = cfg->smoothed;
    if (n <= 0 || n_pass < 1 || n_pass > OR_MAX_PASS || max_levels < 1 || coarse_max < 1)
        return OR_ERR_ARG;
    if (cfg->csolver < 0 || cfg->csolver > 2 || cfg->cb < 1 || cfg->cmaxit < 1 || !(cfg->ctol > 0.0))
        return OR_ERR_ARG;
    if (max_levels > OR_MAX_LEVELS) max_levels = OR_MAX_LEVELS;
    int st = csr_check(n, rp, ci, v);
    if (st) return st;
    hier_t *h = (hier_t *)calloc(1, sizeof(hier_t));
    if (!h) return OR_ERR_OOM;
    h->smoothed = smoothed ? 1 : 0;
    h->cb = cfg->cb; h->cmaxit = cfg->cmaxit; h->ctol = cfg->ctol;
    h->cstat = (int64_t *)calloc(3, sizeof(int64_t));
    if (!h->cstat) { free(h); return OR_ERR_OOM; }
    level_t *l0 = &h->lev[0];
    int64_t z = rp[n];
    l0->A.n = n; l0->A.nnz = z;
    l0->A.rp = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    l0->A.ci = (int32_t *)malloc((size_t)(z > 0 ? z : 1) * sizeof(int32_t));
    l0->A.v = (double *)malloc((size_t)(z > 0 ? z : 1) * sizeof(double));
    l0->w = (double *)malloc((size_t)n * sizeof(double));
    h->nlev = 1;
    if (!l0->A.rp || !l0->A.ci || !l0->A.v || !l0->w) { or_free(h); return OR_ERR_OOM; }
    memcpy(l0->A.rp, rp, ((size_t)n + 1) * sizeof(int32_t));
    memcpy(l0->A.ci, ci, (size_t)z * sizeof(int32_t));
    memcpy(l0->A.v, v, (size_t)z * sizeof(double));
    for (int i = 0; i < n; i++) l0->w[i] = 1.0;

    for (int l = 0;; l++) {
        level_t *lv = &h->lev[l];
        int nl = lv->A.n;
        if (nl <= coarse_max || l == max_levels - 1) break;
        /* n_pass pairwise passes */
        csr_t cur = lv->A;       /* borrowed on the first pass */
        double *curw = lv->w;
        int own = 0;
        int32_t *cagg = (int32_t *)malloc((size_t)nl * sizeof(int32_t));
        double *cp = (double *)malloc((size_t)nl * sizeof(double));
        if (!cagg || !cp) { free(cagg); free(cp); or_free(h); return OR_ERR_OOM; }
        for (int i = 0; i < nl; i++) { cagg[i] = i; cp[i] = 1.0; }
        lv->pass_n[0] = nl;
        for (int ps = 0; ps < n_pass; ps++) {
            int m = cur.n;
            int32_t *mate = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
            int32_t *agg = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
            double *p = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
            double *wc = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
            if (!mate || !agg || !p || !wc) {
                free(mate); free(agg); free(p); free(wc); free(cagg); free(cp);
                if (own) { csr_free(&cur); free(curw); }
                or_free(h); return OR_ERR_OOM;
            }
            int np = or_match(m, cur.rp, cur.ci, cur.v, curw, mate);
            int nc = np < 0 ? 0 : or_aggregate(m, cur.rp, cur.ci, cur.v, mate, curw, agg, p, wc);
            csr_t nxt = {0, 0, NULL, NULL, NULL};
            st = np < 0 ? -np : rap(&cur, agg, p, nc, &nxt);
            free(mate);
            if (st) {
                free(agg); free(p); free(wc); free(cagg); free(cp);
                if (own) { csr_free(&cur); free(curw); }
                or_free(h); return st;
            }
            for (int i = 0; i < nl; i++) {
                if (cagg[i] >= 0) {
                    int a = cagg[i];
                    cp[i] = cp[i] * p[a];
                    cagg[i] = agg[a];
                }
                if (cagg[i] < 0) cp[i] = 0.0;
            }
            lv->pass_agg[ps] = agg;
            lv->pass_n[ps + 1] = nc;
            free(p);
            if (own) { csr_free(&cur); free(curw); }
            cur = nxt; curw = wc; own = 1;
        }
        lv->npass = n_pass;
        int nc = cur.n;
        if (nc == 0 || (double)nc > 0.9 * (double)nl) {
            /* stalled: this level is the coarsest */
            csr_free(&cur); free(curw); free(cagg); free(cp);
            for (int k = 0; k < OR_MAX_PASS; k++) { free(lv->pass_agg[k]); lv->pass_agg[k] = NULL; }
            lv->npass = 0;
            break;
        }
        lv->agg = cagg; lv->p = cp;
        lv->p32 = (float *)malloc((size_t)nl * sizeof(float));
        if (!lv->p32) { csr_free(&cur); free(curw); or_free(h); return OR_ERR_OOM; }
        for (int i = 0; i < nl; i++) lv->p32[i] = (float)cp[i];
        if (h->smoothed) {
            /* P = (I - omega D^-1 A) P_hat and A_c = P^T A P replace the
             * tentative product of the passes */
            csr_t Pm = {0, 0, NULL, NULL, NULL}, Ac = {0, 0, NULL, NULL, NULL};
            st = smooth_prolongator(&lv->A, cagg, cp, nc, smoothing_omega(&lv->A), &Pm);
            if (!st) st = rap_explicit(&lv->A, &Pm, nc, &Ac);
            csr_free(&cur);
            if (st) { csr_free(&Pm); free(curw); or_free(h); return st; }
            cur = Ac;
            lv->P = Pm;
            lv->P32 = (float *)malloc((size_t)(Pm.nnz > 0 ? Pm.nnz : 1) * sizeof(float));
            if (!lv->P32) { csr_free(&cur); free(curw); or_free(h); return OR_ERR_OOM; }
            for (int64_t q = 0; q < Pm.nnz; q++) lv->P32[q] = (float)Pm.v[q];
        }
        level_t *nx = &h->lev[l + 1];
        nx->A = cur; nx->w = curw;
        h->nlev = l + 2;
    }
    for (int l = 0; l < h->nlev; l++) {
        st = level_finish(&h->lev[l]);
        if (st) { or_free(h); return st; }
    }
    /* the coarsest level's solver and its factor */
    int nL = h->lev[h->nlev - 1].A.n;
    h->csolver = cfg->csolver == 2 || (cfg->csolver == 0 && nL > OR_DENSE_MAX) ? 1 : 0;
    st = coarse_build(h);
    if (st) { or_free(h); return st; }
    *out = h;
    return OR_OK;
}

int or_setup_ex(int n, const int32_t *rp, const int32_t *ci, const double *v,
                int coarse_max, int n_pass, int max_levels, int smoothed, hier_t **out) {
    or_cfg_t cfg = {coarse_max, n_pass, max_levels, smoothed, 1, 32, 30, 1e-3};
    return or_setup_cfg(n, rp, ci, v, &cfg, out);
}

int or_setup(int n, const int32_t *rp, const int32_t *ci, const double *v,
             int coarse_max, int n_pass, int max_levels, hier_t **out) {
    return or_setup_ex(n, rp, ci, v, coarse_max, n_pass, max_levels, 0, out);
}

/* Select the smoother: nu = 0 restores the l1-Jacobi sweep of the setup;
 * nu >= 1 sweeps of l1 hybrid Gauss-Seidel over nblocks row blocks per level
 * (nblocks = 0: one row per block). Re-forms D^-1 with the block rule. */
int or_set_smoother(hier_t *h, int nu, int nblocks) {
    if (nu < 0 || nu > 64 || nblocks < 0) return OR_ERR_ARG;
    h->nu = nu;
    h->nblocks = nblocks;
    for (int l = 0; l < h->nlev; l++) {
        level_t *lv = &h->lev[l];
        if (nu > 0) {
            hybrid_l1(&lv->A, gs_rows(h, lv->A.n), lv->dinv, lv->dinv32);
        } else {
            or_l1_diag(lv->A.n, lv->A.rp, lv->A.ci, lv->A.v, lv->dinv);
            for (int i = 0; i < lv->A.n; i++) {
                lv->dinv[i] = 1.0 / lv->dinv[i];
                lv->dinv32[i] = (float)lv->dinv[i];
            }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------- partial reuse (Sec. 4)
 * When the mesh (the sparsity pattern) stays and only the coefficients
 * change, the hierarchy can be rebuilt with the same prolongators: the
 * aggregates of every pass and their weights are kept, and the Galerkin
 * products, the l1 smoothers and the coarsest factor are formed again from
 * the new values (Sec. 4, reuse of the prolongators/restrictors).
 *
 * The weights of a pass depend only on its aggregates and on w (w = 1 on
 * level 0, then the aggregate norms), not on the matrix values, so they are
 * restated here from the kept maps with the arithmetic of or_aggregate:
 * pair {i < j}: p = w / ||(w_i, w_j)||, singleton: p = w / |w|, and a row
 * left out of the coarse space (agg = -1) keeps p = 0.
 */
static void pass_weights(int m, const int32_t *agg, int nc, const double *w, double *p, double *wc) {
    int32_t *first = (int32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
    int32_t *second = (int32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int32_t));
    for (int I = 0; I < nc; I++) { first[I] = -1; second[I] = -1; }
    for (int i = 0; i < m; i++) {
        int I = agg[i];
        if (I < 0) { p[i] = 0.0; continue; }
        if (first[I] < 0) first[I] = i; else second[I] = i;
    }
    for (int I = 0; I < nc; I++) {
        int i = first[I], j = second[I];
        if (j >= 0) {
            double nrm = sqrt(w[i] * w[i] + w[j] * w[j]);
            p[i] = w[i] / nrm; p[j] = w[j] / nrm;
            wc[I] = nrm;
        } else {
            p[i] = w[i] / fabs(w[i]);
            wc[I] = fabs(w[i]);
        }
    }
    free(first); free(second);
}

/* New values v for the finest matrix, whose pattern (rp, ci) must be the one
 * the hierarchy was built on (else OR_ERR_ARG and the hierarchy is kept). */
int or_refresh(hier_t *h, int n, const int32_t *rp, const int32_t *ci, const double *v) {
    level_t *l0 = &h->lev[0];
    if (n != l0->A.n || rp[n] != l0->A.nnz) return OR_ERR_ARG;
    if (memcmp(rp, l0->A.rp, ((size_t)n + 1) * sizeof(int32_t)) != 0) return OR_ERR_ARG;
    if (memcmp(ci, l0->A.ci, (size_t)l0->A.nnz * sizeof(int32_t)) != 0) return OR_ERR_ARG;
    int st = csr_check(n, rp, ci, v);
    if (st) return st;
    memcpy(l0->A.v, v, (size_t)l0->A.nnz * sizeof(double));
    for (int l = 0; l + 1 < h->nlev; l++) {
        level_t *lv = &h->lev[l];
        if (h->smoothed) {
            /* P and A_{l+1} = P^T A_l P formed again; both keep their patterns */
            int nc = h->lev[l + 1].A.n;
            csr_t Pm = {0, 0, NULL, NULL, NULL}, Ac = {0, 0, NULL, NULL, NULL};
            st = smooth_prolongator(&lv->A, lv->agg, lv->p, nc, smoothing_omega(&lv->A), &Pm);
            if (!st) st = rap_explicit(&lv->A, &Pm, nc, &Ac);
            csr_t *An = &h->lev[l + 1].A;
            int same = !st && Pm.nnz == lv->P.nnz &&
                       memcmp(Pm.rp, lv->P.rp, ((size_t)Pm.n + 1) * sizeof(int32_t)) == 0 &&
                       memcmp(Pm.ci, lv->P.ci, (size_t)Pm.nnz * sizeof(int32_t)) == 0 && Ac.nnz == An->nnz &&
                       memcmp(Ac.rp, An->rp, ((size_t)Ac.n + 1) * sizeof(int32_t)) == 0 &&
                       memcmp(Ac.ci, An->ci, (size_t)Ac.nnz * sizeof(int32_t)) == 0;
            if (same) {
                memcpy(lv->P.v, Pm.v, (size_t)Pm.nnz * sizeof(double));
                for (int64_t q = 0; q < Pm.nnz; q++) lv->P32[q] = (float)Pm.v[q];
                memcpy(An->v, Ac.v, (size_t)Ac.nnz * sizeof(double));
            }
            csr_free(&Pm); csr_free(&Ac);
            if (st) return st;
            if (!same) return OR_ERR_ARG;
            continue;
        }
        csr_t cur = lv->A;            /* borrowed on the first pass */
        double *curw = lv->w;
        int own = 0;
        for (int ps = 0; ps < lv->npass; ps++) {
            int m = lv->pass_n[ps], nc = lv->pass_n[ps + 1];
            double *p = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
            double *wc = (double *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(double));
            csr_t nxt = {0, 0, NULL, NULL, NULL};
            if (!p || !wc) st = OR_ERR_OOM;
            else {
                pass_weights(m, lv->pass_agg[ps], nc, curw, p, wc);
                st = rap(&cur, lv->pass_agg[ps], p, nc, &nxt);
            }
            free(p);
            if (own) { csr_free(&cur); free(curw); }
            if (st) { free(wc); return st; }
            cur = nxt; curw = wc; own = 1;
        }
        /* the last pass gives A_{l+1}: same pattern, new values */
        csr_t *An = &h->lev[l + 1].A;
        int same = cur.n == An->n && cur.nnz == An->nnz &&
                   memcmp(cur.rp, An->rp, ((size_t)cur.n + 1) * sizeof(int32_t)) == 0 &&
                   memcmp(cur.ci, An->ci, (size_t)cur.nnz * sizeof(int32_t)) == 0;
        if (same) memcpy(An->v, cur.v, (size_t)cur.nnz * sizeof(double));
        csr_free(&cur); free(curw);
        if (!same) return OR_ERR_ARG;
    }
    for (int l = 0; l < h->nlev; l++) {
        level_t *lv = &h->lev[l];
        free(lv->dinv); free(lv->dinv32); free(lv->v32);
        lv->dinv = NULL; lv->dinv32 = NULL; lv->v32 = NULL;
        st = level_finish(lv);
        if (st) return st;
        if (h->nu > 0) hybrid_l1(&lv->A, gs_rows(h, lv->A.n), lv->dinv, lv->dinv32);
    }
    return coarse_build(h);
}

/* ------------------------------------------------------------ accessors */
int or_nlevels(const hier_t *h) { return h->nlev; }

void or_level_size(const hier_t *h, int l, int *n, int64_t *nnz, int *npass) {
    *n = h->lev[l].A.n; *nnz = h->lev[l].A.nnz; *npass = h->lev[l].npass;
}

void or_level_copy(const hier_t *h, int l, int32_t *rp, int32_t *ci, double *v,
                   double *dinv, double *w) {
    const level_t *lv = &h->lev[l];
    int n = lv->A.n;
    memcpy(rp, lv->A.rp, ((size_t)n + 1) * sizeof(int32_t));
    memcpy(ci, lv->A.ci, (size_t)lv->A.nnz * sizeof(int32_t));
    memcpy(v, lv->A.v, (size_t)lv->A.nnz * sizeof(double));
    memcpy(dinv, lv->dinv, (size_t)n * sizeof(double));
    memcpy(w, lv->w, (size_t)n * sizeof(double));
}

/* composed map of level l (l < nlevels-1) */
void or_level_agg(const hier_t *h, int l, int32_t *agg, double *p) {
    const level_t *lv = &h->lev[l];
    memcpy(agg, lv->agg, (size_t)lv->A.n * sizeof(int32_t));
    memcpy(p, lv->p, (size_t)lv->A.n * sizeof(double));
}

/* map of one pass on level l; its input size is pass_n[ps] */
int or_pass_agg(const hier_t *h, int l, int ps, int32_t *agg) {
    const level_t *lv = &h->lev[l];
    if (ps >= lv->npass) return -1;
    memcpy(agg, lv->pass_agg[ps], (size_t)lv->pass_n[ps] * sizeof(int32_t));
    return lv->pass_n[ps + 1];
}

int or_pass_n(const hier_t *h, int l, int ps) { return h->lev[l].pass_n[ps]; }

/* explicit (smoothed) prolongator of level l: nnz, or -1 when tentative */
int64_t or_level_P_nnz(const hier_t *h, int l) { return h->lev[l].P.rp ? h->lev[l].P.nnz : -1; }

void or_level_P(const hier_t *h, int l, int32_t *rp, int32_t *ci, double *v) {
    const csr_t *P = &h->lev[l].P;
    memcpy(rp, P->rp, ((size_t)P->n + 1) * sizeof(int32_t));
    memcpy(ci, P->ci, (size_t)P->nnz * sizeof(int32_t));
    memcpy(v, P->v, (size_t)P->nnz * sizeof(double));
}

void or_coarse_factor(const hier_t *h, double *L) {
    memcpy(L, h->L, (size_t)h->nL * (size_t)h->nL * sizeof(double));
}

/* coarsest solver: 0 dense, 1 iterative (block-Jacobi ILU(1) + FCG) */
int or_coarse_kind(const hier_t *h) { return h->csolver; }

/* stored entries of the ILU(1) factors (-1 with the dense solver) */
int64_t or_coarse_ilu_nnz(const hier_t *h) { return h->csolver ? (int64_t)h->frp[h->nL] : -1; }

void or_coarse_ilu(const hier_t *h, int32_t *rp, int32_t *ci, double *v, int32_t *dg) {
    int n = h->nL;
    memcpy(rp, h->frp, ((size_t)n + 1) * sizeof(int32_t));
    memcpy(ci, h->fci, (size_t)h->frp[n] * sizeof(int32_t));
    memcpy(v, h->fv, (size_t)h->frp[n] * sizeof(double));
    memcpy(dg, h->fdg, (size_t)n * sizeof(int32_t));
}

/* The coarsest solver alone: x ~ A_L^{-1} b. Returns the inner iterations
 * (0 with the dense solver), or -2 when out of memory. */
int or_coarse_solve(const hier_t *h, const double *b, double *x) {
    if (!h->csolver) {
        or_chol_solve(h->nL, h->L, b, x);
        return 0;
    }
    double *ws = (double *)malloc(4 * (size_t)(h->nL > 0 ? h->nL : 1) * sizeof(double));
    if (!ws) return -2;
    int its = coarse_fcg(h, b, x, ws);
    free(ws);
    return its;
}

/* z = M^{-1} r with the block-Jacobi ILU(1) preconditioner alone */
void or_coarse_prec(const hier_t *h, const double *r, double *z) { bj_apply(h, r, z); }

/* calls of the iterative coarsest solver, inner iterations in total, and the
 * count of the last call */
void or_coarse_stats(const hier_t *h, int64_t *out) {
    out[0] = h->cstat[0]; out[1] = h->cstat[1]; out[2] = h->cstat[2];
}

/* -------------------------------------------------------------- V-cycle
 * Eq. (multiplicative composition) with nu = 1 and M_l = D_l1 (symmetric, so
 * M^{-T} = M^{-1}), started from a zero guess on every level:
 *   x_l = D^{-1} b_l                       (pre-smooth)
 *   b_{l+1} = P^T (b_l - A_l x_l)          (restrict the residual)
 *   x_{l+1} = B_{l+1} b_{l+1}              (recurse; dense solve on the last)
 *   x_l += P x_{l+1}                       (prolong)
 *   x_l += D^{-1} (b_l - A_l x_l)          (post-smooth)
 * The result is z = x_0 = B r.
 */
static int vcycle64(const hier_t *h, const double *r, double *z) {
    int L = h->nlev - 1;
    double *bl[OR_MAX_LEVELS] = {0}, *xl[OR_MAX_LEVELS] = {0}, *t = NULL, *u = NULL;
    int st = OR_OK;
    int nmax = h->lev[0].A.n;
    t = (double *)malloc((size_t)nmax * sizeof(double));
    u = (double *)malloc((size_t)nmax * sizeof(double));
    for (int l = 0; l <= L; l++) {
        int n = h->lev[l].A.n;
        bl[l] = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        xl[l] = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        if (!bl[l] || !xl[l]) st = OR_ERR_OOM;
    }
    if (!t || !u) st = OR_ERR_OOM;
    if (st) goto done;
    memcpy(bl[0], r, (size_t)nmax * sizeof(double));
    for (int l = 0; l < L; l++) {
        const level_t *lv = &h->lev[l];
        int n = lv->A.n, nc = h->lev[l + 1].A.n;
        if (h->nu > 0) {
            /* nu forward sweeps from zero */
            int nb = gs_rows(h, n);
            sweep64(&lv->A, lv->dinv, nb, bl[l], NULL, xl[l], 1);
            for (int s = 1; s < h->nu; s++) {
                memcpy(u, xl[l], (size_t)n * sizeof(double));
                sweep64(&lv->A, lv->dinv, nb, bl[l], u, xl[l], 1);
            }
        } else {
            for (int i = 0; i < n; i++) xl[l][i] = lv->dinv[i] * bl[l][i];
        }
        or_spmv(n, lv->A.rp, lv->A.ci, lv->A.v, xl[l], t);
        for (int I = 0; I < nc; I++) bl[l + 1][I] = 0.0;
        if (lv->P.rp) {
            for (int i = 0; i < n; i++) {
                double res = bl[l][i] - t[i];
                for (int32_t q = lv->P.rp[i]; q < lv->P.rp[i + 1]; q++) bl[l + 1][lv->P.ci[q]] += lv->P.v[q] * res;
            }
        } else {
            for (int i = 0; i < n; i++)
                if (lv->agg[i] >= 0) bl[l + 1][lv->agg[i]] += lv->p[i] * (bl[l][i] - t[i]);
        }
    }
    if (h->csolver) {
        double *ws = (double *)malloc(4 * (size_t)(h->nL > 0 ? h->nL : 1) * sizeof(double));
        if (!ws) { st = OR_ERR_OOM; goto done; }
        coarse_fcg(h, bl[L], xl[L], ws);
        free(ws);
    } else {
        or_chol_solve(h->nL, h->L, bl[L], xl[L]);
    }
    for (int l = L - 1; l >= 0; l--) {
        const level_t *lv = &h->lev[l];
        int n = lv->A.n;
        if (lv->P.rp) {
            for (int i = 0; i < n; i++) {
                double s = 0.0;
                for (int32_t q = lv->P.rp[i]; q < lv->P.rp[i + 1]; q++) s += lv->P.v[q] * xl[l + 1][lv->P.ci[q]];
                xl[l][i] = xl[l][i] + s;
            }
        } else {
            for (int i = 0; i < n; i++)
                if (lv->agg[i] >= 0) xl[l][i] += lv->p[i] * xl[l + 1][lv->agg[i]];
        }
        if (h->nu > 0) {
            /* nu backward sweeps (M^T: the symmetric counterpart) */
            int nb = gs_rows(h, n);
            for (int s = 0; s < h->nu; s++) {
                memcpy(u, xl[l], (size_t)n * sizeof(double));
                sweep64(&lv->A, lv->dinv, nb, bl[l], u, xl[l], 0);
            }
        } else {
            or_spmv(n, lv->A.rp, lv->A.ci, lv->A.v, xl[l], t);
            for (int i = 0; i < n; i++) xl[l][i] = xl[l][i] + lv->dinv[i] * (bl[l][i] - t[i]);
        }
    }
    memcpy(z, xl[0], (size_t)nmax * sizeof(double));
done:
    for (int l = 0; l <= L; l++) { free(bl[l]); free(xl[l]); }
    free(t); free(u);
    return st;
}

/* The same V-cycle in single precision: matrix values, l1 diagonal (formed
 * in float64, then rounded), prolongator weights, smoother, residual and
 * transfers all in float32; the input residual is rounded to float32 on
 * entry and z widened on exit; the coarsest solve stays in float64. */
static void spmv32(const csr_t *a, const float *v32, const float *x, float *y) {
    for (int i = 0; i < a->n; i++) {
        float s = 0.0f;
        for (int32_t k = a->rp[i]; k < a->rp[i + 1]; k++) s += v32[k] * x[a->ci[k]];
        y[i] = s;
    }
}

static int vcycle32(const hier_t *h, const double *r, double *z) {
    int L = h->nlev - 1;
    float *bl[OR_MAX_LEVELS] = {0}, *xl[OR_MAX_LEVELS] = {0}, *t = NULL, *u = NULL;
    double *b64 = NULL, *x64 = NULL;
    int st = OR_OK;
    int nmax = h->lev[0].A.n;
    t = (float *)malloc((size_t)nmax * sizeof(float));
    u = (float *)malloc((size_t)nmax * sizeof(float));
    b64 = (double *)malloc((size_t)h->nL * sizeof(double) + 8);
    x64 = (double *)malloc((size_t)h->nL * sizeof(double) + 8);
    for (int l = 0; l <= L; l++) {
        int n = h->lev[l].A.n;
        bl[l] = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
        xl[l] = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
        if (!bl[l] || !xl[l]) st = OR_ERR_OOM;
    }
    if (!t || !u || !b64 || !x64) st = OR_ERR_OOM;
    if (st) goto done;
    for (int i = 0; i < nmax; i++) bl[0][i] = (float)r[i];
    for (int l = 0; l < L; l++) {
        const level_t *lv = &h->lev[l];
        int n = lv->A.n, nc = h->lev[l + 1].A.n;
        if (h->nu > 0) {
            int nb = gs_rows(h, n);
            sweep32(&lv->A, lv->v32, lv->dinv32, nb, bl[l], NULL, xl[l], 1);
            for (int s = 1; s < h->nu; s++) {
                memcpy(u, xl[l], (size_t)n * sizeof(float));
                sweep32(&lv->A, lv->v32, lv->dinv32, nb, bl[l], u, xl[l], 1);
            }
        } else {
            for (int i = 0; i < n; i++) xl[l][i] = lv->dinv32[i] * bl[l][i];
        }
        spmv32(&lv->A, lv->v32, xl[l], t);
        for (int I = 0; I < nc; I++) bl[l + 1][I] = 0.0f;
        if (lv->P.rp) {
            for (int i = 0; i < n; i++) {
                float res = bl[l][i] - t[i];
                for (int32_t q = lv->P.rp[i]; q < lv->P.rp[i + 1]; q++) bl[l + 1][lv->P.ci[q]] += lv->P32[q] * res;
            }
        } else {
            for (int i = 0; i < n; i++)
                if (lv->agg[i] >= 0) bl[l + 1][lv->agg[i]] += lv->p32[i] * (bl[l][i] - t[i]);
        }
    }
    for (int i = 0; i < h->nL; i++) b64[i] = (double)bl[L][i];
    if (h->csolver) {
        double *ws = (double *)malloc(4 * (size_t)(h->nL > 0 ? h->nL : 1) * sizeof(double));
        if (!ws) { st = OR_ERR_OOM; goto done; }
        coarse_fcg(h, b64, x64, ws);
        free(ws);
    } else {
        or_chol_solve(h->nL, h->L, b64, x64);
    }
    for (int i = 0; i < h->nL; i++) xl[L][i] = (float)x64[i];
    for (int l = L - 1; l >= 0; l--) {
        const level_t *lv = &h->lev[l];
        int n = lv->A.n;
        if (lv->P.rp) {
            for (int i = 0; i < n; i++) {
                float s = 0.0f;
                for (int32_t q = lv->P.rp[i]; q < lv->P.rp[i + 1]; q++) s += lv->P32[q] * xl[l + 1][lv->P.ci[q]];
                xl[l][i] = xl[l][i] + s;
            }
        } else {
            for (int i = 0; i < n; i++)
                if (lv->agg[i] >= 0) xl[l][i] += lv->p32[i] * xl[l + 1][lv->agg[i]];
        }
        if (h->nu > 0) {
            int nb = gs_rows(h, n);
            for (int s = 0; s < h->nu; s++) {
                memcpy(u, xl[l], (size_t)n * sizeof(float));
                sweep32(&lv->A, lv->v32, lv->dinv32, nb, bl[l], u, xl[l], 0);
            }
        } else {
            spmv32(&lv->A, lv->v32, xl[l], t);
            for (int i = 0; i < n; i++) xl[l][i] = xl[l][i] + lv->dinv32[i] * (bl[l][i] - t[i]);
        }
    }
    for (int i = 0; i < nmax; i++) z[i] = (double)xl[0][i];
done:
    for (int l = 0; l <= L; l++) { free(bl[l]); free(xl[l]); }
    free(t); free(u); free(b64); free(x64);
    return st;
}

int or_vcycle(const hier_t *h, const double *r, double *z, int fp32) {
    return fp32 ? vcycle32(h, r, z) : vcycle64(h, r, z);
}

/* ---------------------------------------------------------------- Krylov
 * Sec. 3.1 (AMG as preconditioner for a Krylov solver) and Sec. 5 (FCG, stop
 * when the Euclidean norm of the relative residual is small enough, start
 * from a given guess).
 *
 * mode 0: plain PCG with the float64 V-cycle, beta = rho_k / rho_{k-1}.
 * mode 1: flexible CG with one kept direction, FCG(1), with the float32
 *         V-cycle: beta = -(z_k . q_{k-1}) / (p_{k-1} . q_{k-1}), where
 *         q = A p (Notay's truncated flexible CG; equal to the Polak-Ribiere
 *         form z_k.(r_k - r_{k-1}) / rho_{k-1} in exact arithmetic).
 * With the iterative coarsest solver the V-cycle is not a fixed operator,
 * and mode 0 uses the FCG(1) beta too (with the float64 V-cycle).
 * Both: rho_k = r_k . z_k, alpha = rho_k / (p_k . q_k).
 * Readings: "relative residual" is ||r_k|| / ||b||; when the recursive
 * residual meets rtol the true residual b - A x is formed and must meet it
 * too, otherwise r is replaced by the true residual and the recurrence
 * restarts (p = z). iters counts V-cycle applications; hist[k] holds
 * ||r_k|| / ||b|| (the true one after a replacement). ||b|| = 0 gives x = 0.
 */
int or_solve(const hier_t *h, const double *b, double *x, double rtol, int maxit,
             int mode, int *iters, double *hist, double *true_rel) {
    int n = h->lev[0].A.n;
    const csr_t *A = &h->lev[0].A;
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *z = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)malloc((size_t)n * sizeof(double));
    int st = OR_OK;
    *iters = 0;
    if (true_rel) *true_rel = 0.0;
    if (!r || !z || !p || !q) { st = OR_ERR_OOM; goto done; }
    double bn = sqrt(dot(n, b, b));
    if (!isfinite(bn)) { st = OR_ERR_NAN; goto done; }
    if (bn == 0.0) {
        for (int i = 0; i < n; i++) x[i] = 0.0;
        if (hist) hist[0] = 0.0;
        goto done;
    }
    or_spmv(n, A->rp, A->ci, A->v, x, r);
    for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
    double rn = sqrt(dot(n, r, r));
    if (hist) hist[0] = rn / bn;
    if (true_rel) *true_rel = rn / bn;
    if (!isfinite(rn)) { st = OR_ERR_NAN; goto done; }
    if (rn / bn <= rtol) goto done;
    int restart = 1;
    /* an iterative coarsest solve makes the V-cycle vary from one application
     * to the next, so the flexible recurrence is used in both precisions */
    int flexible = mode == 1 || h->csolver;
    double rho_old = 0.0, pq_old = 0.0;
    for (int k = 1; k <= maxit; k++) {
        st = or_vcycle(h, r, z, mode == 1);
        if (st) goto done;
        *iters = k;
        double rho = dot(n, r, z);
        if (!isfinite(rho)) { st = OR_ERR_NAN; goto done; }
        if (!(rho > 0.0)) { st = OR_ERR_BREAKDOWN; goto done; }
        if (restart) {
            for (int i = 0; i < n; i++) p[i] = z[i];
            restart = 0;
        } else {
            double beta = flexible ? -dot(n, z, q) / pq_old : rho / rho_old;
            for (int i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        }
        or_spmv(n, A->rp, A->ci, A->v, p, q);
        double pq = dot(n, p, q);
        if (!isfinite(pq)) { st = OR_ERR_NAN; goto done; }
        if (!(pq > 0.0)) { st = OR_ERR_BREAKDOWN; goto done; }
        double alpha = rho / pq;
        for (int i = 0; i < n; i++) x[i] = x[i] + alpha * p[i];
        for (int i = 0; i < n; i++) r[i] = r[i] - alpha * q[i];
        rn = sqrt(dot(n, r, r));
        if (!isfinite(rn)) { st = OR_ERR_NAN; goto done; }
        if (hist) hist[k] = rn / bn;
        rho_old = rho; pq_old = pq;
        if (rn / bn <= rtol) {
            or_spmv(n, A->rp, A->ci, A->v, x, z);
            for (int i = 0; i < n; i++) z[i] = b[i] - z[i];
            double tn = sqrt(dot(n, z, z));
            if (true_rel) *true_rel = tn / bn;
            if (tn / bn <= rtol) goto done;
            for (int i = 0; i < n; i++) r[i] = z[i];
            if (hist) hist[k] = tn / bn;
            restart = 1;
        }
    }
    /* maxit V-cycles without meeting rtol */
    st = OR_ERR_NOCONV;
    if (true_rel) {
        or_spmv(n, A->rp, A->ci, A->v, x, z);
        for (int i = 0; i < n; i++) z[i] = b[i] - z[i];
        *true_rel = sqrt(dot(n, z, z)) / bn;
    }
done:
    free(r); free(z); free(p); free(q);
    return st;
}
