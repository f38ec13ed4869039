// Internal declarations shared by the CUDA sources of libpcgamg.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "pcgamg.h"
#include "tail_plan.h"

namespace pcgamg {

constexpr int kSlice = 32;        // sliced-ELL slice height (one warp)
constexpr int kBlock = 256;       // threads per block of the streaming kernels
constexpr int kDenseMax = 4096;   // largest coarsest level solved densely
constexpr int kCoarseBlock = 32;  // rows per block-Jacobi block of the iterative coarsest solve
constexpr int kMaxPass = 8;

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define PCG_CK(call)                                                        \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess)                                              \
            return ::pcgamg::cuda_fail(e_, #call, __FILE__, __LINE__);      \
    } while (0)
#define PCG_TRY(x)              \
    do {                        \
        int s_ = (x);           \
        if (s_) return s_;      \
    } while (0)
#define PCG_LAUNCH_CK() PCG_CK(cudaGetLastError())

// -------------------------------------------- programmatic dependent launch
// A solve kernel launched with launch_k(pdl = true, ...) may be scheduled
// while the kernel before it on the stream is still running. It calls
// pdl_enter() first: that waits until the preceding kernel has completed and
// its writes are visible, then lets the next kernel be scheduled. So the
// order of memory effects is that of plain stream order; only the launch
// and block scheduling of the next kernel overlap the tail of this one.
// Without the launch attribute both instructions return at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// A kernel that reads static data before pdl_enter() passes every pointer to
// data the preceding kernel wrote through after_wait() once pdl_enter() has
// returned: the empty volatile asm stays after the wait (volatile asms keep
// their order) and the pointer it yields is unknown to the compiler before
// it, so no read-only-path load through it can be hoisted above the wait.
template <typename T>
__device__ __forceinline__ T *after_wait(T *p) {
    asm volatile("" : "+l"(p));
    return p;
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// -------------------------------------------------------------- allocator
// Device allocations of one handle: every pointer is tracked with its size
// so the handle can free everything and enforce its byte budget.
struct Mem {
    cudaStream_t stream = nullptr;
    size_t bytes = 0, peak = 0, budget = 0;
    bool dry = false;  // count requests (rounded as real ones) without allocating
    std::unordered_map<void *, size_t> live;
    int alloc_bytes(void **p, size_t bytes);
    void release(void *p);
    void release_all();
};

template <class T>
inline int alloc(Mem &m, T **p, size_t count) {
    return m.alloc_bytes(reinterpret_cast<void **>(p), (count > 0 ? count : 1) * sizeof(T));
}
template <class T>
inline void release(Mem &m, T *&p) {
    if (p) m.release(p);
    p = nullptr;
}

// ------------------------------------------------------------ data layout
struct DevCSR {
    int n = 0;
    int64_t nnz = 0;
    int32_t *rp = nullptr, *ci = nullptr;
    double *v = nullptr;
};

// Sliced ELL with slice height 32: entry k of row 32*s + lane lives at
// sptr[s] + 32*k + lane; rows shorter than the slice width are padded with
// their own index and a zero value. One warp streams one slice.
// First pattern entry of a slice whose rows do not share one offset
// pattern (no stored offset takes this value: 16-bit offsets satisfy
// |col - row| < 2^15, and 32-bit ones are row differences of int32 indices
// inside [0, n)).
template <typename IDX>
constexpr IDX kNoPattern = sizeof(IDX) == 2 ? (IDX)INT16_MIN : (IDX)INT32_MIN;

struct Sell {
    int n = 0, nslices = 0;
    int64_t nnz_pad = 0;
    int32_t *sptr = nullptr;   // nslices + 1 element offsets
    int32_t *col = nullptr;
    int16_t *col16 = nullptr;  // col - row when every |col - row| < 2^15, else null
    double *v64 = nullptr;
    float *v32 = nullptr;
    // Shared offset patterns (null when no slice of the level has one). A slice whose rows
    // all take their columns from one offset pattern (i + o_0 < i + o_1 <
    // ...) is stored in pattern order, each row's absent offsets as explicit
    // zeros, and upat[sptr[s] / 32 + k] = o_k holds the pattern once for the
    // slice; any other slice has upat[sptr[s] / 32] = kNoPattern. The
    // pattern has the column type: upat16 beside col16, else upat. col and
    // col16 stay complete, so a kernel may read either form.
    int32_t *upat = nullptr;
    int16_t *upat16 = nullptr;
    int64_t uniform_slices = 0, uniform_entries = 0;
};

struct Level {
    DevCSR A;
    Sell S;
    double *dinv = nullptr;   // 1 / sum_j |a_ij|
    float *dinv32 = nullptr;
    double *w = nullptr;      // the vector w of this level
    // transfer to level l+1 (unused on the coarsest level)
    int nc = 0;
    int32_t *agg = nullptr;   // composed aggregate map, -1 = left out
    double *p = nullptr;      // composed tentative-prolongator weight
    float *p32 = nullptr;
    int32_t *rptr = nullptr;  // members of each coarse row: rptr[nc+1], ridx[...]
    int32_t *ridx = nullptr;
    float *v32csr = nullptr;  // float32 copy of A.v (CSR order), for the Gauss-Seidel sweeps
    // smoothed aggregation (amg_params.smoothed): the explicit prolongator P
    // (n_l x n_{l+1}, columns sorted) and its transpose Pt (rows of each
    // column in increasing order), float64 and float32 values; ones64/ones32
    // stand in for the tentative weight in the down sweep, which then leaves
    // the plain residual b - A xpre for the restriction by P^T
    DevCSR P, Pt;
    float *P32 = nullptr, *Pt32 = nullptr;
    double *ones64 = nullptr;
    float *ones32 = nullptr;
    // two-phase Gauss-Seidel sweeps (blocks of at most 32 rows): for the
    // forward [0] and backward [1] pass, each row's in-block entries that the
    // pass has already updated (j < r in the block, resp. j > r), width
    // gs_w[d] per row (column -1 pads), storage order; gs_w[d] < 0: the level
    // sweeps with one thread per block instead. gs_acc: per-row sums of the
    // other entries (phase one of a sweep).
    int gs_w[2] = {-1, -1};
    int32_t *gs_ci[2] = {nullptr, nullptr};
    double *gs_v64[2] = {nullptr, nullptr};
    float *gs_v32[2] = {nullptr, nullptr};
    double *gs_acc = nullptr;
    std::vector<int32_t *> pass_agg;
    std::vector<int> pass_n;  // rows entering pass k; pass_n[npass] = nc
    // V-cycle work vectors: right-hand side, solution, restriction input,
    // D^-1 b (xpre) and the prolongated guess (xp)
    double *b64 = nullptr, *x64 = nullptr, *t64 = nullptr, *xpre64 = nullptr, *xp64 = nullptr;
    float *b32 = nullptr, *x32 = nullptr, *t32 = nullptr, *xpre32 = nullptr, *xp32 = nullptr;
    // Launch shape of this level's down and up phases (levels >= 1), per
    // V-cycle precision [0 float, 1 double] and phase [0 down, 1 up]:
    // bit 0 = rows load 16 entries per chunk (else 4), bit 1 = one thread per
    // row (else one wave of resident blocks, grid-stride), bit 2 = one fused
    // launch (down sweep + restriction by aggregate; prolongation formed per
    // gathered entry inside the post sweep) instead of two; the value 8 =
    // rows read by 4 lanes each (separate launches). Set by setup to
    // the fixed rule (16-entry chunks up to kSmallRows rows, one thread per
    // row, separate launches) and by amg_autotune to the fastest measured
    // shape. The shape never changes a result: every shape forms the same
    // values and sums a row's entries in storage order.
    unsigned char shape[2][2] = {{0, 0}, {0, 0}};
};

// Device-resident Krylov state; every scalar of the iteration lives here so
// that an iteration needs no host round trip.
struct Ctl {
    double bnorm;        // ||b||
    double rho, rho_old; // r.z
    double pq, pq_old;   // p.Ap
    double zq;           // z . q_old (FCG)
    double alpha, beta;
    double rel;          // ||r|| / ||b|| of the last update
    double true_rel;     // ||b - A x|| / ||b|| of the last check
    double rtol;
    int iter;            // V-cycles applied
    int maxit;
    int mode;
    int flex;            // FCG(1) beta in either mode (iterative coarsest solve)
    int restart;         // next direction is p = z
    int check;           // recursive residual met rtol: form the true one
    int done;            // 1 converged, 2 error
    int status;          // AMG_* code once done
    int bodies;          // executions of the graph's loop body (2 iterations each)
    unsigned int counter[8];  // last-block-done counters of the reducing kernels
};

// Iterative coarsest solve (flexible CG + block-Jacobi with ILU(1) blocks of
// kCoarseBlock rows): per-block dense data built by setup / refresh.
struct CoarseIter {
    int nb = 0;               // blocks (the last one may be ragged)
    double *F = nullptr;      // ILU(1) factors, 32 x 32 per block, row-major: L strictly below the
                              // diagonal (unit diagonal implied), U on and above; 0 outside the kept
                              // pattern and on rows past n_L
    double *Minv = nullptr;   // (L_b U_b)^{-1}, k-major: Minv[b*1024 + 32k + i] = (M_b^{-1})_{ik};
                              // identity on rows past n_L
    int *zero = nullptr;      // a device int holding 0 ("outer solve running") for amg_coarse_solve
};

// Device state of one iterative coarsest solve over K <= 32 columns.
struct CCtl {
    double bn[32], rho[32], pq[32], alpha[32], beta[32];
    int active[32], its[32];
    int any;                  // some column still iterating
    unsigned counter[2];      // last-block tickets
};

// Work vectors of the iterative coarsest solve: (32 nb) x K row-major.
struct CoarseWS {
    int K = 0, grid = 0, grid_q = 0;   // blocks of the block-local kernels and of the SpMV
    double *x = nullptr, *r = nullptr, *z = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;
    double *partials = nullptr;        // 3 K max(grid, grid_q) doubles
    CCtl *ctl = nullptr;
};

// One level of the fused small-level tail of the V-cycle (device copy).
// Device-resident state of a multi right-hand-side solve (K <= 32 columns).
struct CtlM {
    double bnorm[32], rho[32], rho_old[32], pq[32], pq_old[32], alpha[32], beta[32], rel[32], true_rel[32];
    double rtol;
    int iter[32], active[32], restart[32], check[32], status[32];
    int pending[32];     // column awaits its first residual (new right-hand side)
    int k, K, maxit, mode, iter_all, any_check, done, bodies;
    int flex;            // FCG(1) beta in either mode (iterative coarsest solve)
    unsigned int counter[8];
};

// Per-level n_l x K work blocks of the multi-column V-cycle.
struct MultiLevel {
    float *b32 = nullptr, *x32 = nullptr, *t32 = nullptr, *xpre32 = nullptr, *xp32 = nullptr;
    double *b64 = nullptr, *x64 = nullptr, *t64 = nullptr, *xpre64 = nullptr, *xp64 = nullptr;
};

struct MultiWS {
    int K = 0, hist_cap = 0, grid = 0;
    double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    float *r32 = nullptr;
    std::vector<MultiLevel> lev;
    double *bL = nullptr;
    CoarseWS cws;                          // iterative coarsest solve (when the hierarchy uses it)
    int flex = 0;                          // the hierarchy's V-cycle is flexible (iterative coarsest solve)
    double *partials = nullptr;
    CtlM *ctl = nullptr;
    CtlM *ctl_host = nullptr;
    double *hist = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraph_t step_graph = nullptr;     // fixed chunk of iterations (serving)
    cudaGraphExec_t step_exec = nullptr;
    int step_iters = 0, step_mode = -1;
};

// A whole-solve while node whose body is captured after the outer capture.
struct PendingBody {
    struct ::amg_hier *h = nullptr;
    int mode = 0;
    cudaGraph_t body = nullptr;
    cudaGraphConditionalHandle hc = 0;
};

}  // namespace pcgamg

struct amg_hier {
    int device = 0;
    int mode = AMG_MODE_PCG64;
    amg_params prm{};
    pcgamg::Mem mem;
    std::vector<pcgamg::Level> lev;
    int nL = 0;
    double *Ainv = nullptr;   // inverse of the coarsest matrix, row-major (dense coarsest solve)
    // iterative coarsest solve (Sec. 3.1: FCG + block-Jacobi ILU(1)), used
    // when coarse_iter = 1; the V-cycle is then not a fixed operator and
    // both modes run the flexible FCG(1) recurrence
    int coarse_iter = 0;
    int smoothed = 0;         // smoothed-aggregation prolongators (amg_params.smoothed)
    pcgamg::CoarseIter cit;
    pcgamg::CoarseWS cws;
    double *bL = nullptr;     // coarsest right-hand side in float64
    // Krylov workspace (level-0 length)
    double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *q = nullptr, *p = nullptr;
    float *r32 = nullptr;        // float32 copy of r read by the float32 V-cycle
    double *partials = nullptr;  // per-block partial sums (several slots)
    double *hist = nullptr;      // device history, maxit_cap + 1
    int hist_cap = 0;
    pcgamg::Ctl *ctl = nullptr;
    pcgamg::Ctl *ctl_host = nullptr;  // pinned mirror
    int nblk = 0;                // largest level-0 grid (sizes the partial sums)
    int grid32 = 0, grid64 = 0, gridv = 0;  // one wave of the float32 sweeps, float64 sweeps, vector kernels
    int wave[2][2][2] = {};      // blocks in one wave: [float, double][down, post][4- or 16-entry chunks]
    double last_true_rel = 0.0;
    double setup_ms[4] = {0, 0, 0, 0};
    // kernel timing (amg_profile)
    static constexpr int kKinds = 8;
    int profile = 0;
    std::vector<cudaEvent_t> ev;      // pool: pairs per kind per iteration of a chunk
    int ev_used = 0;
    int ev_kind[256] = {0};
    double prof_ms[kKinds] = {0};
    int64_t prof_n[kKinds] = {0};
    // per-level V-cycle spans: [level][down, up, coarsest]
    static constexpr int kMaxProfLevels = 32;
    double lev_ms[kMaxProfLevels][3] = {};
    int64_t lev_n[kMaxProfLevels][3] = {};
    int64_t launches = 0;
    // whole-solve CUDA graph per mode: prefix kernels, then a device-side
    // while loop whose body runs two iterations
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int graph_prefix_kernels = 0;
    int graph_body_kernels[2] = {0, 0};
    // the same without the shared-memory tail (for solves that share the
    // device: serving lanes; batch graphs capture that way too)
    cudaGraphExec_t gexec_nt[2] = {nullptr, nullptr};
    int graph_body_kernels_nt[2] = {0, 0};
    int no_tail = 0;  // set while capturing a solve that must not use the tail
    int invalid = 0;  // set while a refresh is incomplete (or failed): solves are refused
    // smoother: gs_nu = 0 is the one-sweep l1-Jacobi of the setup; otherwise
    // gs_nu sweeps of l1 hybrid Gauss-Seidel over gs_blocks row blocks per
    // level (amg_set_smoother)
    int gs_nu = 0, gs_blocks = 0;
    int gs_fused = 1;  // one-launch warp sweeps where the blocks fit the slices (PCGAMG_GS_FUSED=0: off)
    double refresh_ms = 0;  // host time of the last amg_refresh
    int use_graph = 1;
    int no_col16 = 0;
    int no_uniform = 0;  // PCGAMG_UNIFORM=0: no shared offset patterns on level 0
    int pdl = 1;  // programmatic dependent launch between solve kernels
    int graph_gen = 0;       // bumped whenever captured graphs go stale
    // shared-memory cluster tail: levels tail_first..L in one cluster launch,
    // per V-cycle precision [float, double]
    int tail_first[2] = {0, 0};  // 0 = no tail (every level launched separately)
    int tail_ctas[2] = {0, 0};   // CTAs of the cluster
    pcgamg::SmemTailPlan tail_plan[2] = {};   // [float, double] V-cycle
    unsigned char *tail_blob[2] = {nullptr, nullptr};
    size_t tail_smem[2] = {0, 0};
    // multi right-hand-side solves
    pcgamg::MultiWS multi;
    int multi_k = 0;
    int multi_status[32] = {0};
    double multi_true_rel[32] = {0};
};

namespace pcgamg {
int setup_impl(amg_hier *h, const amg_csr *A, const amg_params *prm, cudaStream_t s);
int refresh_impl(amg_hier *h, const amg_csr *A, cudaStream_t s);
int set_smoother_impl(amg_hier *h, int nu, int nblocks, cudaStream_t s);
int gs_rows(int n, int nblocks);
int fill_gs_parts(Level &lv, int nblocks, cudaStream_t s);
int refresh_smem_tail(amg_hier *h);
int solve_impl(amg_hier *h, const double *b, double *x, double rtol, int maxit, int *iters,
               double *res_hist, cudaStream_t s);
int alloc_solve_workspace(amg_hier *h);
int set_profile(amg_hier *h, int enable);
void free_profile(amg_hier *h);
int solve_multi_impl(amg_hier *h, int k, const double *B, double *X, double rtol, int maxit, int *iters,
                     double *res_hist, cudaStream_t s);
void free_multi(amg_hier *h);
int solve_prepare(amg_hier *h, int mode, int maxit);
void drop_graphs(amg_hier *h);
int autotune_impl(amg_hier *h, cudaStream_t s, int reps, int *changed);
int setup_smem_tail(amg_hier *h);
template <typename T>
int launch_smem_tail(amg_hier *h, cudaStream_t s);
int solve_launch(amg_hier *h, int mode, const double *b, const double *x0, double rtol, int maxit, cudaStream_t s);
int solve_collect(amg_hier *h, int mode, double *x, cudaStream_t s, int *status, int *iters, double *true_rel,
                  int64_t *kernels);
int mws_alloc(amg_hier *h, Mem &M, MultiWS &W, int K, int hist_cap, int which);
bool gs_multi_ok(const amg_hier *h);
void mws_free(Mem &M, MultiWS &W);
size_t mws_bytes(amg_hier *h, int K, int hist_cap, int which);
int mws_reset(MultiWS &W, int mode, double rtol, int maxit, cudaStream_t s);
int mws_put_column(MultiWS &W, int c, const double *b_dev, const double *x_dev, int n, cudaStream_t s);
int mws_admit(amg_hier *h, MultiWS &W, int mode, unsigned mask, cudaStream_t s);
int mws_iterate(amg_hier *h, MultiWS &W, int mode, int iterations, cudaStream_t s, int launch);
int capture_solve_prefix(amg_hier *h, int mode, cudaStream_t cs, PendingBody *pb, int *prefix_k);
int capture_solve_body(const PendingBody &pb, cudaStream_t s, int *body_k);
int ensure_hist(amg_hier *h, int maxit);
int scan_counts(Mem &M, const int32_t *in, int32_t *out, int64_t n, int32_t *total_host, cudaStream_t s);
// smoothed aggregation (csrc/smoothed.cu)
int build_smoothed(amg_hier *h, Level &lv, int nc, DevCSR *out, cudaStream_t s);
// iterative coarsest solve (csrc/coarse.cu)
int coarse_iter_build(amg_hier *h, cudaStream_t s);
int cws_alloc(amg_hier *h, Mem &M, CoarseWS &W, int K);
void cws_free(Mem &M, CoarseWS &W);
int coarse_iter_launches(const amg_hier *h);
template <typename TO>
int launch_coarse_iter(amg_hier *h, CoarseWS &W, const double *bL, TO *xL, const int *outer_done,
                       const int *outer_live, cudaStream_t s);
}  // namespace pcgamg
