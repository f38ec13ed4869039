/*
 * pcgamg: PCG preconditioned by one aggregation-based AMG V-cycle per
 * iteration, on one GB300 GPU (sm_103a).
 *
 * Method: arxiv 2210.16660, Sec. 3.1 (AMG as a stationary iteration used as
 * a Krylov preconditioner; Galerkin coarse operators A_{l+1} = P_l^T A_l P_l;
 * the V-cycle of Eq. (multiplicative composition); coarsening by compatible
 * weighted matching, Eq. (weights) and Eq. (approximatematch); the tentative
 * prolongator of Eq. (prolongator); aggregates of size up to 2^n_pass by
 * multiplying pairwise prolongators) and Sec. 5 (flexible CG, stop on the
 * Euclidean norm of the relative residual, warm start from the previous
 * time step). Sec. 4: the preconditioner is built once and applied inside
 * the Krylov driver through a single call.
 *
 * Variant implemented (fixed by the library, not by the paper): l1-Jacobi
 * smoothing, one pre- and one post-sweep (M = diag(sum_j |a_ij|)) by default
 * (the paper's hybrid Gauss-Seidel on request, amg_set_smoother); the
 * tentative prolongator without the smoothing step; on the coarsest level a
 * dense float64 direct solve up to 4096 rows, and above that (or on request)
 * the paper's own coarsest solver, flexible CG preconditioned by
 * block-Jacobi with ILU(1) blocks.
 *
 * Conventions for every entry point:
 *  - All functions return an int status (AMG_OK = 0 or an AMG_ERR_* code);
 *    none aborts. amg_last_error() returns a message for the calling thread.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). All device work of a call is ordered on that stream.
 *  - Vectors may be host or device pointers; the library tells them apart
 *    with cudaPointerGetAttributes. Host vectors are copied in and out
 *    inside the call (the call then returns after the copy back).
 *  - The library allocates its own device memory through the allocator set
 *    by amg_set_allocator (cudaMalloc/cudaFree by default). No call frees
 *    or writes caller memory other than its documented outputs.
 *  - All entry points are safe to call from several host threads on
 *    different handles; one handle must not be used by two calls at once.
 */
#ifndef PCGAMG_H
#define PCGAMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status */
#define AMG_OK 0
#define AMG_ERR_ARG 1       /* bad sizes, unsorted/unsymmetric CSR, bad handle */
#define AMG_ERR_OOM 2       /* allocation failed or hbm_budget exceeded */
#define AMG_ERR_BREAKDOWN 3 /* r.z <= 0 or p.Ap <= 0, or coarsest not SPD */
#define AMG_ERR_NOCONV 4    /* maxit V-cycles without meeting rtol; x = last iterate */
#define AMG_ERR_NAN 5       /* NaN or Inf in the iteration */
#define AMG_ERR_CUDA 6      /* a CUDA runtime call failed */
#define AMG_ERR_TIMEOUT 7   /* reserved: no kernel waits on another, no call returns it */
#define AMG_ERR_COARSE 8    /* the dense coarsest solve was asked for (or a single level
                               was left) with more than 4096 rows */
#define AMG_ERR_BUSY 9      /* serving: the request queue is full */
#define AMG_ERR_MATCH 10    /* setup: a matching pass did not finish within 20000 rounds */

/* Coarsest solver (Sec. 3.1). AUTO: the dense direct solve when the coarsest
 * level has at most 4096 rows, else the iterative one. DENSE: the dense
 * direct solve (AMG_ERR_COARSE above 4096 rows). ITER: flexible CG
 * preconditioned by block-Jacobi over blocks of 32 consecutive rows, each
 * block solved by its ILU(1) factorization (level-of-fill 1), started from
 * x = 0 and stopped when ||r|| <= coarse_tol ||b|| or after coarse_maxit
 * iterations (the paper: a reduction of three orders of magnitude or 30
 * iterations). With ITER in use the V-cycle is no longer a fixed linear
 * operator, so both modes run the flexible FCG(1) recurrence. */
#define AMG_COARSE_AUTO 0
#define AMG_COARSE_DENSE 1
#define AMG_COARSE_ITER 2

/* Precision of the V-cycle (Sec. 5 uses flexible CG around the preconditioner). */
#define AMG_MODE_PCG64 0    /* float64 V-cycle, plain PCG */
#define AMG_MODE_FCG32 1    /* float32 V-cycle (values, smoother, transfers) inside
                               float64 FCG(1); the coarsest solve stays float64 */

typedef struct amg_hier *amg_handle;

/* Square sparse matrix in CSR form (the matrix format of Sec. 4).
 * Requirements: row_ptr[0] = 0, row_ptr nondecreasing, row_ptr[n] = nnz;
 * column indices in [0, n), strictly increasing within a row; every row has
 * its diagonal entry and it is > 0; the matrix is exactly symmetric (values
 * equal bit for bit), as symmetric FE assembly gives. nnz < 2^31.
 * on_device = 1 when the three arrays are device pointers. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int32_t *row_ptr;
    const int32_t *col;
    const double *val;
    int on_device;
} amg_csr;

/* Hierarchy options (cf. Table 1 of the paper for the paper's own set). */
typedef struct {
    int coarse_max;   /* stop coarsening when a level has <= this many rows (200) */
    int n_pass;       /* pairwise matching passes per level, |G| <= 2^n_pass (2) */
    int max_levels;   /* at most this many levels, coarsest included (30) */
    int mode;         /* AMG_MODE_PCG64 or AMG_MODE_FCG32 for pcg_solve (PCG64) */
    size_t hbm_budget;/* bytes the handle may allocate; 0 = no limit */
    int coarse_solver;/* AMG_COARSE_AUTO, _DENSE or _ITER (AUTO) */
    int coarse_maxit; /* iterative coarsest solve: at most this many iterations, 1..1000
                         (30; 0 = 30) */
    double coarse_tol;/* iterative coarsest solve: stop at ||r|| <= coarse_tol ||b||, in
                         [0, 1) (1e-3; 0 = 1e-3) */
    int smoothed;     /* 0: tentative prolongator P_hat (restriction and prolongation
                         through the aggregate map); 1: smoothed aggregation,
                         P = (I - omega D^-1 A) P_hat with omega = 1 / ||D^-1 A||_inf and
                         D = diag(A), coarse matrices P^T A P (Sec. 3.1) (0) */
} amg_params;

/* Fill p with the defaults listed above. */
void amg_default_params(amg_params *p);

/* Device allocator used for every allocation made after the call (process
 * wide). alloc returns NULL on failure. Passing NULL functions restores
 * cudaMalloc/cudaFree. */
typedef void *(*amg_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*amg_free_fn)(void *ptr, void *stream, void *ctx);
int amg_set_allocator(amg_alloc_fn alloc, amg_free_fn dealloc, void *ctx);

/* Build the AMG hierarchy of A on the current device (Sec. 3.1).
 * All steps run on the GPU: l1 diagonals, Eq. (weights), the matching
 * (locally-dominant, equal to the greedy matching under a strict total
 * order), aggregates and tentative prolongator weights, pairwise Galerkin
 * products P^T A P, sliced-ELL copies in float64 and float32, and the dense
 * coarsest inverse, or the ILU(1) factors of the coarsest level's blocks and
 * their dense inverses (iterative coarsest solve). The level sizes are read
 * back once per pass.
 * A is copied; the caller may free it after the call returns.
 * Errors: AMG_ERR_ARG (bad CSR or parameters; ITER with a single level),
 * AMG_ERR_OOM, AMG_ERR_BREAKDOWN (coarsest not SPD, or an ILU(1) pivot that
 * is not positive), AMG_ERR_COARSE, AMG_ERR_MATCH, AMG_ERR_CUDA. *out is
 * NULL on error. */
int amg_setup(const amg_csr *A, const amg_params *p, void *stream, amg_handle *out);

/* Partial reuse of the hierarchy (Sec. 4: when the mesh topology stays and
 * only the coefficients change, the same prolongators/restrictors rebuild the
 * hierarchy and its smoothers). A holds new values of the finest matrix on
 * exactly the sparsity pattern h was built on (same n, nnz, row pointers and
 * columns; host or device, as in amg_setup; copied, the caller keeps it).
 * Every pass keeps its aggregates and tentative-prolongator weights (they do
 * not depend on the values); the Galerkin products, the l1 diagonals, the
 * float32 copies and the dense coarsest inverse are formed again, with the
 * arithmetic of amg_setup, so amg_refresh(h, A0) with the values h was built
 * on reproduces h bit for bit. Device arrays keep their addresses: solve
 * graphs, batches and servers built on h stay valid. The call synchronises
 * stream and must not overlap a solve on h.
 * Errors: AMG_ERR_ARG (NULL, other sizes or pattern, invalid or not exactly
 * symmetric values: h is unchanged), AMG_ERR_BREAKDOWN (coarsest matrix not
 * SPD), AMG_ERR_OOM, AMG_ERR_CUDA. After an error other than AMG_ERR_ARG,
 * solves on h (single, multi-column, batched, served) return AMG_ERR_ARG
 * until a later amg_refresh succeeds. */
int amg_refresh(amg_handle h, const amg_csr *A, void *stream);

/* Smoother of h's V-cycle (Sec. 3.1). nu = 0: one l1-Jacobi sweep before and
 * after the coarse correction (the setup's default, M = diag(sum_j |a_ij|)).
 * nu in 1..64: nu sweeps of the l1 hybrid Gauss-Seidel method the paper
 * smooths with (it uses nu = 4): block Jacobi over nblocks contiguous row
 * blocks per level, ceil(n_l / nblocks) rows each (nblocks = 0: one row per
 * block), each block solved by a forward Gauss-Seidel pass before and a
 * backward pass after the coarse correction; d_i = a_ii + sum of |a_ij| over
 * j outside i's block (the l1 form, no damping). One row per block and one
 * sweep give the values of the default. Re-forms every level's smoother
 * diagonal (and a float32 CSR copy of the level matrices for the sweeps);
 * the next solve recaptures its graph; the shared-memory cluster tail is not
 * used while nu > 0. In the float32 V-cycle, where a level's blocks divide
 * its 32-row slices (and no row has more than 8 already-updated in-block
 * entries), a sweep is one launch, one warp per slice; otherwise two. Single and batched solves take nu > 0;
 * multi-column and served solves run the l1-Jacobi kernels only and return
 * AMG_ERR_ARG for such a handle; amg_autotune returns AMG_OK without changes
 * for it. Synchronises stream.
 * Errors: AMG_ERR_ARG (NULL, nu or nblocks out of range), AMG_ERR_OOM,
 * AMG_ERR_CUDA. */
int amg_set_smoother(amg_handle h, int nu, int nblocks, void *stream);

/* Host time (ms) of the last successful amg_refresh of h. */
int amg_refresh_time(amg_handle h, double *ms);

/* Select the solve mode of a handle (AMG_MODE_PCG64 / AMG_MODE_FCG32). */
int amg_set_mode(amg_handle h, int mode);

/* Solve A x = b by PCG (mode PCG64) or FCG(1) (mode FCG32) preconditioned by
 * one V-cycle per iteration (Sec. 3.1, Sec. 5).
 * b: n values (host or device). x: n values, initial guess on entry (the
 * warm start of Sec. 5), solution on exit. Stops when the recursive residual
 * satisfies ||r_k|| / ||b|| <= rtol and the true residual b - A x does too;
 * if the true one does not, r is replaced by it and the recurrence restarts.
 * iters (may be NULL): V-cycles applied. res_hist (may be NULL, host or
 * device, maxit+1 values): ||r_k|| / ||b|| for k = 0..iters.
 * ||b|| = 0 returns x = 0, iters = 0. Returns AMG_ERR_NOCONV after maxit
 * iterations (x holds the last iterate), AMG_ERR_BREAKDOWN, AMG_ERR_NAN. */
int pcg_solve(amg_handle h, const double *b, double *x, double rtol, int maxit,
              int *iters, double *res_hist, void *stream);

/* k right-hand sides at once (1 <= k <= 32), sharing the hierarchy: each
 * stored entry of every level is read once per sweep for all columns (the
 * multi-vector form of the same method). B and X are n x k row-major
 * (column c of row i at [i*k + c]), host or device; X holds the initial
 * guesses on entry and the solutions on exit. Each column runs its own
 * recurrence (PCG or FCG(1) per amg_set_mode), stops on its own
 * ||r_c|| / ||b_c|| <= rtol (confirmed on the true residual) and keeps its x
 * while the others go on. iters: k values (host, may be NULL). res_hist
 * (may be NULL, host or device): k rows of maxit+1 values, column c's
 * history at [c*(maxit+1)]. Returns AMG_OK when every column converged, else
 * the status of the first column that did not (per-column statuses from
 * amg_multi_info). Needs a hierarchy with at least two levels. */
int pcg_solve_multi(amg_handle h, int k, const double *B, double *X, double rtol, int maxit, int *iters,
                    double *res_hist, void *stream);

/* Per-column outcome of the last pcg_solve_multi on h: *k columns, status[c]
 * (AMG_* code) and true_rel[c] = ||b_c - A x_c|| / ||b_c||. Arrays of 32
 * (host) or NULL. */
int amg_multi_info(amg_handle h, int *k, int *status, double *true_rel);

/* Batched solve of independent systems, each with its own hierarchy (own
 * handle; handles may differ in size and mode). amg_batch_create fixes the
 * list of handles; pcg_solve_batch then solves system i: A_i x_i = B[i]
 * (x_i: initial guess in X[i], solution on exit) for all i in one CUDA-graph
 * launch whose branches run concurrently on the GPU, each with its own
 * device-side iteration loop. Each system's result equals that handle's own
 * pcg_solve bit for bit. B[i], X[i]: host or device, n_i values each.
 * iters, status: m values each (host, may be NULL). Returns AMG_OK when all
 * systems converged, else the first failing status. A handle must not be
 * destroyed while a batch holding it exists, nor used by two calls at once. */
typedef struct amg_batch_s *amg_batch;
int amg_batch_create(int m, const amg_handle *hs, amg_batch *out);
int pcg_solve_batch(amg_batch b, const double *const *B, double *const *X, double rtol, int maxit, int *iters,
                    int *status, void *stream);
void amg_batch_destroy(amg_batch b);

/* ---------------------------------------------------------------------------
 * Serving: pressure solves of many time steps over meshes whose hierarchies
 * stay resident on the device. The paper builds the hierarchy of a fixed
 * mesh once and reuses it for every time step's solve (Sec. 1, Sec. 4), each
 * solve starting from the previous step's pressure (Sec. 5); it has no
 * serving layer of its own, this is the way to run many such solves at once
 * on one GPU.
 *
 * A request is (mesh, b, x0): solve A_mesh x = b from x0 to
 * ||b - A x|| / ||b|| <= rtol with the server's mode. Every mesh gets engines
 * of `slots` right-hand-side slots (the kernels of pcg_solve_multi) and, with
 * `solo`, a whole-solve lane (the kernels of pcg_solve, one graph launch per
 * solve, on the hierarchy's own vectors). A queued request goes to its
 * mesh's lane when the lane is idle, else to a free engine slot; between
 * chunks of `chunk` iterations the host hands finished requests back and
 * starts queued ones in the freed slots, while the other slots carry on
 * where they were (continuous batching). Lanes and engines run on their own
 * streams and overlap on the device. A request's result depends only on its
 * own (mesh, b, x0), the server parameters and the kind of place it ran in
 * (reported by amg_server_result), not on what else is running: in a lane it
 * equals pcg_solve's result bit for bit; in a slot it is the same bit for bit
 * as in any other slot or mix and equals column c of pcg_solve_multi with
 * the same K. Both meet rtol; they differ by summation order only.
 *
 * Memory: the resident hierarchies (all device bytes each handle holds) plus
 * every engine fit in hbm_budget bytes (0: the hierarchies' bytes plus the
 * free device memory less 1 GiB). amg_serve_plan decides the engines per
 * mesh; a mesh whose hierarchy and one engine do not fit gets no engine and
 * its requests are refused with AMG_ERR_OOM.
 *
 * The server is driven by one host thread (submit / progress / result); a
 * mesh's handle must stay alive and must not be used by other calls while
 * the server exists.
 * ------------------------------------------------------------------------- */
typedef struct amg_server_s *amg_server;

typedef struct {
    int mode;          /* AMG_MODE_FCG32 or AMG_MODE_PCG64, for every request */
    int slots;         /* right-hand sides per engine: 4, 8, 16 or 32 */
    int max_engines;   /* engines per mesh, at most (>= 1) */
    int chunk;         /* iterations per device step between host visits (>= 1) */
    int queue_cap;     /* requests waiting for a slot, at most (>= 0) */
    int maxit;         /* iterations per request, at most */
    double rtol;       /* relative residual target per request */
    size_t hbm_budget; /* device bytes for hierarchies plus engines; 0: see above */
    int solo;          /* 1: a whole-solve lane per admitted mesh (no extra memory) */
    int batch_min;     /* with a lane: an idle engine starts once this many requests wait (>= 1) */
    int lane_priority; /* 1: lanes on the highest stream priority, engines on the lowest */
} amg_server_params;

/* FCG32, 4 slots, 2 engines per mesh, chunk 4, queue 4096, maxit 1000,
 * rtol 1e-8, budget 0, solo 1, batch_min 3, lane_priority 0. */
void amg_server_default_params(amg_server_params *p);

/* Engine plan (host only, no device call). Mesh i needs resident[i] bytes for
 * its hierarchy and engine_bytes[i] per engine. In mesh order, a mesh is
 * admitted with one engine if its hierarchy and one engine fit in what is
 * left of budget; then engines are added one at a time to the admitted mesh
 * with the largest load[i] / engines[i] (ties: lowest i; load NULL: all 1)
 * that still fits and has fewer than max_engines. engines: m values out
 * (0 = not admitted); *total (may be NULL): bytes planned. Returns AMG_OK if
 * at least one mesh was admitted, AMG_ERR_OOM if none, AMG_ERR_ARG on bad
 * arguments. */
int amg_serve_plan(int m, const size_t *resident, const size_t *engine_bytes, const double *load, size_t budget,
                   int max_engines, int *engines, size_t *total);

/* Creates a server over m resident hierarchies (distinct handles with at
 * least two levels). load: m relative request loads for the plan (NULL: all
 * equal). Allocates every engine up front. Errors: AMG_ERR_ARG, AMG_ERR_OOM
 * (nothing fits, or an allocation failed), AMG_ERR_CUDA. */
int amg_server_create(const amg_server_params *p, int m, const amg_handle *meshes, const double *load,
                      amg_server *out);

/* Plan of one mesh: engines, slots per engine, bytes per engine, resident
 * hierarchy bytes (each pointer may be NULL). */
int amg_server_mesh_info(amg_server s, int mesh, int *engines, int *slots, size_t *engine_bytes,
                         size_t *resident_bytes);

/* Budget in use and state: budget, planned bytes, requests waiting, requests
 * in slots, kernels launched so far (each may be NULL). */
int amg_server_info(amg_server s, size_t *budget, size_t *used, int *queued, int *running, int64_t *launches);

/* Queues a request. b, x0 (n values, host or device) must stay valid until
 * the request has started (its first progress call that admits it); x (n
 * values, host or device) receives the solution when it finishes and must
 * stay valid until then. *ticket names it in amg_server_result. Errors:
 * AMG_ERR_ARG, AMG_ERR_OOM (mesh not admitted), AMG_ERR_BUSY (queue full;
 * nothing queued). */
int amg_server_submit(amg_server s, int mesh, const double *b, const double *x0, double *x, int64_t *ticket);

/* One visit of every engine: engines whose chunk has finished hand back their
 * finished requests (x written, result recorded), then every idle engine
 * starts queued requests in its free slots and launches its next chunk if a
 * slot is in use. wait != 0: first wait until some running chunk finishes
 * (returns at once if none is running). *finished (may be NULL): requests
 * finished by this call. */
int amg_server_progress(amg_server s, int wait, int *finished);

/* Outcome of a request. *done = 0 while it is queued or running; once it is
 * 1 the record is released and the ticket is no longer known. status: the
 * request's AMG_* code (AMG_ERR_NOCONV with x = last iterate, as pcg_solve);
 * iters; true_rel = ||b - A x|| / ||b||; lane: 0 if it ran in a whole-solve
 * lane, 1 in an engine slot; times (3 doubles, may be NULL): ms waiting in
 * the queue, ms running, ms from submit to finish. Returns AMG_ERR_ARG for an
 * unknown ticket. */
int amg_server_result(amg_server s, int64_t ticket, int *done, int *status, int *iters, double *true_rel, int *lane,
                      double *times);

/* Waits for running chunks and frees every engine (not the hierarchies). */
void amg_server_destroy(amg_server s);

/* Launch-shape tuner (no counterpart in the paper: it picks how the sweeps
 * are launched on this device, not what they compute). For every level
 * l >= 1 with sweeps, each V-cycle precision and each of the down phase
 * (down sweep + restriction) and the up phase (prolongation + post sweep),
 * it times nine launch shapes -- rows loading 4 or 16 entries per chunk,
 * times a one-wave grid-stride grid or one thread per row, times two
 * launches or one fused launch (down sweep and restriction by aggregate;
 * prolongation formed per gathered entry inside the post sweep); and rows
 * read by 4 lanes each, every entry of a row gathered at once and the sum
 * chained through the lanes in storage order -- `reps`
 * runs each (reps < 1: 1) on `stream`, and moves to the fastest when it
 * beats the current shape by more than 3%. Every shape forms the same
 * values and sums a row's entries in storage order, so solves give the same
 * bits before and after tuning; only their speed changes. The level work
 * vectors are overwritten; captured solve graphs are rebuilt on the next
 * solve. *changed (may be NULL): shapes that differ from before. Call it
 * between solves, not while a batch or server holding h is in use. */
int amg_autotune(amg_handle h, int reps, int *changed, void *stream);

/* Launch shapes of a level (4 ints: float down, float up, float64 down,
 * float64 up; bit 0 = 16-entry chunks, bit 1 = one thread per row, bit 2 =
 * fused launch; 8 = rows read by 4 lanes each, separate launches). Level
 * 0's sweeps have a fixed shape and report 0. */
int amg_level_shape(amg_handle h, int level, int *shape);

/* Sets the launch shapes of level 1..L (same 4-int layout, values 0..8);
 * for manual tuning and for tests that check every shape gives the same
 * result. Errors: AMG_ERR_ARG. */
int amg_set_level_shape(amg_handle h, int level, const int *shape);

/* True relative residual ||b - A x|| / ||b|| at the end of the last solve on h. */
double amg_last_true_residual(amg_handle h);

/* Hierarchy description: number of levels and, when the arrays are not NULL
 * (host, length >= levels), rows and stored entries per level. */
int amg_info(amg_handle h, int *levels, int64_t *n_l, int64_t *nnz_l);

/* Aggregate map of one matching pass (host output, length = rows entering
 * the pass): agg[i] = coarse index or -1 for a row left out of the coarse
 * space. pass = -1 gives the composed map of the level. *n_out receives the
 * rows entering the pass (call with agg = NULL to size the buffer), *nc_out
 * the coarse rows it produces. */
int amg_level_agg(amg_handle h, int level, int pass, int32_t *agg, int64_t *n_out,
                  int64_t *nc_out);

/* Stored layout of level l's matrix as the solve kernels read it: sliced
 * ELL with slice height *slice (32), *stored entries including padding, and
 * *index_bytes per entry (2 when every |col - row| < 2^15 so columns are kept
 * as int16 offsets from the row, else 4). Any pointer may be NULL. */
int amg_level_layout(amg_handle h, int level, int *slice, int64_t *stored, int *index_bytes);

/* Slices of level l stored with a shared offset pattern (0 with
 * PCGAMG_UNIFORM=0 in the environment at setup): the rows of such a slice
 * take their columns from one pattern of offsets i + o_k (each row's absent
 * offsets kept as explicit zeros, so a row still sums its entries in
 * increasing column order), and the V-cycle sweeps and q = A p read that
 * pattern once per slice instead of one column index per entry. On a
 * structured mesh nearly every level-0 slice has one, and most of level
 * 1's. *slices such slices, *entries their stored entries (padding
 * included). Any pointer may be NULL. Errors: AMG_ERR_ARG. */
int amg_level_pattern(amg_handle h, int level, int64_t *slices, int64_t *entries);

/* Copy level l's matrix in CSR form to host buffers (row_ptr n+1, col/val nnz). */
int amg_level_csr(amg_handle h, int level, int32_t *row_ptr, int32_t *col, double *val);

/* Smoothed prolongator of level l (amg_params.smoothed = 1; AMG_ERR_ARG
 * otherwise, and for the coarsest level) in CSR form, columns sorted: *nnz
 * stored entries; row_ptr (n_l + 1), col and val (nnz) host buffers, each may
 * be NULL (call with NULL arrays to size them). */
int amg_level_prolongator(amg_handle h, int level, int64_t *nnz, int32_t *row_ptr, int32_t *col, double *val);

/* Setup time split, milliseconds (host buffer of 4): total, matching,
 * Galerkin products, everything else. */
int amg_setup_times(amg_handle h, double *ms);

/* Kernel timing of later solves on h (enable = 1) or off (0). When on, each
 * solve records CUDA events on its stream around the level-0 kernels and
 * around the coarse-level part of the V-cycle. Adds no work to the kernels. */
int amg_profile(amg_handle h, int enable);

/* Accumulated device time (ms) and launch count per kernel kind since the
 * last read, then reset. kinds: 0 level-0 pre-smooth/residual, 1 level-0
 * post-smooth (+ r.z; with the Gauss-Seidel smoother the whole level-0 up
 * phase), 2 q = A p (+ p.q), 3 x/r update, 4 true residual, 5 levels >= 1
 * incl. restriction and coarsest solve (one span per V-cycle), 6 p = z +
 * beta p, 7 level-0 prolongation. ms and counts are host arrays of length
 * nkinds (<= 8). */
int amg_profile_read(amg_handle h, double *ms, int64_t *counts, int nkinds);

/* Per-level V-cycle time (ms) and span counts since the last read, then
 * reset (recorded while amg_profile is on). For level l, entries 3l, 3l+1,
 * 3l+2: the down phase (level l's down sweep, l >= 1, and the restriction
 * to level l+1), the up phase (prolongation to level l and its post sweep,
 * l >= 1) and the coarsest solve (on the coarsest level's entry, or on the
 * first level of the cluster tail when that is on). ms, counts: host arrays
 * of 3 nlev values (nlev <= 32), or NULL. */
int amg_profile_levels(amg_handle h, int nlev, double *ms, int64_t *counts);

/* Kernels launched by solves on h since setup (every launch, including the
 * ones that find the solve finished and return at once). */
int64_t amg_launch_count(amg_handle h);

/* r = b - A x on the finest level of h, with norms[0] = ||r||_2 and
 * norms[1] = ||b||_2, computed without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they solve, such as an application
 * that gives the whole GPU to its own memory pool, or a time-step loop that
 * cannot take the device synchronisation an allocation may cause.
 * b, x, r: device pointers to n values on the handle's device, which must
 * be the current one (r is written and must not overlap b or x); norms: 2
 * doubles, host or device (a host pointer makes the call wait for the
 * result, so a call on a stream being captured needs a device pointer).
 * Scratch: a fixed 512 KiB array inside the library (per GPU, kept until the
 * process exits) holds one partial sum pair per 256 rows, so at most
 * 8,388,608 rows are accepted; larger levels return AMG_ERR_ARG. The first
 * call on a device looks up that array's device address, so make it before
 * any stream capture. All calls share the array: calls that overlap on the
 * GPU (different streams, threads or handles) race and must be ordered by
 * the caller. Calls no cudaMalloc, cudaFree or allocating library routine.
 * Errors: AMG_ERR_ARG (NULL or host b/x/r, r overlapping b or x, another
 * current device, too many rows, host norms during a capture), AMG_ERR_CUDA. */
int amg_residual_noalloc(amg_handle h, const double *b, const double *x, double *r, double *norms,
                         void *stream);

/* Coarsest solver of h: *kind = AMG_COARSE_DENSE or AMG_COARSE_ITER (the
 * one in use), *rows = rows of the coarsest level, *blocks = its 32-row
 * ILU(1) blocks (0 for the dense solve). Any pointer may be NULL. */
int amg_coarse_info(amg_handle h, int *kind, int *rows, int *blocks);

/* ILU(1) factors of the coarsest level's blocks (iterative coarsest solve;
 * AMG_ERR_ARG otherwise), copied to the host buffer F of blocks * 1024
 * doubles: block b's local row i, column j at F[b*1024 + 32 i + j]; L
 * strictly below the diagonal (unit diagonal not stored), U on and above;
 * 0 outside the kept level-1 pattern and on rows past the last row. The
 * factorization is the level-of-fill ILU(1) in row order with every
 * operation rounded on its own, so equal inputs give these bits on any
 * device. */
int amg_coarse_factors(amg_handle h, double *F);

/* The iterative coarsest solve alone (AMG_ERR_ARG when h uses the dense
 * one): x ~ A_L^{-1} b for the coarsest matrix A_L, from x = 0, with h's
 * coarse_tol and coarse_maxit. b, x: n_L values, host or device. *iters
 * (may be NULL): iterations run. Synchronises stream; must not overlap a
 * solve on h. */
int amg_coarse_solve(amg_handle h, const double *b, double *x, int *iters, void *stream);

/* Release every device allocation of the handle (NULL is ignored). */
void amg_destroy(amg_handle h);

/* Message of the last error raised on the calling thread ("" if none). */
const char *amg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PCGAMG_H */
