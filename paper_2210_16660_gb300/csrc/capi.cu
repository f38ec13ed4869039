// C-ABI entry points of libpcgamg (declared in pcgamg.h), the allocator
// hook and the per-thread error message.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace pcgamg {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
    return e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA;
}

// ------------------------------------------------------------ allocator
static amg_alloc_fn g_alloc = nullptr;
static amg_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

int Mem::alloc_bytes(void **p, size_t n) {
    *p = nullptr;
    n = (n + 255) & ~(size_t)255;
    if (budget && bytes + n > budget) {
        set_error("device memory budget exceeded (%zu + %zu > %zu bytes)", bytes, n, budget);
        return AMG_ERR_OOM;
    }
    if (dry) {
        // Counting only: a distinct, never dereferenced address per call.
        bytes += n;
        if (bytes > peak) peak = bytes;
        *p = reinterpret_cast<void *>(bytes);
        return AMG_OK;
    }
    void *q = nullptr;
    if (g_alloc) {
        q = g_alloc(n, (void *)stream, g_alloc_ctx);
        if (!q) {
            set_error("allocator hook failed for %zu bytes", n);
            return AMG_ERR_OOM;
        }
    } else {
        cudaError_t e = cudaMalloc(&q, n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc of %zu bytes failed: %s", n, cudaGetErrorString(e));
            return AMG_ERR_OOM;
        }
    }
    live[q] = n;
    bytes += n;
    if (bytes > peak) peak = bytes;
    *p = q;
    return AMG_OK;
}

void Mem::release(void *p) {
    auto it = live.find(p);
    if (it == live.end()) return;
    bytes -= it->second;
    live.erase(it);
    if (g_free) g_free(p, (void *)stream, g_alloc_ctx);
    else cudaFree(p);
}

void Mem::release_all() {
    for (auto &kv : live) {
        if (g_free) g_free(kv.first, (void *)stream, g_alloc_ctx);
        else cudaFree(kv.first);
    }
    live.clear();
    bytes = 0;
}

}  // namespace pcgamg

using namespace pcgamg;

extern "C" {

void amg_default_params(amg_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->coarse_max = 200;
    p->n_pass = 2;
    p->max_levels = 30;
    p->mode = AMG_MODE_PCG64;
    p->hbm_budget = 0;
    p->coarse_solver = AMG_COARSE_AUTO;
    p->coarse_maxit = 30;
    p->coarse_tol = 1e-3;
}

int amg_set_allocator(amg_alloc_fn alloc, amg_free_fn dealloc, void *ctx) {
    if ((alloc == nullptr) != (dealloc == nullptr)) {
        set_error("amg_set_allocator: give both functions or neither");
        return AMG_ERR_ARG;
    }
    g_alloc = alloc;
    g_free = dealloc;
    g_alloc_ctx = ctx;
    return AMG_OK;
}

int amg_setup(const amg_csr *A, const amg_params *p, void *stream, amg_handle *out) {
    set_error("");
    if (!out) {
        set_error("amg_setup: out is NULL");
        return AMG_ERR_ARG;
    }
    *out = nullptr;
    amg_params prm;
    if (p) prm = *p;
    else amg_default_params(&prm);
    amg_hier *h = new (std::nothrow) amg_hier();
    if (!h) {
        set_error("amg_setup: host allocation failed");
        return AMG_ERR_OOM;
    }
    int st = setup_impl(h, A, &prm, (cudaStream_t)stream);
    if (st) {
        char keep[512];
        snprintf(keep, sizeof(keep), "%s", amg_last_error());
        cudaStreamSynchronize((cudaStream_t)stream);
        h->mem.release_all();
        if (h->ctl_host) cudaFreeHost(h->ctl_host);
        delete h;
        set_error("%s", keep);
        return st;
    }
    *out = h;
    return AMG_OK;
}

int amg_set_mode(amg_handle h, int mode) {
    if (!h || (mode != AMG_MODE_PCG64 && mode != AMG_MODE_FCG32)) {
        set_error("amg_set_mode: bad handle or mode");
        return AMG_ERR_ARG;
    }
    h->mode = mode;
    return AMG_OK;
}

int pcg_solve(amg_handle h, const double *b, double *x, double rtol, int maxit, int *iters,
              double *res_hist, void *stream) {
    set_error("");
    if (iters) *iters = 0;
    if (!h) {
        set_error("pcg_solve: NULL handle");
        return AMG_ERR_ARG;
    }
    if (h->invalid) {
        set_error("pcg_solve: the handle's last amg_refresh failed; refresh it again first");
        return AMG_ERR_ARG;
    }
    return solve_impl(h, b, x, rtol, maxit, iters, res_hist, (cudaStream_t)stream);
}

int amg_refresh(amg_handle h, const amg_csr *A, void *stream) {
    set_error("");
    if (!h) {
        set_error("amg_refresh: NULL handle");
        return AMG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamSynchronize(s);
    return refresh_impl(h, A, s);
}

int amg_set_smoother(amg_handle h, int nu, int nblocks, void *stream) {
    set_error("");
    if (!h || nu < 0 || nu > 64 || nblocks < 0) {
        set_error("amg_set_smoother: NULL handle, or nu outside 0..64, or nblocks < 0");
        return AMG_ERR_ARG;
    }
    return set_smoother_impl(h, nu, nblocks, (cudaStream_t)stream);
}

int amg_refresh_time(amg_handle h, double *ms) {
    if (!h || !ms) {
        set_error("amg_refresh_time: NULL argument");
        return AMG_ERR_ARG;
    }
    *ms = h->refresh_ms;
    return AMG_OK;
}

double amg_last_true_residual(amg_handle h) { return h ? h->last_true_rel : -1.0; }

int amg_autotune(amg_handle h, int reps, int *changed, void *stream) {
    set_error("");
    int c = 0;
    if (changed) *changed = 0;
    if (!h) {
        set_error("amg_autotune: NULL handle");
        return AMG_ERR_ARG;
    }
    int st = autotune_impl(h, (cudaStream_t)stream, reps, &c);
    if (changed) *changed = c;
    return st;
}

int amg_set_level_shape(amg_handle h, int level, const int *shape) {
    set_error("");
    if (!h || !shape || level < 1 || level >= (int)h->lev.size()) {
        set_error("amg_set_level_shape: bad handle, level (1..L) or input");
        return AMG_ERR_ARG;
    }
    for (int i = 0; i < 4; i++)
        if (shape[i] < 0 || shape[i] > 8 || (h->smoothed && (shape[i] & 4))) {
            set_error("amg_set_level_shape: shape values are 0..7 (0..3 with smoothed aggregation: the fused "
                      "shapes transfer through the aggregate map)");
            return AMG_ERR_ARG;
        }
    for (int p = 0; p < 2; p++)
        for (int k = 0; k < 2; k++) h->lev[level].shape[p][k] = (unsigned char)shape[2 * p + k];
    drop_graphs(h);
    return AMG_OK;
}

int amg_level_shape(amg_handle h, int level, int *shape) {
    set_error("");
    if (!h || !shape || level < 0 || level >= (int)h->lev.size()) {
        set_error("amg_level_shape: bad handle, level or output");
        return AMG_ERR_ARG;
    }
    for (int p = 0; p < 2; p++)
        for (int k = 0; k < 2; k++) shape[2 * p + k] = h->lev[level].shape[p][k];
    return AMG_OK;
}

int pcg_solve_multi(amg_handle h, int k, const double *B, double *X, double rtol, int maxit, int *iters,
                    double *res_hist, void *stream) {
    set_error("");
    if (!h || h->invalid || !gs_multi_ok(h) || h->smoothed) {
        set_error("pcg_solve_multi: NULL handle, its last amg_refresh failed, it smooths by Gauss-Seidel with "
                  "blocks the one-warp sweeps cannot take (block sizes must divide 32), or it uses smoothed "
                  "aggregation (the multi-column kernels implement the tentative transfers only)");
        return AMG_ERR_ARG;
    }
    return solve_multi_impl(h, k, B, X, rtol, maxit, iters, res_hist, (cudaStream_t)stream);
}

int amg_multi_info(amg_handle h, int *k, int *status, double *true_rel) {
    if (!h) {
        set_error("amg_multi_info: NULL handle");
        return AMG_ERR_ARG;
    }
    if (k) *k = h->multi_k;
    for (int c = 0; c < h->multi_k; c++) {
        if (status) status[c] = h->multi_status[c];
        if (true_rel) true_rel[c] = h->multi_true_rel[c];
    }
    return AMG_OK;
}

int amg_info(amg_handle h, int *levels, int64_t *n_l, int64_t *nnz_l) {
    if (!h) {
        set_error("amg_info: NULL handle");
        return AMG_ERR_ARG;
    }
    int L = (int)h->lev.size();
    if (levels) *levels = L;
    for (int l = 0; l < L; l++) {
        if (n_l) n_l[l] = h->lev[l].A.n;
        if (nnz_l) nnz_l[l] = h->lev[l].A.nnz;
    }
    return AMG_OK;
}

int amg_level_agg(amg_handle h, int level, int pass, int32_t *agg, int64_t *n_out, int64_t *nc_out) {
    if (!h || level < 0 || level + 1 >= (int)h->lev.size()) {
        set_error("amg_level_agg: bad handle or level (the coarsest level has no map)");
        return AMG_ERR_ARG;
    }
    Level &lv = h->lev[level];
    const int32_t *src;
    int64_t n, nc;
    if (pass < 0) {
        src = lv.agg;
        n = lv.A.n;
        nc = lv.nc;
    } else {
        if (pass >= (int)lv.pass_agg.size()) {
            set_error("amg_level_agg: pass out of range");
            return AMG_ERR_ARG;
        }
        src = lv.pass_agg[pass];
        n = lv.pass_n[pass];
        nc = lv.pass_n[pass + 1];
    }
    if (n_out) *n_out = n;
    if (nc_out) *nc_out = nc;
    if (agg) {
        PCG_CK(cudaMemcpy(agg, src, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    }
    return AMG_OK;
}

int amg_level_layout(amg_handle h, int level, int *slice, int64_t *stored, int *index_bytes) {
    if (!h || level < 0 || level >= (int)h->lev.size()) {
        set_error("amg_level_layout: bad handle or level");
        return AMG_ERR_ARG;
    }
    const Sell &S = h->lev[level].S;
    if (slice) *slice = kSlice;
    if (stored) *stored = S.nnz_pad;
    if (index_bytes) *index_bytes = S.col16 ? 2 : 4;
    return AMG_OK;
}

int amg_level_pattern(amg_handle h, int level, int64_t *slices, int64_t *entries) {
    if (!h || level < 0 || level >= (int)h->lev.size()) {
        set_error("amg_level_pattern: bad handle or level");
        return AMG_ERR_ARG;
    }
    const Sell &S = h->lev[level].S;
    if (slices) *slices = S.upat ? S.uniform_slices : 0;
    if (entries) *entries = S.upat ? S.uniform_entries : 0;
    return AMG_OK;
}

int amg_level_csr(amg_handle h, int level, int32_t *row_ptr, int32_t *col, double *val) {
    if (!h || level < 0 || level >= (int)h->lev.size()) {
        set_error("amg_level_csr: bad handle or level");
        return AMG_ERR_ARG;
    }
    DevCSR &a = h->lev[level].A;
    if (row_ptr) PCG_CK(cudaMemcpy(row_ptr, a.rp, sizeof(int32_t) * ((size_t)a.n + 1), cudaMemcpyDeviceToHost));
    if (col) PCG_CK(cudaMemcpy(col, a.ci, sizeof(int32_t) * a.nnz, cudaMemcpyDeviceToHost));
    if (val) PCG_CK(cudaMemcpy(val, a.v, sizeof(double) * a.nnz, cudaMemcpyDeviceToHost));
    return AMG_OK;
}

int amg_level_prolongator(amg_handle h, int level, int64_t *nnz, int32_t *row_ptr, int32_t *col, double *val) {
    set_error("");
    if (!h || !h->smoothed || level < 0 || level + 1 >= (int)h->lev.size()) {
        set_error("amg_level_prolongator: bad handle or level, or the handle uses the tentative prolongator");
        return AMG_ERR_ARG;
    }
    const DevCSR &P = h->lev[level].P;
    if (nnz) *nnz = P.nnz;
    if (row_ptr) PCG_CK(cudaMemcpy(row_ptr, P.rp, sizeof(int32_t) * ((size_t)P.n + 1), cudaMemcpyDeviceToHost));
    if (col) PCG_CK(cudaMemcpy(col, P.ci, sizeof(int32_t) * P.nnz, cudaMemcpyDeviceToHost));
    if (val) PCG_CK(cudaMemcpy(val, P.v, sizeof(double) * P.nnz, cudaMemcpyDeviceToHost));
    return AMG_OK;
}

int amg_setup_times(amg_handle h, double *ms) {
    if (!h || !ms) {
        set_error("amg_setup_times: NULL argument");
        return AMG_ERR_ARG;
    }
    for (int k = 0; k < 4; k++) ms[k] = h->setup_ms[k];
    return AMG_OK;
}

int amg_profile(amg_handle h, int enable) {
    if (!h) {
        set_error("amg_profile: NULL handle");
        return AMG_ERR_ARG;
    }
    return set_profile(h, enable);
}

int amg_profile_read(amg_handle h, double *ms, int64_t *counts, int nkinds) {
    if (!h || nkinds < 0 || nkinds > amg_hier::kKinds) {
        set_error("amg_profile_read: bad handle or nkinds");
        return AMG_ERR_ARG;
    }
    for (int k = 0; k < nkinds; k++) {
        if (ms) ms[k] = h->prof_ms[k];
        if (counts) counts[k] = h->prof_n[k];
    }
    for (int k = 0; k < amg_hier::kKinds; k++) {
        h->prof_ms[k] = 0;
        h->prof_n[k] = 0;
    }
    return AMG_OK;
}

int amg_profile_levels(amg_handle h, int nlev, double *ms, int64_t *counts) {
    set_error("");
    if (!h || nlev < 0 || nlev > amg_hier::kMaxProfLevels) {
        set_error("amg_profile_levels: bad handle or nlev (at most %d)", amg_hier::kMaxProfLevels);
        return AMG_ERR_ARG;
    }
    for (int l = 0; l < nlev; l++)
        for (int p = 0; p < 3; p++) {
            if (ms) ms[3 * l + p] = h->lev_ms[l][p];
            if (counts) counts[3 * l + p] = h->lev_n[l][p];
        }
    for (int l = 0; l < amg_hier::kMaxProfLevels; l++)
        for (int p = 0; p < 3; p++) {
            h->lev_ms[l][p] = 0;
            h->lev_n[l][p] = 0;
        }
    return AMG_OK;
}

int64_t amg_launch_count(amg_handle h) { return h ? h->launches : -1; }

void amg_destroy(amg_handle h) {
    if (!h) return;
    cudaDeviceSynchronize();
    free_profile(h);
    free_multi(h);
    h->mem.release_all();
    if (h->ctl_host) cudaFreeHost(h->ctl_host);
    delete h;
}

const char *amg_last_error(void) { return g_err; }

}  // extern "C"
