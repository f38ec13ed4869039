// Batched solve of independent systems, each with its own hierarchy (the
// time-step pressure solves of several meshes at once; Sec. 3.1 / Sec. 5 per
// system): one CUDA graph holds, for every system, a branch with its whole
// solve (prefix kernels, then a device-side while loop over iterations).
// One launch runs all systems; the branches run concurrently on the GPU,
// small systems filling the machine while large ones stream, with no host
// round trip until every system has finished. Every branch runs the same
// kernels as that handle's own pcg_solve, so each system's result is the
// same bit for bit as solving it alone.
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.cuh"

struct amg_batch_s {
    std::vector<amg_hier *> hs;
    std::vector<int> modes, gens, prefix_k, body_k;
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> ev;  // fork, then one join per system
    cudaStream_t cs0 = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace pcgamg {
namespace {

int batch_capture(amg_batch_s *b);

bool batch_is_dev(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void batch_release_graph(amg_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// The systems' solves share the device, so they are captured without the
// shared-memory tail (a 16-SM cluster waits for 16 free SMs while the other
// branches hold them).
int batch_build(amg_batch_s *b) {
    batch_release_graph(b);
    int m = (int)b->hs.size();
    for (amg_hier *h : b->hs) h->no_tail = 1;
    int st = batch_capture(b);
    for (amg_hier *h : b->hs) h->no_tail = 0;
    return st;
}

int batch_capture(amg_batch_s *b) {
    int m = (int)b->hs.size();
    std::vector<PendingBody> pb(m);
    PCG_CK(cudaStreamBeginCapture(b->cs0, cudaStreamCaptureModeThreadLocal));
    int st = AMG_OK;
    cudaError_t e = cudaEventRecord(b->ev[0], b->cs0);
    for (int i = 0; i < m && !st && e == cudaSuccess; i++) {
        e = cudaStreamWaitEvent(b->branch[i], b->ev[0], 0);
        if (e != cudaSuccess) break;
        st = capture_solve_prefix(b->hs[i], b->modes[i], b->branch[i], &pb[i], &b->prefix_k[i]);
        if (st) break;
        e = cudaEventRecord(b->ev[1 + i], b->branch[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cs0, b->ev[1 + i], 0);
    }
    cudaGraph_t full = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cs0, &full);
    if (!st && e != cudaSuccess) st = cuda_fail(e, "batch graph capture", __FILE__, __LINE__);
    if (!st && e2 != cudaSuccess) st = cuda_fail(e2, "batch graph capture end", __FILE__, __LINE__);
    for (int i = 0; i < m && !st; i++) st = capture_solve_body(pb[i], b->cs0, &b->body_k[i]);
    if (st) {
        if (full) cudaGraphDestroy(full);
        return st;
    }
    e = cudaGraphInstantiate(&b->exec, full, 0);
    cudaGraphDestroy(full);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate (batch)", __FILE__, __LINE__);
    }
    for (int i = 0; i < m; i++) b->gens[i] = b->hs[i]->graph_gen;
    return AMG_OK;
}

}  // namespace
}  // namespace pcgamg

using namespace pcgamg;

extern "C" {

int amg_batch_create(int m, const amg_handle *hs, amg_batch *out) {
    set_error("");
    if (!out || m < 1 || !hs) {
        set_error("amg_batch_create: need m >= 1 handles and an output pointer");
        return AMG_ERR_ARG;
    }
    *out = nullptr;
    for (int i = 0; i < m; i++) {
        if (!hs[i]) {
            set_error("amg_batch_create: handle %d is NULL", i);
            return AMG_ERR_ARG;
        }
        for (int j = 0; j < i; j++)
            if (hs[j] == hs[i]) {
                set_error("amg_batch_create: handle %d appears twice (each system needs its own handle)", i);
                return AMG_ERR_ARG;
            }
    }
    amg_batch_s *b = new amg_batch_s();
    b->hs.assign(hs, hs + m);
    b->modes.assign(m, -1);
    b->gens.assign(m, -1);
    b->prefix_k.assign(m, 0);
    b->body_k.assign(m, 0);
    b->branch.assign(m, nullptr);
    b->ev.assign(m + 1, nullptr);
    int st = AMG_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&b->cs0, cudaStreamNonBlocking);
    for (int i = 0; i < m && e == cudaSuccess; i++) e = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking);
    for (int i = 0; i <= m && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) st = cuda_fail(e, "amg_batch_create streams/events", __FILE__, __LINE__);
    if (st) {
        amg_batch_destroy(b);
        return st;
    }
    *out = b;
    return AMG_OK;
}

int pcg_solve_batch(amg_batch b, const double *const *B, double *const *X, double rtol, int maxit, int *iters,
                    int *status, void *stream) {
    set_error("");
    if (!b || !B || !X || !(rtol >= 0.0) || maxit < 0) {
        set_error("pcg_solve_batch: bad arguments");
        return AMG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int m = (int)b->hs.size();
    bool rebuild = b->exec == nullptr;
    for (int i = 0; i < m; i++) {
        amg_hier *h = b->hs[i];
        if (!B[i] || !X[i]) {
            set_error("pcg_solve_batch: NULL vector for system %d", i);
            return AMG_ERR_ARG;
        }
        if (h->invalid) {
            set_error("pcg_solve_batch: system %d: its last amg_refresh failed", i);
            return AMG_ERR_ARG;
        }
        h->mem.stream = s;
        PCG_TRY(ensure_hist(h, maxit));
        if (b->modes[i] != h->mode || b->gens[i] != h->graph_gen) rebuild = true;
    }
    if (rebuild) {
        for (int i = 0; i < m; i++) b->modes[i] = b->hs[i]->mode;
        PCG_TRY(batch_build(b));
    }
    std::vector<char> xdev(m);
    for (int i = 0; i < m; i++) {
        amg_hier *h = b->hs[i];
        size_t bytes = sizeof(double) * (size_t)h->lev[0].A.n;
        xdev[i] = batch_is_dev(X[i]);
        PCG_CK(cudaMemcpyAsync(h->b, B[i], bytes, cudaMemcpyDefault, s));
        PCG_CK(cudaMemcpyAsync(h->x, X[i], bytes, cudaMemcpyDefault, s));
        Ctl c0;
        memset(&c0, 0, sizeof(c0));
        c0.rtol = rtol;
        c0.maxit = maxit;
        c0.mode = h->mode;
        c0.flex = h->coarse_iter;
        c0.restart = 1;
        *h->ctl_host = c0;
        PCG_CK(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    }
    PCG_CK(cudaGraphLaunch(b->exec, s));
    for (int i = 0; i < m; i++)
        PCG_CK(cudaMemcpyAsync(b->hs[i]->ctl_host, b->hs[i]->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    PCG_CK(cudaStreamSynchronize(s));
    int st = AMG_OK;
    for (int i = 0; i < m; i++) {
        amg_hier *h = b->hs[i];
        Ctl &c = *h->ctl_host;
        size_t bytes = sizeof(double) * (size_t)h->lev[0].A.n;
        if (c.done == 1 && c.bnorm == 0.0) PCG_CK(cudaMemsetAsync(h->x, 0, bytes, s));
        PCG_CK(cudaMemcpyAsync(X[i], h->x, bytes, cudaMemcpyDefault, s));
        int si = c.done ? c.status : AMG_ERR_NOCONV;
        if (iters) iters[i] = c.iter;
        if (status) status[i] = si;
        h->last_true_rel = c.true_rel;
        h->launches += b->prefix_k[i] + (int64_t)c.bodies * b->body_k[i];
        if (si != AMG_OK && st == AMG_OK) st = si;
    }
    PCG_CK(cudaStreamSynchronize(s));
    if (st) set_error("pcg_solve_batch: some systems did not converge (status %d; see the status array)", st);
    return st;
}

void amg_batch_destroy(amg_batch b) {
    if (!b) return;
    cudaDeviceSynchronize();
    batch_release_graph(b);
    for (auto e : b->ev)
        if (e) cudaEventDestroy(e);
    for (auto s : b->branch)
        if (s) cudaStreamDestroy(s);
    if (b->cs0) cudaStreamDestroy(b->cs0);
    delete b;
}

}  // extern "C"
