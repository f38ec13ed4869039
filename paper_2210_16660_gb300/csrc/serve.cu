// Serving: many time-step pressure solves over meshes whose hierarchies stay
// resident on the device. The hierarchy of a fixed mesh is built once and
// reused for every solve (arxiv 2210.16660, Sec. 1 and Sec. 4: the matrix does
// not change between time steps); each request is one solve A_m x = b started
// from the previous step's solution (Sec. 5).
//
// Continuous batching: every mesh has engines of K right-hand-side slots
// (the multi-column kernels) and a whole-solve lane (the single-column
// kernels, one graph launch per solve). A request goes to its mesh's lane if
// the lane is idle (at low load a request runs at the speed of a lone
// solve), else to a free slot; the host visits an engine between chunks of
// `chunk` iterations, hands finished columns back, and starts queued
// requests in the freed slots while the other columns carry on from where
// they were. Each lane and engine has its own stream (engines their own
// captured chunk graph), so they overlap on the device. A request's
// arithmetic is that of its own column only, so its result does not depend
// on what shares the engine.
//
// Memory: the resident hierarchies and all engine workspaces fit in a byte
// budget; amg_serve_plan (host only) picks the engine count per mesh.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace pcgamg {
namespace {

constexpr int kSB = 256;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

__global__ void k_col_out(const double *__restrict__ X, double *__restrict__ x, int K, int c, int n, int zero) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = zero ? 0.0 : X[(int64_t)i * K + c];
}

struct Request {
    int mesh = 0;
    const double *b = nullptr, *x0 = nullptr;
    double *x = nullptr;
    bool done = false;
    int status = AMG_OK, iters = 0;
    double true_rel = 0.0;
    double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
    int lane = 0;  // 0: whole-solve lane, 1: a slot of a batching engine
};

// Whole-solve lane of one mesh: the single right-hand-side kernels (one graph
// launch per solve) on the hierarchy's own resident vectors.
struct Lane {
    amg_hier *h = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    int64_t ticket = -1;
};

struct Engine {
    int mesh = 0;
    amg_hier *h = nullptr;
    Mem mem;
    MultiWS W;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    bool inflight = false;
    std::vector<int64_t> slot;  // ticket per slot, -1 free
    double *stage_b = nullptr, *stage_x = nullptr;
    int64_t step_kernels = 0;
};

}  // namespace
}  // namespace pcgamg

using namespace pcgamg;

struct amg_server_s {
    amg_server_params prm;
    std::vector<amg_hier *> meshes;
    std::vector<int> engines_of;
    std::vector<size_t> engine_bytes, resident;
    std::vector<Engine *> eng;
    std::vector<Lane> lane;  // per mesh; h == nullptr: none
    std::vector<std::deque<int64_t>> queue;
    std::unordered_map<int64_t, Request> req;
    int64_t next_ticket = 1;
    int queued = 0, running = 0;
    size_t budget = 0, used = 0;
    int64_t launches = 0;
};

namespace pcgamg {
namespace {

void engine_free(Engine *e) {
    if (!e) return;
    if (e->s) cudaStreamSynchronize(e->s);
    mws_free(e->mem, e->W);
    release(e->mem, e->stage_b);
    release(e->mem, e->stage_x);
    e->mem.release_all();
    if (e->ev) cudaEventDestroy(e->ev);
    if (e->s) cudaStreamDestroy(e->s);
    delete e;
}

// Device bytes of one engine of mesh h: its K-column workspace (one V-cycle
// precision) and two staging vectors for host-side requests.
size_t engine_bytes_of(amg_hier *h, const amg_server_params &p) {
    int which = p.mode == AMG_MODE_FCG32 ? 1 : 2;
    size_t ws = mws_bytes(h, p.slots, p.maxit + 1, which);
    if (ws == (size_t)-1) return ws;
    size_t vec = ((sizeof(double) * (size_t)h->lev[0].A.n) + 255) & ~(size_t)255;
    return ws + 2 * vec;
}

int engine_create(amg_server_s *sv, int mesh, Engine **out) {
    Engine *e = new Engine();
    *out = nullptr;
    e->mesh = mesh;
    e->h = sv->meshes[mesh];
    amg_hier *h = e->h;
    int n = h->lev[0].A.n;
    int K = sv->prm.slots;
    int st = AMG_OK;
    // With lane_priority, engines run at the lowest stream priority: they fill
    // what the whole-solve lanes leave of the device.
    int least = 0, greatest = 0;
    cudaError_t ce = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    int prio = sv->prm.lane_priority ? least : 0;
    if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&e->s, cudaStreamNonBlocking, prio);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) st = cuda_fail(ce, "serving engine stream", __FILE__, __LINE__);
    e->mem.stream = e->s;
    int which = sv->prm.mode == AMG_MODE_FCG32 ? 1 : 2;
    if (!st) st = mws_alloc(h, e->mem, e->W, K, sv->prm.maxit + 1, which);
    if (!st) st = alloc(e->mem, &e->stage_b, (size_t)n);
    if (!st) st = alloc(e->mem, &e->stage_x, (size_t)n);
    if (!st) st = mws_reset(e->W, sv->prm.mode, sv->prm.rtol, sv->prm.maxit, e->s);
    if (!st) {
        // Capture the chunk graph now, so serving never captures mid-stream.
        st = mws_iterate(h, e->W, sv->prm.mode, sv->prm.chunk, nullptr, /*launch=*/0);
    }
    if (!st) {
        // Kernel nodes per chunk, for the launch count.
        size_t nodes = 0;
        if (e->W.step_graph && cudaGraphGetNodes(e->W.step_graph, nullptr, &nodes) == cudaSuccess) {
            std::vector<cudaGraphNode_t> v(nodes);
            cudaGraphGetNodes(e->W.step_graph, v.data(), &nodes);
            for (auto nd : v) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) e->step_kernels++;
            }
        }
    }
    if (st) {
        engine_free(e);
        return st;
    }
    e->slot.assign(K, -1);
    *out = e;
    return AMG_OK;
}

// The chunk on this engine has finished: hand back every column that is no
// longer iterating (converged, failed, or never started because b = 0 or x0
// already met rtol) and free its slot.
int harvest(amg_server_s *sv, Engine *e, int *finished) {
    const CtlM &c = *e->W.ctl_host;
    int n = e->h->lev[0].A.n;
    int K = e->W.K;
    std::vector<int64_t> out;
    for (int q = 0; q < K; q++) {
        int64_t t = e->slot[q];
        if (t < 0 || c.active[q]) continue;
        Request &r = sv->req[t];
        r.status = c.status[q];
        r.iters = c.iter[q];
        r.true_rel = c.true_rel[q];
        int zero = c.bnorm[q] == 0.0;
        if (on_device(r.x)) {
            k_col_out<<<(n + kSB - 1) / kSB, kSB, 0, e->s>>>(e->W.x, r.x, K, q, n, zero);
            sv->launches++;
        } else {
            k_col_out<<<(n + kSB - 1) / kSB, kSB, 0, e->s>>>(e->W.x, e->stage_x, K, q, n, zero);
            sv->launches++;
            PCG_CK(cudaMemcpyAsync(r.x, e->stage_x, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, e->s));
        }
        PCG_LAUNCH_CK();
        out.push_back(t);
        e->slot[q] = -1;
    }
    if (out.empty()) return AMG_OK;
    PCG_CK(cudaStreamSynchronize(e->s));
    double t1 = now_s();
    for (int64_t t : out) {
        Request &r = sv->req[t];
        r.done = true;
        r.t_done = t1;
        sv->running--;
    }
    if (finished) *finished += (int)out.size();
    return AMG_OK;
}

// Starts queued requests of this engine's mesh in its free slots. An idle
// engine starts only once batch_min requests wait (when the mesh has a lane:
// a lone request is served faster by waiting for the lane than by a slot).
int admit(amg_server_s *sv, Engine *e) {
    auto &qu = sv->queue[e->mesh];
    if (qu.empty()) return AMG_OK;
    bool idle = true;
    for (int64_t t : e->slot) idle &= t < 0;
    if (idle && sv->lane[e->mesh].h && (int)qu.size() < sv->prm.batch_min) return AMG_OK;
    int n = e->h->lev[0].A.n;
    size_t bytes = sizeof(double) * (size_t)n;
    unsigned mask = 0;
    double t0 = now_s();
    for (int q = 0; q < e->W.K && !qu.empty(); q++) {
        if (e->slot[q] >= 0) continue;
        int64_t t = qu.front();
        qu.pop_front();
        Request &r = sv->req[t];
        const double *b = r.b, *x0 = r.x0;
        if (!on_device(b)) {
            PCG_CK(cudaMemcpyAsync(e->stage_b, b, bytes, cudaMemcpyHostToDevice, e->s));
            b = e->stage_b;
        }
        if (!on_device(x0)) {
            PCG_CK(cudaMemcpyAsync(e->stage_x, x0, bytes, cudaMemcpyHostToDevice, e->s));
            x0 = e->stage_x;
        }
        PCG_TRY(mws_put_column(e->W, q, b, x0, n, e->s));
        sv->launches++;
        e->slot[q] = t;
        r.t_start = t0;
        r.lane = 1;
        mask |= 1u << q;
        sv->queued--;
        sv->running++;
    }
    if (!mask) return AMG_OK;
    PCG_TRY(mws_admit(e->h, e->W, sv->prm.mode, mask, e->s));
    sv->launches += 2;
    return AMG_OK;
}

int lane_start(amg_server_s *sv, Lane &ln, int mesh) {
    auto &qu = sv->queue[mesh];
    if (qu.empty() || ln.ticket >= 0) return AMG_OK;
    int64_t t = qu.front();
    qu.pop_front();
    Request &r = sv->req[t];
    PCG_TRY(solve_launch(ln.h, sv->prm.mode, r.b, r.x0, sv->prm.rtol, sv->prm.maxit, ln.s));
    PCG_CK(cudaEventRecord(ln.ev, ln.s));
    ln.ticket = t;
    r.t_start = now_s();
    r.lane = 0;
    sv->queued--;
    sv->running++;
    return AMG_OK;
}

int lane_finish(amg_server_s *sv, Lane &ln, int *finished) {
    Request &r = sv->req[ln.ticket];
    int64_t k = 0;
    PCG_TRY(solve_collect(ln.h, sv->prm.mode, r.x, ln.s, &r.status, &r.iters, &r.true_rel, &k));
    PCG_CK(cudaStreamSynchronize(ln.s));
    sv->launches += k;
    r.done = true;
    r.t_done = now_s();
    sv->running--;
    ln.ticket = -1;
    if (finished) (*finished)++;
    return AMG_OK;
}

int launch_chunk(amg_server_s *sv, Engine *e) {
    PCG_TRY(mws_iterate(e->h, e->W, sv->prm.mode, sv->prm.chunk, e->s, /*launch=*/1));
    PCG_CK(cudaEventRecord(e->ev, e->s));
    e->inflight = true;
    sv->launches += e->step_kernels;
    return AMG_OK;
}

}  // namespace
}  // namespace pcgamg

extern "C" {

void amg_server_default_params(amg_server_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->mode = AMG_MODE_FCG32;
    p->slots = 4;
    p->max_engines = 2;
    p->solo = 1;
    p->batch_min = 3;
    p->lane_priority = 0;
    p->chunk = 4;
    p->queue_cap = 4096;
    p->maxit = 1000;
    p->rtol = 1e-8;
    p->hbm_budget = 0;
}

int amg_serve_plan(int m, const size_t *resident, const size_t *engine_bytes, const double *load, size_t budget,
                   int max_engines, int *engines, size_t *total) {
    set_error("");
    if (m < 1 || !resident || !engine_bytes || !engines || max_engines < 1) {
        set_error("amg_serve_plan: need m >= 1, byte arrays, an output array and max_engines >= 1");
        return AMG_ERR_ARG;
    }
    size_t used = 0;
    int admitted = 0;
    // Meshes in order: resident hierarchy plus one engine, if that fits.
    for (int i = 0; i < m; i++) {
        engines[i] = 0;
        size_t need = resident[i] + engine_bytes[i];
        if (need >= resident[i] && used + need >= used && used + need <= budget) {
            used += need;
            engines[i] = 1;
            admitted++;
        }
    }
    // Then one engine at a time to the mesh with the most load per engine.
    for (;;) {
        int best = -1;
        double best_score = -1.0;
        for (int i = 0; i < m; i++) {
            if (engines[i] < 1 || engines[i] >= max_engines) continue;
            if (used + engine_bytes[i] < used || used + engine_bytes[i] > budget) continue;
            double w = load ? load[i] : 1.0;
            double score = w / engines[i];
            if (score > best_score) {
                best_score = score;
                best = i;
            }
        }
        if (best < 0) break;
        engines[best]++;
        used += engine_bytes[best];
    }
    if (total) *total = used;
    if (!admitted) {
        set_error("amg_serve_plan: no mesh fits the budget of %zu bytes", budget);
        return AMG_ERR_OOM;
    }
    return AMG_OK;
}

int amg_server_create(const amg_server_params *p, int m, const amg_handle *meshes, const double *load,
                      amg_server *out) {
    set_error("");
    if (!out || !p || m < 1 || !meshes) {
        set_error("amg_server_create: bad arguments");
        return AMG_ERR_ARG;
    }
    *out = nullptr;
    const amg_server_params &P = *p;
    if ((P.mode != AMG_MODE_FCG32 && P.mode != AMG_MODE_PCG64) ||
        (P.slots != 4 && P.slots != 8 && P.slots != 16 && P.slots != 32) || P.max_engines < 1 || P.chunk < 1 ||
        P.queue_cap < 0 || P.maxit < 0 || !(P.rtol >= 0.0) || (P.solo != 0 && P.solo != 1) || P.batch_min < 1 ||
        (P.lane_priority != 0 && P.lane_priority != 1)) {
        set_error("amg_server_create: bad parameters (mode, slots in {4,8,16,32}, max_engines >= 1, chunk >= 1, "
                  "solo 0 or 1, batch_min >= 1, lane_priority 0 or 1)");
        return AMG_ERR_ARG;
    }
    for (int i = 0; i < m; i++) {
        if (!meshes[i]) {
            set_error("amg_server_create: mesh %d is NULL", i);
            return AMG_ERR_ARG;
        }
        if (!gs_multi_ok(meshes[i]) || meshes[i]->smoothed) {
            set_error("amg_server_create: mesh %d smooths by Gauss-Seidel with blocks the engines cannot take "
                      "(block sizes must divide 32), or uses smoothed aggregation (engines run the tentative "
                      "transfers)", i);
            return AMG_ERR_ARG;
        }
        if (meshes[i]->lev.size() < 2) {
            set_error("amg_server_create: mesh %d has a single level (serving needs a coarse level)", i);
            return AMG_ERR_ARG;
        }
        for (int j = 0; j < i; j++)
            if (meshes[j] == meshes[i]) {
                set_error("amg_server_create: mesh %d appears twice", i);
                return AMG_ERR_ARG;
            }
    }
    amg_server_s *sv = new amg_server_s();
    sv->prm = P;
    sv->meshes.assign(meshes, meshes + m);
    sv->queue.resize(m);
    sv->engines_of.assign(m, 0);
    sv->engine_bytes.assign(m, 0);
    sv->resident.assign(m, 0);
    size_t resident_total = 0;
    for (int i = 0; i < m; i++) {
        PCG_CK(cudaSetDevice(sv->meshes[i]->device));
        sv->resident[i] = sv->meshes[i]->mem.bytes;
        sv->engine_bytes[i] = engine_bytes_of(sv->meshes[i], P);
        resident_total += sv->resident[i];
    }
    size_t budget = P.hbm_budget;
    if (!budget) {
        size_t fr = 0, tot = 0;
        PCG_CK(cudaMemGetInfo(&fr, &tot));
        size_t reserve = (size_t)1 << 30;
        budget = resident_total + (fr > reserve ? fr - reserve : 0);
    }
    sv->budget = budget;
    int st = amg_serve_plan(m, sv->resident.data(), sv->engine_bytes.data(), load, budget, P.max_engines,
                            sv->engines_of.data(), &sv->used);
    sv->lane.resize(m);
    for (int i = 0; i < m && !st && P.solo; i++) {
        if (!sv->engines_of[i]) continue;
        Lane &ln = sv->lane[i];
        ln.h = sv->meshes[i];
        // With lane_priority, lanes run at the highest priority, so a request
        // that finds its lane idle runs at close to the speed of a lone solve.
        int least = 0, greatest = 0;
        cudaError_t ce = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        int prio = P.lane_priority ? greatest : 0;
        if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&ln.s, cudaStreamNonBlocking, prio);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ln.ev, cudaEventDisableTiming);
        if (ce != cudaSuccess) st = cuda_fail(ce, "serving lane stream", __FILE__, __LINE__);
        if (!st) st = solve_prepare(ln.h, P.mode, P.maxit);
    }
    for (int i = 0; i < m && !st; i++)
        for (int k = 0; k < sv->engines_of[i] && !st; k++) {
            Engine *e = nullptr;
            st = engine_create(sv, i, &e);
            if (!st) sv->eng.push_back(e);
        }
    if (st) {
        amg_server_destroy(sv);
        return st;
    }
    *out = sv;
    return AMG_OK;
}

int amg_server_mesh_info(amg_server sv, int mesh, int *engines, int *slots, size_t *engine_bytes,
                         size_t *resident_bytes) {
    set_error("");
    if (!sv || mesh < 0 || mesh >= (int)sv->meshes.size()) {
        set_error("amg_server_mesh_info: bad server or mesh");
        return AMG_ERR_ARG;
    }
    if (engines) *engines = sv->engines_of[mesh];
    if (slots) *slots = sv->prm.slots;
    if (engine_bytes) *engine_bytes = sv->engine_bytes[mesh];
    if (resident_bytes) *resident_bytes = sv->resident[mesh];
    return AMG_OK;
}

int amg_server_info(amg_server sv, size_t *budget, size_t *used, int *queued, int *running, int64_t *launches) {
    set_error("");
    if (!sv) {
        set_error("amg_server_info: NULL server");
        return AMG_ERR_ARG;
    }
    if (budget) *budget = sv->budget;
    if (used) *used = sv->used;
    if (queued) *queued = sv->queued;
    if (running) *running = sv->running;
    if (launches) *launches = sv->launches;
    return AMG_OK;
}

int amg_server_submit(amg_server sv, int mesh, const double *b, const double *x0, double *x, int64_t *ticket) {
    set_error("");
    if (ticket) *ticket = 0;
    if (!sv || !ticket || !b || !x0 || !x || mesh < 0 || mesh >= (int)sv->meshes.size()) {
        set_error("amg_server_submit: bad arguments");
        return AMG_ERR_ARG;
    }
    if (sv->engines_of[mesh] == 0) {
        set_error("amg_server_submit: mesh %d was not admitted (its hierarchy and one engine exceed the budget)",
                  mesh);
        return AMG_ERR_OOM;
    }
    if (sv->meshes[mesh]->invalid || !gs_multi_ok(sv->meshes[mesh]) || sv->meshes[mesh]->smoothed) {
        set_error("amg_server_submit: mesh %d: its last amg_refresh failed, or its smoother or prolongator "
                  "changed to one the engines cannot take", mesh);
        return AMG_ERR_ARG;
    }
    if (sv->queued >= sv->prm.queue_cap) {
        set_error("amg_server_submit: queue full (%d requests waiting)", sv->queued);
        return AMG_ERR_BUSY;
    }
    int64_t t = sv->next_ticket++;
    Request r;
    r.mesh = mesh;
    r.b = b;
    r.x0 = x0;
    r.x = x;
    r.t_submit = now_s();
    sv->req.emplace(t, r);
    sv->queue[mesh].push_back(t);
    sv->queued++;
    *ticket = t;
    return AMG_OK;
}

int amg_server_progress(amg_server sv, int wait, int *finished) {
    set_error("");
    if (finished) *finished = 0;
    if (!sv) {
        set_error("amg_server_progress: NULL server");
        return AMG_ERR_ARG;
    }
    int fin = 0;
    for (;;) {
        bool busy = false, ready = false;
        for (Lane &ln : sv->lane) {
            if (ln.ticket < 0) continue;
            cudaError_t q = cudaEventQuery(ln.ev);
            if (q == cudaErrorNotReady) {
                busy = true;
                continue;
            }
            if (q != cudaSuccess) return cuda_fail(q, "serving lane", __FILE__, __LINE__);
            ready = true;
            PCG_TRY(lane_finish(sv, ln, &fin));
        }
        for (Engine *e : sv->eng) {
            if (!e->inflight) continue;
            cudaError_t q = cudaEventQuery(e->ev);
            if (q == cudaErrorNotReady) {
                busy = true;
                continue;
            }
            if (q != cudaSuccess) return cuda_fail(q, "serving chunk", __FILE__, __LINE__);
            e->inflight = false;
            ready = true;
            PCG_TRY(harvest(sv, e, &fin));
        }
        if (ready || !busy || !wait) break;
        std::this_thread::yield();
    }
    // An idle whole-solve lane takes the head of its mesh's queue; idle engines
    // take what is left, then run one chunk if any slot is in use.
    for (int i = 0; i < (int)sv->lane.size(); i++)
        if (sv->lane[i].h) PCG_TRY(lane_start(sv, sv->lane[i], i));
    for (Engine *e : sv->eng) {
        if (e->inflight) continue;
        PCG_TRY(admit(sv, e));
        bool any = false;
        for (int64_t t : e->slot) any |= t >= 0;
        if (any) PCG_TRY(launch_chunk(sv, e));
    }
    if (finished) *finished = fin;
    return AMG_OK;
}

int amg_server_result(amg_server sv, int64_t ticket, int *done, int *status, int *iters, double *true_rel,
                      int *lane, double *times) {
    set_error("");
    if (done) *done = 0;
    if (!sv) {
        set_error("amg_server_result: NULL server");
        return AMG_ERR_ARG;
    }
    auto it = sv->req.find(ticket);
    if (it == sv->req.end()) {
        set_error("amg_server_result: unknown ticket %lld", (long long)ticket);
        return AMG_ERR_ARG;
    }
    Request &r = it->second;
    if (!r.done) return AMG_OK;
    if (done) *done = 1;
    if (status) *status = r.status;
    if (iters) *iters = r.iters;
    if (true_rel) *true_rel = r.true_rel;
    if (lane) *lane = r.lane;
    if (times) {
        times[0] = 1e3 * (r.t_start - r.t_submit);
        times[1] = 1e3 * (r.t_done - r.t_start);
        times[2] = 1e3 * (r.t_done - r.t_submit);
    }
    sv->req.erase(it);
    return AMG_OK;
}

void amg_server_destroy(amg_server sv) {
    if (!sv) return;
    for (Lane &ln : sv->lane) {
        if (ln.s) cudaStreamSynchronize(ln.s);
        if (ln.ev) cudaEventDestroy(ln.ev);
        if (ln.s) cudaStreamDestroy(ln.s);
    }
    for (Engine *e : sv->eng) engine_free(e);
    delete sv;
}

}  // extern "C"
