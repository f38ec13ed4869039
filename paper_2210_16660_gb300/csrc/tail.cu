// Shared-memory cluster tail: the V-cycle phases of the smallest levels
// (first..L, every one a chain of dependent loads rather than a stream of
// bytes) run in one launch of a single thread-block cluster whose CTAs hold
// those levels' matrices, transfer maps and vectors in shared memory. Each
// CTA owns a contiguous block of rows of every tail level; a gather from a
// row another CTA owns is a distributed-shared-memory load, so no step of
// the tail goes to L2 after the first copy. Phases are separated by the
// cluster barrier (release/acquire at cluster scope).
//
// The arithmetic is that of the separate kernels, in the same order: a row
// sums its stored entries in column order (the sliced-ELL sweeps sum the same
// entries in the same order, then their zero padding), t, the restriction
// (members in increasing index order), the dense coarsest product (lane-
// strided partial sums and the same shuffle tree as k_coarse), prolongation
// and post-smoothing use the same expressions, so a solve gives the same
// bits with and without the tail.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "tail_plan.h"

namespace cg = cooperative_groups;

namespace pcgamg {
namespace {

constexpr int kTThreads = 1024;
template <typename T>
__device__ __forceinline__ T *remote(cg::cluster_group &cl, T *p, uint32_t ref) {
    return cl.map_shared_rank(p, (unsigned)(ref >> 24)) + (ref & 0xffffffu);
}

template <typename T>
__device__ __forceinline__ T *at(unsigned char *smem, int off) { return reinterpret_cast<T *>(smem + off); }

// sum_q val[q] vec(cp[q]) over row i, entries in storage order. The remote
// loads of 8 entries are issued before their FMAs (the last chunk masked),
// so a row costs about one distributed-shared-memory latency per 8 entries
// instead of one per entry; the FMAs keep their order.
template <typename T>
__device__ __forceinline__ T row_dot(cg::cluster_group &cl, const int32_t *rp, const uint32_t *cp, const T *val,
                                     T *vec, int i) {
    constexpr int U = 8;
    T acc = 0;
    int e = rp[i + 1];
    for (int q = rp[i]; q < e; q += U) {
        T x[U];
#pragma unroll
        for (int u = 0; u < U; u++) x[u] = (q + u < e) ? *remote(cl, vec, cp[q + u]) : T(0);
#pragma unroll
        for (int u = 0; u < U; u++)
            if (q + u < e) acc += val[q + u] * x[u];
    }
    return acc;
}

template <typename T>
__global__ void __launch_bounds__(kTThreads, 1) k_tail_smem(SmemTailPlan plan, const unsigned char *__restrict__ blob,
                                                            const T *__restrict__ bF, const T *__restrict__ xpreF,
                                                            T *__restrict__ xF, const Ctl *__restrict__ ctl) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, nth = blockDim.x;
    // 1. this CTA's static data (matrices, maps, coarsest rows) in one copy.
    // It is written once at setup, so the copy runs before the wait for the
    // preceding kernel and overlaps that kernel's end. 16-byte asynchronous
    // copies (global to shared, no registers): every piece of a thread is in
    // flight at once.
    {
        const unsigned char *src = blob + (size_t)rank * plan.static_bytes;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
        for (int k = tid; k < plan.static_bytes / 16; k += nth)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16 * k), "l"(src + 16 * k)
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    pdl_enter();
    bF = after_wait(bF);
    xpreF = after_wait(xpreF);
    xF = after_wait(xF);
    if (ctl->done) {
        asm volatile("cp.async.wait_all;" ::: "memory");  // no copy may outlive the block
        return;
    }
    // ... and the entry level's b and xpre rows (written by the previous kernel)
    {
        const SmemTailLevel &F = plan.lev[0];
        int r0 = rank * F.rpc, r1 = min(F.n, r0 + F.rpc);
        T *b = at<T>(smem, F.off_b), *xp = at<T>(smem, F.off_xpre);
        for (int i = r0 + tid; i < r1; i += nth) {
            b[i - r0] = bF[i];
            xp[i - r0] = xpreF[i];
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    cl.sync();
    // 2. down sweep and restriction, level by level
    for (int k = 0; k + 1 < plan.nt; k++) {
        const SmemTailLevel &Lv = plan.lev[k];
        const SmemTailLevel &Cv = plan.lev[k + 1];
        int rows = min(Lv.rpc, Lv.n - rank * Lv.rpc);
        const int32_t *rp = at<int32_t>(smem, Lv.off_rp);
        const uint32_t *cp = at<uint32_t>(smem, Lv.off_col);
        const T *val = at<T>(smem, Lv.off_val);
        const T *p = at<T>(smem, Lv.off_p);
        T *b = at<T>(smem, Lv.off_b), *t = at<T>(smem, Lv.off_t), *xpre = at<T>(smem, Lv.off_xpre);
        for (int i = tid; i < rows; i += nth) {
            T acc = row_dot(cl, rp, cp, val, xpre, i);
            t[i] = p[i] * (b[i] - acc);
        }
        cl.sync();
        bool last = (k + 2 == plan.nt);
        int crows = min(Cv.rpc, Cv.n - rank * Cv.rpc);
        const int32_t *mp = at<int32_t>(smem, Lv.off_mp);
        const uint32_t *mem = at<uint32_t>(smem, Lv.off_mem);
        for (int I = tid; I < crows; I += nth) {
            // members in increasing index order; the first four loaded together
            const int q0 = mp[I], q1 = mp[I + 1];
            T tv[4];
#pragma unroll
            for (int u = 0; u < 4; u++) tv[u] = q0 + u < q1 ? *remote(cl, t, mem[q0 + u]) : T(0);
            T s = 0;
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (q0 + u < q1) s += tv[u];
            for (int q = q0 + 4; q < q1; q++) s += *remote(cl, t, mem[q]);
            if (last) {
                at<double>(smem, plan.off_bl)[I] = (double)s;
            } else {
                at<T>(smem, Cv.off_b)[I] = s;
                at<T>(smem, Cv.off_xpre)[I] = at<T>(smem, Cv.off_dinv)[I] * s;
            }
        }
        cl.sync();
    }
    // 3. coarsest: x_L = A_L^{-1} b_L, one warp per row (rows of this CTA)
    {
        const SmemTailLevel &C = plan.lev[plan.nt - 1];
        int rows = min(C.rpc, C.n - rank * C.rpc);
        const double *ainv = at<double>(smem, plan.off_ainv);
        double *bl = at<double>(smem, plan.off_bl);
        T *xL = at<T>(smem, C.off_x);
        int warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
        for (int row = warp; row < rows; row += nw) {
            const double *a = ainv + (size_t)row * C.n;
            double s = 0.0;
            // the lane's entries j = lane, lane + 32, ... in the order of
            // k_coarse, their b_L values loaded 4 at a time ahead of the FMAs
            for (int j0 = lane; j0 < C.n; j0 += 4 * 32) {
                double bv[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    int j = j0 + 32 * u;
                    bv[u] = j < C.n ? *remote(cl, bl, pack(j / C.rpc, j % C.rpc)) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (j0 + 32 * u < C.n) s += a[j0 + 32 * u] * bv[u];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) xL[row] = (T)s;
        }
    }
    cl.sync();
    // 4. prolongation and post sweep, level by level back up
    for (int k = plan.nt - 2; k >= 0; k--) {
        const SmemTailLevel &Lv = plan.lev[k];
        const SmemTailLevel &Cv = plan.lev[k + 1];
        int rows = min(Lv.rpc, Lv.n - rank * Lv.rpc);
        const uint32_t *agg = at<uint32_t>(smem, Lv.off_agg);
        const T *p = at<T>(smem, Lv.off_p);
        T *xpre = at<T>(smem, Lv.off_xpre), *xp = at<T>(smem, Lv.off_xp);
        T *xc = at<T>(smem, Cv.off_x);
        for (int i = tid; i < rows; i += nth) {
            T x = xpre[i];
            uint32_t a = agg[i];
            if (a != kNone) x += p[i] * *remote(cl, xc, a);
            xp[i] = x;
        }
        cl.sync();
        const int32_t *rp = at<int32_t>(smem, Lv.off_rp);
        const uint32_t *cp = at<uint32_t>(smem, Lv.off_col);
        const T *val = at<T>(smem, Lv.off_val);
        const T *dinv = at<T>(smem, Lv.off_dinv);
        T *b = at<T>(smem, Lv.off_b), *x = at<T>(smem, Lv.off_x);
        for (int i = tid; i < rows; i += nth) {
            T acc = row_dot(cl, rp, cp, val, xp, i);
            x[i] = xp[i] + dinv[i] * (b[i] - acc);
        }
        if (k > 0) cl.sync();
    }
    // 5. the entry level's x back to global memory for the next prolongation
    {
        const SmemTailLevel &F = plan.lev[0];
        int r0 = rank * F.rpc, r1 = min(F.n, r0 + F.rpc);
        const T *x = at<T>(smem, F.off_x);
        for (int i = r0 + tid; i < r1; i += nth) xF[i] = x[i - r0];
    }
    // no CTA may leave while another still reads its shared memory
    cl.sync();
}

template <typename X>
int fetch(std::vector<X> &dst, const X *src, size_t n) {
    dst.resize(n);
    if (n) PCG_CK(cudaMemcpy(dst.data(), src, n * sizeof(X), cudaMemcpyDeviceToHost));
    return AMG_OK;
}

// The kernel's attributes are per function, shared by every hierarchy: the
// dynamic shared-memory limit is set to the device maximum (never to one
// plan's size, which a later hierarchy's setup would then shrink under an
// earlier one's launches).
template <typename T>
int cluster_fits(int ctas, size_t smem, int smem_max) {
    if (cudaFuncSetAttribute(k_tail_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess ||
        cudaFuncSetAttribute(k_tail_smem<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kTThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_tail_smem<T>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n >= 1;
}

}  // namespace

// Plans the shared-memory tail of h for each V-cycle precision: the first
// level l >= 1 from which every level has at most kSmemTailRows rows and
// whose tail's data fit the cluster's shared memory, if at least one level
// lies between it and the coarsest; otherwise no tail for that precision
// (tail_first[p] = 0).
// Host copies of what the tail levels F..L need.
int fetch_tail_levels(amg_hier *h, int F, std::vector<HostLevel> &hl) {
    int L = (int)h->lev.size() - 1;
    int nt = L - F + 1;
    hl.assign(nt, HostLevel());
    for (int k = 0; k < nt; k++) {
        Level &lv = h->lev[F + k];
        HostLevel &H = hl[k];
        H.n = lv.A.n;
        PCG_TRY(fetch(H.dinv, lv.dinv, H.n));
        PCG_TRY(fetch(H.dinv32, lv.dinv32, H.n));
        if (k + 1 < nt) {
            PCG_TRY(fetch(H.rp, lv.A.rp, H.n + 1));
            PCG_TRY(fetch(H.ci, lv.A.ci, (size_t)lv.A.nnz));
            PCG_TRY(fetch(H.v, lv.A.v, (size_t)lv.A.nnz));
            PCG_TRY(fetch(H.p, lv.p, H.n));
            PCG_TRY(fetch(H.p32, lv.p32, H.n));
            PCG_TRY(fetch(H.agg, lv.agg, H.n));
            PCG_TRY(fetch(H.rptr, lv.rptr, lv.nc + 1));
            PCG_TRY(fetch(H.ridx, lv.ridx, (size_t)H.rptr[lv.nc]));
        }
    }
    return AMG_OK;
}

template <typename T>
int plan_precision(amg_hier *h, int smem_max) {
    const int pi = sizeof(T) == 4 ? 0 : 1;
    h->tail_first[pi] = 0;
    int L = (int)h->lev.size() - 1;
    std::vector<double> ainv;
    PCG_TRY(fetch(ainv, h->Ainv, (size_t)h->nL * h->nL));
    for (int F = 1; F < L; F++) {
        if (h->lev[F].A.n > kSmemTailRows) continue;
        int nt = L - F + 1;
        if (nt > kMaxTailLevels) continue;
        std::vector<HostLevel> hl;
        PCG_TRY(fetch_tail_levels(h, F, hl));
        for (int ctas : {16, 8}) {
            SmemTailPlan plan = {};
            std::vector<unsigned char> blob;
            size_t bytes = build_plan<T>(hl, ainv, ctas, plan, blob);
            if (bytes > (size_t)smem_max || !cluster_fits<T>(ctas, bytes, smem_max)) continue;
            PCG_TRY(alloc(h->mem, &h->tail_blob[pi], blob.size()));
            PCG_CK(cudaMemcpy(h->tail_blob[pi], blob.data(), blob.size(), cudaMemcpyHostToDevice));
            h->tail_plan[pi] = plan;
            h->tail_smem[pi] = bytes;
            h->tail_ctas[pi] = ctas;
            h->tail_first[pi] = F;
            return AMG_OK;
        }
        // this level's tail does not fit: try the tail from the next level
    }
    return AMG_OK;
}

// The static blob of a planned tail formed again from the hierarchy's
// current values (same levels, same layout) and written over the old one, so
// captured launches keep their arguments.
template <typename T>
int refresh_precision(amg_hier *h) {
    const int pi = sizeof(T) == 4 ? 0 : 1;
    int F = h->tail_first[pi];
    if (F <= 0) return AMG_OK;
    std::vector<double> ainv;
    PCG_TRY(fetch(ainv, h->Ainv, (size_t)h->nL * h->nL));
    std::vector<HostLevel> hl;
    PCG_TRY(fetch_tail_levels(h, F, hl));
    SmemTailPlan plan = {};
    std::vector<unsigned char> blob;
    size_t bytes = build_plan<T>(hl, ainv, h->tail_ctas[pi], plan, blob);
    if (bytes != h->tail_smem[pi] || plan.static_bytes != h->tail_plan[pi].static_bytes) {
        set_error("amg_refresh: the shared-memory tail changed its layout");
        return AMG_ERR_CUDA;
    }
    PCG_CK(cudaMemcpy(h->tail_blob[pi], blob.data(), blob.size(), cudaMemcpyHostToDevice));
    return AMG_OK;
}

int setup_smem_tail(amg_hier *h) {
    h->tail_first[0] = h->tail_first[1] = 0;
    if ((int)h->lev.size() < 3) return AMG_OK;
    int smem_max = 0;
    PCG_CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    PCG_TRY(plan_precision<float>(h, smem_max));
    PCG_TRY(plan_precision<double>(h, smem_max));
    return AMG_OK;
}

int refresh_smem_tail(amg_hier *h) {
    PCG_TRY(refresh_precision<float>(h));
    PCG_TRY(refresh_precision<double>(h));
    return AMG_OK;
}

// Launches the tail for the V-cycle precision T (reads b and xpre of level
// tail_first[T], writes its x).
template <typename T>
int launch_smem_tail(amg_hier *h, cudaStream_t s) {
    int pi = sizeof(T) == 4 ? 0 : 1;
    Level &F = h->lev[h->tail_first[pi]];
    const T *b, *xpre;
    T *x;
    if constexpr (sizeof(T) == 4) {
        b = F.b32; xpre = F.xpre32; x = F.x32;
    } else {
        b = F.b64; xpre = F.xpre64; x = F.x64;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h->tail_ctas[pi]);
    cfg.blockDim = dim3(kTThreads);
    cfg.dynamicSmemBytes = h->tail_smem[pi];
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = h->tail_ctas[pi];
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = h->pdl ? 2 : 1;
    PCG_CK(cudaLaunchKernelEx(&cfg, k_tail_smem<T>, h->tail_plan[pi], (const unsigned char *)h->tail_blob[pi], b,
                              xpre, x, (const Ctl *)h->ctl));
    return AMG_OK;
}

template int launch_smem_tail<float>(amg_hier *, cudaStream_t);
template int launch_smem_tail<double>(amg_hier *, cudaStream_t);

}  // namespace pcgamg
