// amg_residual_noalloc: the true residual r = b - A x and its norm without
// allocating any device memory.
//
// Some callers cannot allocate device memory once their solve loop runs: an
// application that hands the whole device to its own memory pool (a CFD code
// sharing the GPU with other solvers, say) or a time-step loop that cannot
// afford the device-wide synchronisation a cudaMalloc/cudaFree may imply.
// This entry point serves them: the caller passes the inputs and outputs, and
// the only scratch (per-block partial sums and a completion counter) lives in
// a fixed-size array that is part of the library image.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds kNaScratchBytes of it until the process exits. In host code
// its name is only a stand-in, not a device address, so the address is
// looked up once per device with cudaGetSymbolAddress (on the first call made
// with that device current) and passed to the kernel. Every call shares the
// array; calls that overlap on the GPU race on it.
#include <cstdio>
#include <mutex>

#include "internal.cuh"

namespace pcgamg {
namespace {

constexpr int kNaBlock = 256;
constexpr int kNaMaxBlocks = 32768;                        // one row per thread
constexpr int64_t kNaMaxRows = (int64_t)kNaMaxBlocks * kNaBlock;  // 8,388,608 rows
// layout: partial sums [2 * kNaMaxBlocks doubles] | norms [2 doubles] | counter
constexpr size_t kNaPartialBytes = 2 * sizeof(double) * (size_t)kNaMaxBlocks;
constexpr size_t kNaScratchBytes = kNaPartialBytes + 256;

static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
void *g_na_addr[kNaMaxDevices] = {};

// Device address of the scratch array for the current device (looked up on
// the first call per device).
int na_scratch(void **out) {
    int dev = 0;
    PCG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("amg_residual_noalloc: device ordinal %d out of range", dev);
        return AMG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error("amg_residual_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return AMG_ERR_CUDA;
        }
        g_na_addr[dev] = p;
    }
    *out = g_na_addr[dev];
    return AMG_OK;
}

__device__ __forceinline__ int na_col(int32_t c, int) { return c; }
__device__ __forceinline__ int na_col(int16_t c, int row) { return row + (int)c; }

// One row per thread over the sliced-ELL level-0 matrix; block sums of
// ||r||^2 and ||b||^2 go to the scratch partials; the last block to finish
// adds them in block order and writes both norms.
template <typename IDX>
__global__ void __launch_bounds__(kNaBlock) k_residual_na(int n, const int32_t *__restrict__ sptr,
                                                          const IDX *__restrict__ col,
                                                          const double *__restrict__ val,
                                                          const double *__restrict__ b,
                                                          const double *__restrict__ x, double *__restrict__ r,
                                                          double *partials, double *norms, unsigned *counter) {
    __shared__ double sa[kNaBlock / 32], sb[kNaBlock / 32];
    __shared__ bool last;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0.0, bb = 0.0;
    if (i < n) {
        int s = i >> 5, lane = i & 31;
        int32_t base = __ldg(sptr + s);
        int w = (__ldg(sptr + s + 1) - base) >> 5;
        double acc = 0.0;
        for (int k = 0; k < w; k++) {
            int32_t e = base + 32 * k + lane;
            acc += __ldg(val + e) * __ldg(x + na_col(__ldg(col + e), i));
        }
        double bi = __ldg(b + i);
        double ri = bi - acc;
        r[i] = ri;
        rr = ri * ri;
        bb = bi * bi;
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sa[w] = rr; sb[w] = bb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int k = 0; k < kNaBlock / 32; k++) { a += sa[k]; c += sb[k]; }
        partials[blockIdx.x] = a;
        partials[gridDim.x + blockIdx.x] = c;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        a += __ldcg(partials + k);
        c += __ldcg(partials + gridDim.x + k);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    __syncthreads();
    if (lane == 0) { sa[w] = a; sb[w] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tc = 0.0;
        for (int k = 0; k < kNaBlock / 32; k++) { ta += sa[k]; tc += sb[k]; }
        norms[0] = sqrt(ta);
        norms[1] = sqrt(tc);
        *counter = 0;
    }
}

// [a, a + n) and [b, b + n) share an address
bool na_overlap(const double *a, const double *b, int64_t n) {
    uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b, len = (uintptr_t)n * sizeof(double);
    return a0 < b0 + len && b0 < a0 + len;
}

bool na_is_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace pcgamg

using namespace pcgamg;

extern "C" int amg_residual_noalloc(amg_handle h, const double *b, const double *x, double *r, double *norms,
                                    void *stream) {
    set_error("");
    if (!h || !b || !x || !r || !norms) {
        set_error("amg_residual_noalloc: NULL argument");
        return AMG_ERR_ARG;
    }
    const Level &l0 = h->lev[0];
    int n = l0.A.n;
    if ((int64_t)n > kNaMaxRows) {
        set_error("amg_residual_noalloc: %d rows exceed the limit of %lld rows (the fixed scratch holds %d "
                  "block partial sums)", n, (long long)kNaMaxRows, kNaMaxBlocks);
        return AMG_ERR_ARG;
    }
    if (!na_is_device(b) || !na_is_device(x) || !na_is_device(r)) {
        set_error("amg_residual_noalloc: b, x and r must be device pointers (host vectors would need staging "
                  "memory)");
        return AMG_ERR_ARG;
    }
    // r is written while other threads still read x and b as gathered
    // columns: it must not share memory with either
    if (na_overlap(r, b, n) || na_overlap(r, x, n)) {
        set_error("amg_residual_noalloc: r overlaps b or x");
        return AMG_ERR_ARG;
    }
    int dev = 0;
    PCG_CK(cudaGetDevice(&dev));
    if (dev != h->device) {
        set_error("amg_residual_noalloc: the current device %d is not the handle's device %d", dev, h->device);
        return AMG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool host_norms = !na_is_device(norms);
    if (host_norms) {
        // a host norms pointer makes the call wait, which a stream capture forbids
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        PCG_CK(cudaStreamIsCapturing(s, &cap));
        if (cap != cudaStreamCaptureStatusNone) {
            set_error("amg_residual_noalloc: norms must be a device pointer while the stream is captured");
            return AMG_ERR_ARG;
        }
    }
    void *base = nullptr;
    PCG_TRY(na_scratch(&base));
    double *partials = static_cast<double *>(base);
    double *dnorms = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + kNaPartialBytes);
    unsigned *counter = reinterpret_cast<unsigned *>(static_cast<unsigned char *>(base) + kNaPartialBytes + 64);
    PCG_CK(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
    int blocks = (n + kNaBlock - 1) / kNaBlock;
    if (blocks < 1) blocks = 1;
    if (l0.S.col16)
        k_residual_na<int16_t><<<blocks, kNaBlock, 0, s>>>(n, l0.S.sptr, l0.S.col16, l0.S.v64, b, x, r, partials,
                                                           dnorms, counter);
    else
        k_residual_na<int32_t><<<blocks, kNaBlock, 0, s>>>(n, l0.S.sptr, l0.S.col, l0.S.v64, b, x, r, partials,
                                                           dnorms, counter);
    PCG_LAUNCH_CK();
    PCG_CK(cudaMemcpyAsync(norms, dnorms, 2 * sizeof(double), cudaMemcpyDefault, s));
    if (host_norms) PCG_CK(cudaStreamSynchronize(s));
    return AMG_OK;
}
