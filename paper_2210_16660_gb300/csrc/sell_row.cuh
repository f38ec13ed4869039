// Row dot product over the sliced-ELL layout, shared by the solve kernels.
#pragma once

#include <cstdint>

namespace pcgamg {

// Sum over the stored entries of one sliced-ELL row: acc = sum_k a_k x(j_k),
// k in storage order. Column/value loads of U entries are issued before their
// gathers so each warp keeps several independent loads in flight. Large
// levels use U = 4 (bandwidth-bound, keeps registers low); small levels
// U = 16 so a row's loads take about two dependent round trips.
constexpr int kUnroll = 4;
constexpr int kUnrollSmall = 16;
constexpr int kSmallRows = 65536;

// Loads of the matrix stream: level-0 sweeps use evict-first loads (the
// matrix is read once per sweep and is larger than L2), coarser levels keep
// the default so the matrix can stay in L2 between the down and up sweeps.
template <bool STREAM, typename X>
__device__ __forceinline__ X ld_mat(const X *p) {
    if (STREAM) return __ldcs(p);
    return __ldg(p);
}

// Column of an entry: int32 column index, or an int16 offset from the row
// for levels whose every |col - row| fits in 16 bits.
__device__ __forceinline__ int col_of(int32_t c, int) { return c; }
__device__ __forceinline__ int col_of(int16_t c, int row) { return row + (int)c; }

template <int U, bool STREAM, typename IDX, typename T, typename F>
__device__ __forceinline__ T sell_row(const IDX *__restrict__ c, const T *__restrict__ a, int w, int row, F xval) {
    T acc = 0;
    int k = 0;
    for (; k + U <= w; k += U) {
        int j[U];
        T v[U], x[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            j[u] = col_of(ld_mat<STREAM>(c + 32 * (k + u)), row);
            v[u] = ld_mat<STREAM>(a + 32 * (k + u));
        }
#pragma unroll
        for (int u = 0; u < U; u++) x[u] = xval(j[u]);
#pragma unroll
        for (int u = 0; u < U; u++) acc += v[u] * x[u];
    }
    for (; k < w; k++) acc += ld_mat<STREAM>(a + 32 * k) * xval(col_of(ld_mat<STREAM>(c + 32 * k), row));
    return acc;
}

}  // namespace pcgamg
