// Row dot product over the sliced-ELL layout, shared by the solve kernels.
#pragma once

#include <cstdint>
#include <type_traits>

#include "internal.cuh"

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

// Column/value loads of entries k..k+U-1 of a row (masked past w: column =
// row, value 0, never used).
template <int U, bool STREAM, typename IDX, typename T>
__device__ __forceinline__ void sell_chunk(const IDX *__restrict__ c, const T *__restrict__ a, int k, int w, int row,
                                           int (&j)[U], T (&v)[U]) {
#pragma unroll
    for (int u = 0; u < U; u++) {
        if (k + u < w) {
            j[u] = col_of(ld_mat<STREAM>(c + 32 * (k + u)), row);
            v[u] = ld_mat<STREAM>(a + 32 * (k + u));
        } else {
            j[u] = row;
            v[u] = T(0);
        }
    }
}

// Entries are summed one by one in storage order (acc += a_k x(j_k)), so
// the result does not depend on U or on the pipelining. For U <= 4 (large
// levels) the column/value loads of the next chunk are issued before the
// FMAs of the current one, so a chunk costs about one dependent round trip
// (its gathers) instead of two, and the last, partial chunk is loaded as one
// masked chunk. U = 16 (small levels) loads whole chunks, then the rest one
// entry at a time (its registers allow no second buffer).
template <int U, bool STREAM, typename IDX, typename T, typename F>
__device__ __forceinline__ T sell_row(const IDX *__restrict__ c, const T *__restrict__ a, int w, int row, F xval) {
    T acc = 0;
    if constexpr (U <= 4) {
        int j[U];
        T v[U];
        sell_chunk<U, STREAM>(c, a, 0, w, row, j, v);
        for (int k = 0; k < w; k += U) {
            T x[U];
#pragma unroll
            for (int u = 0; u < U; u++) x[u] = (k + u < w) ? xval(j[u]) : T(0);
            int jn[U];
            T vn[U];
            sell_chunk<U, STREAM>(c, a, k + U, w, row, jn, vn);
#pragma unroll
            for (int u = 0; u < U; u++)
                if (k + u < w) acc += v[u] * x[u];
#pragma unroll
            for (int u = 0; u < U; u++) {
                j[u] = jn[u];
                v[u] = vn[u];
            }
        }
    } else {
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
    }
    return acc;
}

// One sliced-ELL row split into its static part, loaded by load() (slice
// base and width, the first chunk's columns and values: matrix data, written
// only by setup and refresh, so a kernel may load it before it waits for the
// preceding kernel), and the product, dot(), which gathers x. Every chunk of
// U entries is loaded masked, the next chunk's loads issued before the
// current chunk's gathers, so a row of w entries costs about ceil(w / U)
// dependent gather round trips whatever U is. Entries are summed one by one
// in storage order (acc += a_k x(j_k)), as in sell_row.
//
// With upat (the level's shared offset patterns), a slice stored with one takes
// column i + o_k from the pattern, one offset per entry column of the slice
// read by every lane of the warp, instead of one column index per entry: the
// column of entry k is rb + c[cs k], with (c, cs, rb) = (the row's column
// indices, 32, row or 0) or (the slice's pattern, 1, row).
template <typename IDX>
__device__ __forceinline__ int col_base(int row);
template <>
__device__ __forceinline__ int col_base<int32_t>(int) { return 0; }
template <>
__device__ __forceinline__ int col_base<int16_t>(int row) { return row; }

template <int U, bool STREAM, typename IDX, typename T>
struct SellRow {
    const IDX *c;
    const T *a;
    int w, cs, rb;
    int j[U];
    T v[U];

    __device__ __forceinline__ void chunk(int k, int row, int (&jj)[U], T (&vv)[U]) {
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (k + u < w) {
                jj[u] = rb + (int)ld_mat<STREAM>(c + cs * (k + u));
                vv[u] = ld_mat<STREAM>(a + 32 * (k + u));
            } else {
                jj[u] = row;
                vv[u] = T(0);
            }
        }
    }

    __device__ __forceinline__ void load(const int32_t *__restrict__ sptr, const IDX *__restrict__ col,
                                         const T *__restrict__ val, int row,
                                         const IDX *__restrict__ upat = nullptr) {
        const int s = row >> 5, lane = row & 31;
        const int32_t base = __ldg(sptr + s);
        w = (__ldg(sptr + s + 1) - base) >> 5;
        a = val + base + lane;
        c = col + base + lane;
        cs = 32;
        rb = col_base<IDX>(row);
        if (upat && __ldg(upat + (base >> 5)) != kNoPattern<IDX>) {
            c = upat + (base >> 5);
            cs = 1;
            rb = row;
        }
        chunk(0, row, j, v);
    }

    template <typename F>
    __device__ __forceinline__ T dot(int row, F xval) {
        T acc = 0;
        for (int k = 0; k < w; k += U) {
            T x[U];
#pragma unroll
            for (int u = 0; u < U; u++) x[u] = (k + u < w) ? xval(j[u]) : T(0);
            int jn[U];
            T vn[U];
            chunk(k + U, row, jn, vn);
#pragma unroll
            for (int u = 0; u < U; u++)
                if (k + u < w) acc += v[u] * x[u];
#pragma unroll
            for (int u = 0; u < U; u++) {
                j[u] = jn[u];
                v[u] = vn[u];
            }
        }
        return acc;
    }
};

// Rows of level-0 slices stored with a shared offset pattern and at most
// kPatW entries per row: load() requests every value of the row at once
// (kPatW registers), and dot() gathers x in chunks of kPatG entries whose
// columns come from the pattern alone (L1-resident), so the gathers do not
// wait for the values and a row costs about one DRAM latency, overlapped
// with ceil(w / kPatG) gather round trips. Rows of other slices go through a
// 4-entry SellRow. Entries are summed one by one in storage order.
constexpr int kPatW = 32, kPatG = 8;
// chunk depth that selects PatRow in the sweeps' Row type
constexpr int kPatRow = 32;

template <bool STREAM, typename IDX, typename T>
struct PatRow {
    const IDX *pat;
    int w;
    bool uni;
    T v[kPatW];
    SellRow<4, STREAM, IDX, T> R;

    __device__ __forceinline__ void load(const int32_t *__restrict__ sptr, const IDX *__restrict__ col,
                                         const T *__restrict__ val, int row,
                                         const IDX *__restrict__ upat = nullptr) {
        const int s = row >> 5, lane = row & 31;
        const int32_t base = __ldg(sptr + s);
        w = (__ldg(sptr + s + 1) - base) >> 5;
        pat = upat + (base >> 5);
        uni = upat && w <= kPatW && __ldg(pat) != kNoPattern<IDX>;
        if (uni) {
            const T *a = val + base + lane;
#pragma unroll
            for (int k = 0; k < kPatW; k++) v[k] = k < w ? ld_mat<STREAM>(a + 32 * k) : T(0);
        } else {
            R.load(sptr, col, val, row, upat);
        }
    }

    template <typename F>
    __device__ __forceinline__ T dot(int row, F xval) {
        if (!uni) return R.dot(row, xval);
        T acc = 0;
#pragma unroll
        for (int k0 = 0; k0 < kPatW; k0 += kPatG) {
            if (k0 >= w) break;
            T x[kPatG];
#pragma unroll
            for (int u = 0; u < kPatG; u++) x[u] = k0 + u < w ? xval(row + (int)__ldg(pat + k0 + u)) : T(0);
#pragma unroll
            for (int u = 0; u < kPatG; u++)
                if (k0 + u < w) acc += v[k0 + u] * x[u];
        }
        return acc;
    }
};

// Rows read by kMlL lanes each (the multi-lane launch shape of the coarse
// levels). In a pass, lane q of a row loads the entries [k0 + q c,
// min(w, k0 + (q + 1) c)) with c = min(ceil(w / kMlL), kMlC), and gathers x
// for all of them at once; the row's sum is then chained through its lanes
// in storage order (lane q continues from lane q - 1's accumulator, passed by
// a shuffle), so the FMAs are those of SellRow, in the same order. A row
// costs one gather round trip per pass (rows of up to kMlL kMlC entries take
// one pass). The lanes of a warp are 8 rows of one slice, so every lane runs
// the same number of passes; a row past the last one (live = false) loads
// and gathers nothing but takes part in the shuffles.
constexpr int kMlL = 4, kMlC = 12;

template <bool STREAM, typename IDX, typename T>
struct MlRow {
    const IDX *cp;
    const T *ap;
    int w, c, k0, q;
    bool live;
    int j[kMlC];
    T v[kMlC];

    __device__ __forceinline__ int count() const {
        const int lo = k0 + q * c;
        const int hi = min(w, k0 + (q + 1) * c);
        return live && hi > lo ? hi - lo : 0;
    }

    __device__ __forceinline__ void fill(int row) {
        const int lo = k0 + q * c, cnt = count();
#pragma unroll
        for (int m = 0; m < kMlC; m++) {
            if (m < cnt) {
                j[m] = col_of(ld_mat<STREAM>(cp + 32 * (lo + m)), row);
                v[m] = ld_mat<STREAM>(ap + 32 * (lo + m));
            } else {
                j[m] = row;
                v[m] = T(0);
            }
        }
    }

    __device__ __forceinline__ void load(const int32_t *__restrict__ sptr, const IDX *__restrict__ col,
                                         const T *__restrict__ val, int row, int lane_q, bool is_live) {
        const int s = row >> 5, r = row & 31;
        const int32_t base = __ldg(sptr + s);
        w = (__ldg(sptr + s + 1) - base) >> 5;
        cp = col + base + r;
        ap = val + base + r;
        c = min((w + kMlL - 1) / kMlL, kMlC);
        k0 = 0;
        q = lane_q;
        live = is_live;
        fill(row);
    }

    template <typename F>
    __device__ __forceinline__ T dot(int row, F xval) {
        const int g0 = (int)(threadIdx.x & 31) & ~(kMlL - 1);
        T acc = 0;
        for (;;) {
            const int cnt = count();
            T x[kMlC];
#pragma unroll
            for (int m = 0; m < kMlC; m++) x[m] = m < cnt ? xval(j[m]) : T(0);
#pragma unroll
            for (int qq = 0; qq < kMlL; qq++) {
                if (q == qq) {
#pragma unroll
                    for (int m = 0; m < kMlC; m++)
                        if (m < cnt) acc += v[m] * x[m];
                }
                acc = __shfl_sync(0xffffffffu, acc, g0 + qq);
            }
            k0 += kMlL * c;
            if (k0 >= w) break;
            fill(row);
        }
        return acc;
    }
};

template <int U, bool STREAM, typename IDX, typename T>
using RowOf = typename std::conditional<U == kPatRow, PatRow<STREAM, IDX, T>, SellRow<U, STREAM, IDX, T>>::type;

}  // namespace pcgamg
