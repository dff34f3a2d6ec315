// split_launch.cuh -- the warp-pair temporal kernel (RDCNN_VARIANT_TEMPORAL2,
// temporal_split.cuh) and its host launcher for one (element type, depth);
// the split_*.cu units instantiate them so that the many (dtype, K, reaction,
// boundary) kernels compile in parallel.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "temporal_split.cuh"

namespace rdk {

// One warp pair per (band, strip): stages split between the two warps.  Both
// warps of a pair see the same `item`.
template <typename T, int K, int RX, int BC>
__global__ void __launch_bounds__(kSplitBlock)
k_temporal_split(const T *__restrict__ u, const T *__restrict__ v, T *__restrict__ un,
                 T *__restrict__ vn, int nn, int nm, int bands, int nitems, int rows, Coef<T> p) {
    pdl_wait();
    const int item = blockIdx.x * kSplitPairs + ((threadIdx.x >> 5) >> 1);
    if (item >= nitems) return;  // the whole pair, before any barrier
    temporal_split_item<T, K, RX, BC>(item, bands, u, v, un, vn, nn, nm, rows, p);
    pdl_trigger();
}

template <typename T, int K, int RX, int BC>
int split_blocks_per_sm() {
    static int cached = -1;
    if (cached < 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_temporal_split<T, K, RX, BC>, kSplitBlock, 0) !=
            cudaSuccess)
            nb = 1;
        cached = nb;
    }
    return cached;
}

// Rows per warp-pair strip for the requested rows (rows <= 0: the
// wave-quantisation model's choice).
template <typename T, int K>
int split_rows(int reaction, int boundary, int64_t nn, int64_t nm, int rows) {
    if (rows > 0) return rows;
    constexpr int V = Vec<T>::N;
    constexpr int H = (K + V - 1) / V;
    constexpr int OUTW = (32 - 2 * H) * V;
    const int bands = (int)((nm + OUTW - 1) / OUTW);
    int bps = 1;
    with_model(reaction, boundary, [&](auto rx, auto bc) {
        bps = split_blocks_per_sm<T, K, decltype(rx)::value, decltype(bc)::value>();
        return cudaSuccess;
    });
    return auto_rows_temporal(K, nn, nm, bands, bps, kSplitPairs);
}

// One launch of depth K (K >= 2; FP32 / FP64 planes, every model).
template <typename T, int K>
cudaError_t split_tk(int reaction, int boundary, const void *u, const void *v, void *un, void *vn, int64_t nn,
                     int64_t nm, const rdcnn_params &p, int rows, cudaStream_t s) {
    constexpr int V = Vec<T>::N;
    constexpr int H = (K + V - 1) / V;
    constexpr int OUTW = (32 - 2 * H) * V;
    const int bands = (int)((nm + OUTW - 1) / OUTW);
    rows = split_rows<T, K>(reaction, boundary, nn, nm, rows);
    const int strips = (int)((nn + rows - 1) / rows);
    const int64_t nitems = (int64_t)bands * strips;
    const unsigned grid = (unsigned)((nitems + kSplitPairs - 1) / kSplitPairs);
    const Coef<T> c = make_coef<T>(p, reaction);
    return with_model(reaction, boundary, [&](auto rx, auto bc) {
        const cudaError_t e = launch_k(k_temporal_split<T, K, decltype(rx)::value, decltype(bc)::value>, grid,
                                       kSplitBlock, 0, s, (const T *)u, (const T *)v, (T *)un, (T *)vn, (int)nn,
                                       (int)nm, bands, (int)nitems, rows, c);
        count_launches(1);
        return e;
    });
}

}  // namespace rdk

// Explicit instantiation of split_tk<TT, KK> and split_rows<TT, KK> / a
// declaration that another unit instantiates them.
#define RDK_SPLIT_TK_SIG(TT, KK)                                                                         \
    cudaError_t rdk::split_tk<TT, KK>(int, int, const void *, const void *, void *, void *, int64_t, int64_t, \
                                      const rdcnn_params &, int, cudaStream_t)
#define RDK_SPLIT_ROWS_SIG(TT, KK) int rdk::split_rows<TT, KK>(int, int, int64_t, int64_t, int)
#define RDK_INSTANTIATE_SPLIT(TT, KK) template RDK_SPLIT_TK_SIG(TT, KK); template RDK_SPLIT_ROWS_SIG(TT, KK);
#define RDK_EXTERN_SPLIT(TT, KK) extern template RDK_SPLIT_TK_SIG(TT, KK); extern template RDK_SPLIT_ROWS_SIG(TT, KK);
