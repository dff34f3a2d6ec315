// temporal_launch.cuh -- host launcher of k_temporal for one depth K; each
// temporal_*.cu unit instantiates it for a range of depths, so the many
// (dtype, K, reaction, boundary) kernels compile in parallel.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "temporal.cuh"

namespace rdk {

template <typename T, int K, int RX, int BC>
int temporal_blocks_per_sm() {
    static int cached = -1;
    if (cached < 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_temporal<T, K, RX, BC>, kTemporalBlock, 0) !=
            cudaSuccess)
            nb = 1;
        cached = nb;
    }
    return cached;
}

template <typename T, int K>
constexpr int temporal_bands(int64_t nm) {
    constexpr int V = Vec<T>::N;
    constexpr int H = (K + V - 1) / V;
    constexpr int OUTW = (32 - 2 * H) * V;
    return (int)((nm + OUTW - 1) / OUTW);
}

template <typename T, int K>
int temporal_rows(int reaction, int boundary, int64_t nn, int64_t nm, int rows) {
    if (rows > 0) return rows;
    int r = 0;
    with_model(reaction, boundary, [&](auto rx, auto bc) {
        r = auto_rows_temporal(K, nn, nm, temporal_bands<T, K>(nm),
                               temporal_blocks_per_sm<T, K, decltype(rx)::value, decltype(bc)::value>(),
                               kTemporalBlock / 32);
        return cudaSuccess;
    });
    return r;
}

template <typename T, int K>
cudaError_t temporal_launch(int reaction, int boundary, const void *u, const void *v, void *un,
                            void *vn, int64_t nn, int64_t nm, const rdcnn_params &p, int rows,
                            cudaStream_t s) {
    const int bands = temporal_bands<T, K>(nm);
    const Coef<CT<T>> c = make_coef<CT<T>>(p, reaction);
    const int r = temporal_rows<T, K>(reaction, boundary, nn, nm, rows);
    return with_model(reaction, boundary, [&](auto rx, auto bc) {
        constexpr int RX = decltype(rx)::value;
        constexpr int BC = decltype(bc)::value;
        const int strips = (int)((nn + r - 1) / r);
        const int64_t nwarps = (int64_t)bands * strips;
        const int wpb = kTemporalBlock / 32;
        const unsigned grid = (unsigned)((nwarps + wpb - 1) / wpb);
        const cudaError_t e = launch_k(k_temporal<T, K, RX, BC>, grid, kTemporalBlock, 0, s, (const T *)u,
                                       (const T *)v, (T *)un, (T *)vn, (int)nn, (int)nm, bands, (int)nwarps, r, c);
        count_launches(1);
        return e;
    });
}

}  // namespace rdk

// Explicit instantiation of temporal_launch<TT, KK> and temporal_rows<TT, KK>.
#define RDK_INSTANTIATE_TEMPORAL(TT, KK)                                                        \
    template cudaError_t rdk::temporal_launch<TT, KK>(int, int, const void *, const void *, void *, \
                                                      void *, int64_t, int64_t, const rdcnn_params &, \
                                                      int, cudaStream_t);                       \
    template int rdk::temporal_rows<TT, KK>(int, int, int64_t, int64_t, int);
