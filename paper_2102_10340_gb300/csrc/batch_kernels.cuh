// batch_kernels.cuh -- the batched temporal kernel: many independent RD-CNN
// instances (a parameter sweep in the sense of Sec. III.A-III.B), each with
// its own size and gene, advanced by one launch per k time steps.  A warp
// finds its instance by binary search over the table's warp offsets and runs
// the single-grid pipeline of temporal.cuh with that instance's gene.  The
// launchers for each (element type, halo) are instantiated in the batch_*.cu
// units so that they compile in parallel.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "temporal.cuh"

namespace rdk {

constexpr int kBatchBlock = 32 * kTemporalWarps;

struct BatchDesc {
    const void *u, *v;
    void *su, *sv;
    int nn, nm, bands, rows;
    long long warp_begin;
    double dt, Du, Dv, cm4, mthird, meps, ebm4, mepsa;  // as Coef<double>
};

template <typename T, int K, int H, int RX, int BC>
__global__ void __launch_bounds__(kBatchBlock)
k_batch_temporal(const BatchDesc *__restrict__ tab, int n, long long nwarps, int flip) {
    pdl_wait();
    const long long wid = (long long)blockIdx.x * (kBatchBlock / 32) + (threadIdx.x >> 5);
    if (wid >= nwarps) return;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].warp_begin <= wid) lo = mid; else hi = mid - 1;
    }
    const BatchDesc &d = tab[lo];
    const int local = (int)(wid - d.warp_begin);
    const int bands = d.bands;
    typedef CT<T> C;  // arithmetic type (FP32 for 16-bit planes)
    Coef<C> p;
    p.dt = C(d.dt); p.Du = C(d.Du); p.Dv = C(d.Dv); p.cm4 = C(d.cm4);
    p.mthird = C(d.mthird); p.meps = C(d.meps); p.ebm4 = C(d.ebm4); p.mepsa = C(d.mepsa);
    const T *su = (const T *)(flip ? d.su : d.u);
    const T *sv = (const T *)(flip ? d.sv : d.v);
    T *du = (T *)(flip ? d.u : d.su);
    T *dv = (T *)(flip ? d.v : d.sv);
    temporal_strip<T, K, H, RX, BC>(local % bands, local / bands, su, sv, du, dv, d.nn, d.nm, d.rows, p);
    pdl_trigger();
}

// One depth, every model of the single-grid kernels (T = float, double,
// __nv_bfloat16 or __half planes; 16-bit planes round once per launch).
template <typename T, int K, int H>
cudaError_t batch_launch_khr(int reaction, int boundary, const BatchDesc *tab, int n, long long nwarps,
                             int flip, cudaStream_t s) {
    const int wpb = kBatchBlock / 32;
    const unsigned grid = (unsigned)((nwarps + wpb - 1) / wpb);
    return with_model(reaction, boundary, [&](auto rx, auto bc) {
        const cudaError_t e = launch_k(k_batch_temporal<T, K, H, decltype(rx)::value, decltype(bc)::value>,
                                       grid, kBatchBlock, 0, s, tab, n, nwarps, flip);
        count_launches(1);
        return e;
    });
}

}  // namespace rdk

// Explicit instantiation of batch_launch_khr<TT, KK, HH> / a declaration that
// another unit instantiates it.
#define RDK_BATCH_KHR_SIG(TT, KK, HH)                                                                  \
    cudaError_t rdk::batch_launch_khr<TT, KK, HH>(int, int, const rdk::BatchDesc *, int, long long, int, \
                                                  cudaStream_t)
#define RDK_INSTANTIATE_BATCH(TT, KK, HH) template RDK_BATCH_KHR_SIG(TT, KK, HH);
#define RDK_EXTERN_BATCH(TT, KK, HH) extern template RDK_BATCH_KHR_SIG(TT, KK, HH);
