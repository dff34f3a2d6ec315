// forward.cu -- forward kernels for Eq. 1-3 (Sec. II.A) and the launchers of
// every forward variant (torus or zero flux; FitzHugh-Nagumo, pure diffusion
// or CeNN cell; float / double planes, or bf16 / half planes computed in FP32).
//
//  k_step1     one time step per launch (float / double planes).  A warp owns a band of 32*V columns
//              (V = 4 floats / 2 doubles per lane, one 16-byte load) and walks
//              down a strip of rows, keeping rows i-1, i, i+1 in registers and
//              prefetching row i+2.  Horizontal neighbours come from the
//              adjacent lane by warp shuffle; the two band-edge values are
//              read from global memory (L1/L2 hits).  Each input byte is read
//              once from DRAM and each output byte written once: 16 B per
//              cell-step in FP32, the algorithmic minimum.
//  k_temporal  K time steps per launch.  A warp loads a band of 32*V columns
//              that overlaps its neighbours by H = ceil(K/V) lanes on each
//              side, and walks down rows r0-K .. r0+R+K-1 of its strip.  Stage
//              s of a K-deep register pipeline turns three rows of stage s-1
//              into one row of stage s, so a row is read once and leaves as
//              K-step-advanced output: DRAM traffic is 16 B per cell per K
//              steps.  Lanes within K columns of the band edge hold stale
//              values after K steps and do not store.
//  k_generic   one thread per cell, scalar loads: any size and alignment.
//
// All three evaluate cells with rdk::cell_update, so they produce identical
// bits for identical inputs (for 16-bit planes: at the same steps per
// launch, which is also the rounding interval).  Under the zero-flux boundary the single-step
// and generic kernels clamp neighbour indices into the grid (the ghost cell
// is the edge cell); the temporal kernel loads mirrored halos instead
// (temporal.cuh).  k_temporal's launchers live in temporal_launch.cuh and are
// instantiated in the temporal_*.cu units, the warp-pair variant's
// (k_temporal_split) in split_launch.cuh and the split_*.cu units; they
// compile in parallel.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "temporal.cuh"
#include "split_launch.cuh"

// the warp-pair kernels compile in split_f32a.cu .. split_f32c.cu and split_f64.cu
RDK_EXTERN_SPLIT(float, 2) RDK_EXTERN_SPLIT(float, 3) RDK_EXTERN_SPLIT(float, 4) RDK_EXTERN_SPLIT(float, 5)
RDK_EXTERN_SPLIT(float, 6) RDK_EXTERN_SPLIT(float, 7) RDK_EXTERN_SPLIT(float, 8)
RDK_EXTERN_SPLIT(double, 2) RDK_EXTERN_SPLIT(double, 3) RDK_EXTERN_SPLIT(double, 4)

namespace rdk {

namespace {

// 72 registers.  4096^2 FP32, 400 back-to-back launches (Gcell-updates/s; 2 / 4 / 8 rows per warp):
// 32 threads 245 / 389 / 372, 64 threads 398 / 392 / 364, 128 threads 393 / 393 / 362,
// 256 threads 369 / 385 / 345.
constexpr int kStep1Block = 64;

// --------------------------------------------------------------------------- single step

// FP32 / FP64 planes (16-bit planes take the ring-staged pipeline at k = 1,
// see step1_t).
template <typename T, int RX, int BC>
__global__ void __launch_bounds__(kStep1Block)
k_step1(const T *__restrict__ u, const T *__restrict__ v, T *__restrict__ un,
        T *__restrict__ vn, int nn, int nm, int bands, int nwarps, int rows, Coef<T> p) {
    constexpr int V = Vec<T>::N;
    constexpr bool zf = (BC == BC_MIRROR);
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * (kStep1Block / 32) + (threadIdx.x >> 5);
    if (wid >= nwarps) return;  // whole warps only
    const int band = wid % bands;
    const int strip = wid / bands;
    const int col = band * 32 * V + lane * V;
    const bool active = col < nm;
    // neighbour columns beyond the edges: wrapped, or the edge cell itself
    const int colw = (col == 0) ? (zf ? 0 : nm - 1) : col - 1;
    const int cole = (col + V >= nm) ? (zf ? nm - 1 : 0) : col + V;
    const bool edge_w = (lane == 0);
    const bool edge_e = active && (lane == 31 || col + V >= nm);
    const int r0 = strip * rows;
    const int r1 = min(r0 + rows, nn);

    Slice<T> nor, cen, sou, pre;
    T cw_u = 0, ce_u = 0, cw_v = 0, ce_v = 0;  // band-edge values of row "cen"
    T sw_u = 0, se_u = 0, sw_v = 0, se_v = 0;  // ... of row "sou"
    T pw_u = 0, pe_u = 0, pw_v = 0, pe_v = 0;  // ... of row "pre"
    zero_slice(nor); zero_slice(cen); zero_slice(sou); zero_slice(pre);

    int rn = (r0 == 0) ? (zf ? 0 : nn - 1) : r0 - 1;
    int rc = r0;
    int rs = (r0 + 1 == nn) ? (zf ? nn - 1 : 0) : r0 + 1;
    if (active) {
        load_slice(nor, u, v, (int64_t)rn * nm + col);
        load_slice(cen, u, v, (int64_t)rc * nm + col);
        load_slice(sou, u, v, (int64_t)rs * nm + col);
    }
    if (edge_w) {
        cw_u = __ldg(u + (int64_t)rc * nm + colw); cw_v = __ldg(v + (int64_t)rc * nm + colw);
        sw_u = __ldg(u + (int64_t)rs * nm + colw); sw_v = __ldg(v + (int64_t)rs * nm + colw);
    }
    if (edge_e) {
        ce_u = __ldg(u + (int64_t)rc * nm + cole); ce_v = __ldg(v + (int64_t)rc * nm + cole);
        se_u = __ldg(u + (int64_t)rs * nm + cole); se_v = __ldg(v + (int64_t)rs * nm + cole);
    }

    for (int r = r0; r < r1; ++r) {
        // prefetch row r+2 (wrapped) while row r is computed
        const bool more = (r + 1 < r1);
        const int rp = (rs + 1 == nn) ? (zf ? nn - 1 : 0) : rs + 1;
        if (more) {
            if (active) load_slice(pre, u, v, (int64_t)rp * nm + col);
            if (edge_w) { pw_u = __ldg(u + (int64_t)rp * nm + colw); pw_v = __ldg(v + (int64_t)rp * nm + colw); }
            if (edge_e) { pe_u = __ldg(u + (int64_t)rp * nm + cole); pe_v = __ldg(v + (int64_t)rp * nm + cole); }
        }
        T wu = __shfl_up_sync(kFull, cen.u[V - 1], 1);
        T eu = __shfl_down_sync(kFull, cen.u[0], 1);
        T wv = __shfl_up_sync(kFull, cen.v[V - 1], 1);
        T ev = __shfl_down_sync(kFull, cen.v[0], 1);
        if (edge_w) { wu = cw_u; wv = cw_v; }
        if (edge_e) { eu = ce_u; ev = ce_v; }
        Slice<T> out;
        slice_update<T, RX>(nor, cen, sou, wu, eu, wv, ev, p, out);
        if (active) {
            const int64_t off = (int64_t)r * nm + col;
            store_vec<T>(un + off, out.u);
            store_vec<T>(vn + off, out.v);
        }
        nor = cen; cen = sou; sou = pre;
        cw_u = sw_u; ce_u = se_u; cw_v = sw_v; ce_v = se_v;
        sw_u = pw_u; se_u = pe_u; sw_v = pw_v; se_v = pe_v;
        rs = rp;
    }
    pdl_trigger();
}

// --------------------------------------------------------------------------- temporal blocking

// --------------------------------------------------------------------------- generic

template <typename T, int RX, int BC>
__global__ void __launch_bounds__(256)
k_generic(const T *__restrict__ u, const T *__restrict__ v, T *__restrict__ un,
          T *__restrict__ vn, int nn, int nm, Coef<CT<T>> p) {
    constexpr bool zf = (BC == BC_MIRROR);
    pdl_wait();
    const int64_t n = (int64_t)nn * nm;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / nm);
        const int j = (int)(idx - (int64_t)i * nm);
        const int ip = (i + 1 == nn) ? (zf ? i : 0) : i + 1;
        const int im = (i == 0) ? (zf ? 0 : nn - 1) : i - 1;
        const int jp = (j + 1 == nm) ? (zf ? j : 0) : j + 1;
        const int jm = (j == 0) ? (zf ? 0 : nm - 1) : j - 1;
        const int64_t ri = (int64_t)i * nm;
        const int64_t rp = (int64_t)ip * nm;
        const int64_t rm = (int64_t)im * nm;
        CT<T> ou, ov;
        cell_update<CT<T>, RX>(load1(u + ri + j), load1(u + rm + j), load1(u + rp + j), load1(u + ri + jm),
                               load1(u + ri + jp), load1(v + ri + j), load1(v + rm + j), load1(v + rp + j),
                               load1(v + ri + jm), load1(v + ri + jp), p, ou, ov);
        un[idx] = to_storage<T>(ou);
        vn[idx] = to_storage<T>(ov);
    }
    pdl_trigger();
}

template <typename T>
__global__ void __launch_bounds__(256)
k_init(const T *x, T *u, T *v, CT<T> ka, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const T t = to_storage<T>(mul_rn(ka, to_compute<T>(x[i])));  // x may alias u: plain loads
        u[i] = t;
        v[i] = t;
    }
}

template <typename T>
cudaError_t step1_t(int reaction, int boundary, const void *u, const void *v, void *un, void *vn,
                    int64_t nn, int64_t nm, const rdcnn_params &p, int rows, cudaStream_t s) {
    if constexpr (!is_f32_f64<T>()) {
        // 16-bit planes: a row carries half the bytes, and keeping HBM busy needs
        // more rows in flight than the register prefetch above holds; the
        // cp.async ring of the temporal pipeline at depth 1 keeps three per warp
        // (same arithmetic, one rounding per step: the same bits), with 8 values
        // (16 bytes) per lane when NM and the alignment allow.
        if (nm % 8 == 0 && aligned16(u) && aligned16(v) && aligned16(un) && aligned16(vn))
            return temporal_launch<Wide<T>, 1>(reaction, boundary, u, v, un, vn, nn, nm, p, rows, s);
        return temporal_launch<T, 1>(reaction, boundary, u, v, un, vn, nn, nm, p, rows, s);
    } else {
        constexpr int V = Vec<T>::N;
        const int bands = (int)((nm + 32 * V - 1) / (32 * V));
        const int strips = (int)((nn + rows - 1) / rows);
        const int64_t nwarps = (int64_t)bands * strips;
        const int wpb = kStep1Block / 32;
        const unsigned grid = (unsigned)((nwarps + wpb - 1) / wpb);
        const Coef<T> c = make_coef<T>(p, reaction);
        return with_model(reaction, boundary, [&](auto rx, auto bc) {
            const cudaError_t e = launch_k(k_step1<T, decltype(rx)::value, decltype(bc)::value>, grid,
                                           kStep1Block, 0, s, (const T *)u, (const T *)v, (T *)un, (T *)vn,
                                           (int)nn, (int)nm, bands, (int)nwarps, rows, c);
            count_launches(1);
            return e;
        });
    }
}

}  // namespace

// Rows per warp strip when the caller gives none.  Small grids use short
// strips (few warps exist at all); large grids pick, among a few lengths,
// the one that minimises waves x (rows + 2K) -- the work of the slowest SM
// when every resident warp slot is busy -- so a launch does not spill a
// nearly empty second wave (e.g. 4096^2, K=8: 128 rows = 1184 warps, one
// wave on 152 SMs at 8 warps each; 112 rows = 1369 warps, two waves).
int auto_rows_temporal(int K, int64_t nn, int64_t nm, int bands, int blocks_per_sm,
                       int warps_per_block) {
    const int64_t cells = nn * nm;
    // size classes from a sweep at 256^2 .. 2048^2 (with the light-cone fill):
    // 512^2, k = 6: 4 rows 150 Gcell/s, 8 rows 127
    if (cells < (int64_t(1) << 19)) return 4;
    if (cells < (int64_t(1) << 22)) return 16;
    const int64_t cap = (int64_t)sm_count() * std::max(1, blocks_per_sm) * warps_per_block;
    static const int cand[] = {32, 48, 64, 96, 128, 160, 192, 256};
    int best = 64;
    double best_cost = 1e300;
    for (int r : cand) {
        const int64_t warps = (int64_t)bands * ((nn + r - 1) / r);
        const int64_t waves = (warps + cap - 1) / cap;
        const double cost = (double)waves * (double)(std::min<int64_t>(r, nn) + 2 * K);
        if (cost < best_cost) { best_cost = cost; best = r; }
    }
    return best;
}

namespace {

template <typename T>
cudaError_t generic_t(int reaction, int boundary, const void *u, const void *v, void *un, void *vn,
                      int64_t nn, int64_t nm, const rdcnn_params &p, cudaStream_t s) {
    const int64_t n = nn * nm;
    const int64_t want = (n + 255) / 256;
    const unsigned grid = (unsigned)std::min<int64_t>(want, (int64_t)sm_count() * 16);
    const Coef<CT<T>> c = make_coef<CT<T>>(p, reaction);
    return with_model(reaction, boundary, [&](auto rx, auto bc) {
        const cudaError_t e = launch_k(k_generic<T, decltype(rx)::value, decltype(bc)::value>, grid, 256, 0, s,
                                       (const T *)u, (const T *)v, (T *)un, (T *)vn, (int)nn, (int)nm, c);
        count_launches(1);
        return e;
    });
}

}  // namespace

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
        return n;
    return 152;
}

cudaError_t launch_step1(int dtype, int reaction, int boundary, const void *u, const void *v,
                         void *un, void *vn, int64_t nn, int64_t nm, const rdcnn_params &p, int rows,
                         cudaStream_t s) {
    return with_dtype(dtype, [&](auto tag) {
        return step1_t<decltype(tag)>(reaction, boundary, u, v, un, vn, nn, nm, p, rows, s);
    });
}

cudaError_t launch_temporal(int dtype, int reaction, int boundary, int k, const void *u,
                            const void *v, void *un, void *vn, int64_t nn, int64_t nm,
                            const rdcnn_params &p, int rows, cudaStream_t s) {
    return with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        return with_depth(k, [&](auto kk) -> cudaError_t {
            constexpr int K = decltype(kk)::value;
            if constexpr (K <= MaxDepth<T>::value)
                return temporal_launch<T, K>(reaction, boundary, u, v, un, vn, nn, nm, p, rows, s);
            else
                return cudaErrorInvalidValue;
        });
    });
}

cudaError_t launch_temporal_wide(int dtype, int reaction, int boundary, int k, const void *u,
                                 const void *v, void *un, void *vn, int64_t nn, int64_t nm,
                                 const rdcnn_params &p, int rows, cudaStream_t s) {
    if (dtype == RDCNN_F64) return cudaErrorInvalidValue;
    return with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        return with_depth(k, [&](auto kk) -> cudaError_t {
            constexpr int K = decltype(kk)::value;
            if constexpr (K <= kMaxKWide && !std::is_same<T, double>::value)
                return temporal_launch<Wide<T>, K>(reaction, boundary, u, v, un, vn, nn, nm, p, rows, s);
            else
                return cudaErrorInvalidValue;
        });
    });
}

// FP32 / FP64 storage (the caller checks), every model.
cudaError_t launch_temporal_split(int dtype, int reaction, int boundary, int k, const void *u, const void *v,
                                  void *un, void *vn, int64_t nn, int64_t nm, const rdcnn_params &p,
                                  int rows, cudaStream_t s) {
    if (dtype != RDCNN_F32 && dtype != RDCNN_F64) return cudaErrorInvalidValue;
    return with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        return with_depth(k, [&](auto kk) -> cudaError_t {
            constexpr int K = decltype(kk)::value;
            if constexpr (K >= 2 && K <= MaxDepth<T>::value &&
                          is_f32_f64<T>())
                return split_tk<T, K>(reaction, boundary, u, v, un, vn, nn, nm, p, rows, s);
            else
                return cudaErrorInvalidValue;
        });
    });
}

cudaError_t launch_generic(int dtype, int reaction, int boundary, const void *u, const void *v,
                           void *un, void *vn, int64_t nn, int64_t nm, const rdcnn_params &p,
                           cudaStream_t s) {
    return with_dtype(dtype, [&](auto tag) {
        return generic_t<decltype(tag)>(reaction, boundary, u, v, un, vn, nn, nm, p, s);
    });
}

cudaError_t launch_init(int dtype, const void *x, void *u, void *v, double ka, int64_t n,
                        cudaStream_t s) {
    const int64_t want = (n + 255) / 256;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * 16));
    return with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        k_init<T><<<grid, 256, 0, s>>>((const T *)x, (T *)u, (T *)v, (CT<T>)ka, n);
        count_launches(1);
        return cudaGetLastError();
    });
}

int plan_rows(int dtype, int reaction, int boundary, int variant, int k, int64_t nn, int64_t nm,
              int rows) {
    if (variant == RDCNN_VARIANT_STEP1) return rows > 0 ? rows : default_rows_step1(dtype, nn, nm);
    if (variant == RDCNN_VARIANT_GENERIC) return 0;
    int out = 0;
    with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        return with_depth(k, [&](auto kk) -> cudaError_t {
            constexpr int K = decltype(kk)::value;
            if constexpr (K <= MaxDepth<T>::value) {
                if constexpr (K >= 2 && is_f32_f64<T>()) {
                    if (variant == RDCNN_VARIANT_TEMPORAL2) {
                        out = split_rows<T, K>(reaction, boundary, nn, nm, rows);
                        return cudaSuccess;
                    }
                }
                if constexpr (K <= kMaxKWide && !std::is_same<T, double>::value) {
                    if (variant == RDCNN_VARIANT_TEMPORAL_WIDE) {
                        out = temporal_rows<Wide<T>, K>(reaction, boundary, nn, nm, rows);
                        return cudaSuccess;
                    }
                }
                out = temporal_rows<T, K>(reaction, boundary, nn, nm, rows);
            }
            return cudaSuccess;
        });
    });
    return out;
}

// Temporal depth by grid size, from a launch-shape sweep on GB300 (FP32,
// square grids): 128^2-256^2 k=4, 512^2 k=6, 1024^2 k=4, >= 2048^2 k=8.
// Small grids are latency/launch bound, where fewer, shallower stages in
// more warps win; large grids are FP32-pipe bound, where depth amortises
// the halo.  FP64 is capped at its maximum depth.
int default_k(int dtype, int64_t nn, int64_t nm) {
    const int64_t cells = nn * nm;
    int k;
    if (cells >= (int64_t(1) << 21)) k = 8;
    else if (cells >= (int64_t(1) << 19)) k = 4;
    else if (cells >= (int64_t(1) << 17)) k = 6;
    else k = 4;
    return std::min(k, max_k(dtype));
}

// The single-step kernel is fastest with short strips (more warps in flight);
// the 16-bit single step (the ring pipeline at depth 1, 8 values per lane)
// with 32-row strips (measured at 4096^2, bf16: 4 / 8 / 16 / 32 / 64 rows =
// 507 / 570 / 627 / 672 / 574 Gcell/s).
int default_rows_step1(int dtype, int64_t nn, int64_t nm) {
    (void)nn; (void)nm;
    return is_16bit(dtype) ? 32 : dtype == RDCNN_F32 ? 2 : 4;
}

}  // namespace rdk
