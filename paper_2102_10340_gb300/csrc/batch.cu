// batch.cu -- many independent RD-CNN instances (a parameter sweep in the
// sense of Sec. III.A-III.B) advanced by ONE launch per K time steps: the
// host side (kernels in batch_kernels.cuh, instantiated in batch_*.cu).
//
// The host lays the instances out as a table of descriptors in device memory
// with a running warp offset: instance i owns warps
// [warp_begin_i, warp_begin_i + bands_i * strips_i).  A warp finds its instance
// by binary search over warp_begin, then runs the same K-stage register
// pipeline as the single-grid temporal kernel (temporal.cuh) with that
// instance's gene.  All launches of one call use the same halo width H (the
// one the deepest launch needs), so one table serves launches of any depth.
// Launches alternate between the state planes and the scratch planes; the
// host arranges an even number of launches whenever T allows it, so the
// result lands in the state planes without a copy.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "temporal.cuh"
#include "batch_kernels.cuh"

// the kernels compile in batch_f32a.cu .. batch_f32c.cu, batch_f64.cu,
// batch_bf16a.cu .. batch_bf16c.cu and batch_f16a.cu .. batch_f16c.cu
#define RDK_EXTERN_BATCH_32(TT)                                                                  \
    RDK_EXTERN_BATCH(TT, 1, 1) RDK_EXTERN_BATCH(TT, 2, 1) RDK_EXTERN_BATCH(TT, 3, 1)            \
    RDK_EXTERN_BATCH(TT, 4, 1) RDK_EXTERN_BATCH(TT, 1, 2) RDK_EXTERN_BATCH(TT, 2, 2)            \
    RDK_EXTERN_BATCH(TT, 3, 2) RDK_EXTERN_BATCH(TT, 4, 2) RDK_EXTERN_BATCH(TT, 5, 2)            \
    RDK_EXTERN_BATCH(TT, 6, 2) RDK_EXTERN_BATCH(TT, 7, 2) RDK_EXTERN_BATCH(TT, 8, 2)
RDK_EXTERN_BATCH_32(float)
RDK_EXTERN_BATCH_32(__nv_bfloat16)
RDK_EXTERN_BATCH_32(__half)
RDK_EXTERN_BATCH(double, 1, 1) RDK_EXTERN_BATCH(double, 2, 1)
RDK_EXTERN_BATCH(double, 1, 2) RDK_EXTERN_BATCH(double, 2, 2) RDK_EXTERN_BATCH(double, 3, 2)
RDK_EXTERN_BATCH(double, 4, 2)

namespace rdk {

namespace {

// Depths 1 .. H*V for halo H.
template <typename T, int H>
cudaError_t batch_launch_h(int reaction, int boundary, int k, const BatchDesc *tab, int n, long long nwarps,
                           int flip, cudaStream_t s) {
    constexpr int V = Vec<T>::N;
    if (k < 1 || k > H * V) return cudaErrorInvalidValue;
    return with_depth(k, [&](auto kk) -> cudaError_t {
        constexpr int K = decltype(kk)::value;
        if constexpr (K <= H * V)
            return batch_launch_khr<T, K, H>(reaction, boundary, tab, n, nwarps, flip, s);
        else
            return cudaErrorInvalidValue;
    });
}

cudaError_t batch_launch(int dtype, int reaction, int boundary, int k, int H, const BatchDesc *tab, int n,
                         long long nwarps, int flip, cudaStream_t s) {
    return with_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        if (H == 1) return batch_launch_h<T, 1>(reaction, boundary, k, tab, n, nwarps, flip, s);
        return batch_launch_h<T, 2>(reaction, boundary, k, tab, n, nwarps, flip, s);
    });
}

int batch_default_rows(int64_t nn) { return nn >= 1024 ? 64 : 32; }

// Split T into launch depths (each <= k), with an even count when possible.
std::vector<int> plan_depths(int64_t T, int k) {
    std::vector<int> d;
    for (int64_t left = T; left > 0; left -= k) d.push_back((int)std::min<int64_t>(k, left));
    if (d.size() % 2 == 1) {
        for (size_t i = d.size(); i-- > 0;) {
            if (d[i] >= 2) {
                const int a = d[i] / 2, b = d[i] - d[i] / 2;
                d[i] = a;
                d.insert(d.begin() + (long)i + 1, b);
                break;
            }
        }
    }
    return d;
}

int validate_batch(const rdcnn_instance *inst, int n, int dtype, int reaction, int boundary, int *warn) {
    if (!inst || n < 1) return set_error(RDCNN_EINVAL, "need at least one instance");
    if (dtype != RDCNN_F32 && dtype != RDCNN_F64 && !is_16bit(dtype)) return set_error(RDCNN_EINVAL, "bad dtype");
    if (reaction != RDCNN_REACTION_FHN && reaction != RDCNN_REACTION_NONE && reaction != RDCNN_REACTION_CENN)
        return set_error(RDCNN_EINVAL, "bad reaction");
    if (boundary != RDCNN_BC_PERIODIC && boundary != RDCNN_BC_ZEROFLUX)
        return set_error(RDCNN_EINVAL, "bad boundary");
    const int V = vec_width(dtype);
    const size_t align = vec_align(dtype);
    *warn = RDCNN_OK;
    for (int i = 0; i < n; ++i) {
        const rdcnn_instance &x = inst[i];
        if (x.nn < 1 || x.nm < 1 || x.nn > 0x7fffffff || x.nm > 0x7fffffff)
            return set_error(RDCNN_EINVAL, "instance %d: bad grid size", i);
        if (x.nm % V != 0)
            return set_error(RDCNN_EINVAL, "instance %d: NM must be a multiple of %d", i, V);
        if (!x.u || !x.v || !x.su || !x.sv)
            return set_error(RDCNN_EINVAL, "instance %d: NULL plane", i);
        if (!aligned_to(x.u, align) || !aligned_to(x.v, align) || !aligned_to(x.su, align) ||
            !aligned_to(x.sv, align))
            return set_error(RDCNN_EINVAL, "instance %d: planes must be %zu-byte aligned", i, align);
        const int pc = check_params(&x.params, reaction);
        if (pc < 0) {
            char why[256];
            snprintf(why, sizeof(why), "%s", rdcnn_last_error());
            return set_error(pc, "instance %d: %s", i, why);
        }
        if (pc == RDCNN_WARN_CFL) *warn = RDCNN_WARN_CFL;
    }
    return RDCNN_OK;
}

int resolve_tune(const rdcnn_tune *tune, int dtype, int *k, int *rows) {
    *k = (tune && tune->k) ? tune->k : std::min(4, max_k(dtype));
    *rows = (tune && tune->rows) ? tune->rows : 0;
    if (*k < 1 || *k > max_k(dtype)) return set_error(RDCNN_EINVAL, "k must be in 1..%d", max_k(dtype));
    if (*rows < 0) return set_error(RDCNN_EINVAL, "rows must be >= 0");
    return RDCNN_OK;
}

size_t table_bytes(int n) { return ((size_t)n * sizeof(BatchDesc) + 255) & ~(size_t)255; }

}  // namespace

}  // namespace rdk

using namespace rdk;

extern "C" {

int rdcnn_batch_workspace_bytes(const rdcnn_instance *inst, int n, int dtype,
                                const rdcnn_tune *tune, size_t *bytes) {
    (void)inst; (void)dtype; (void)tune;
    if (!bytes || n < 1) return set_error(RDCNN_EINVAL, "bad argument");
    *bytes = table_bytes(n);
    return RDCNN_OK;
}

int rdcnn_batch_run(const rdcnn_instance *inst, int n, int64_t T, int dtype, int reaction,
                    const rdcnn_tune *tune, void *workspace, size_t workspace_bytes,
                    void *stream) {
    return rdcnn_batch_run_model(inst, n, T, dtype, reaction, RDCNN_BC_PERIODIC, tune, workspace,
                                 workspace_bytes, stream);
}

int rdcnn_batch_run_model(const rdcnn_instance *inst, int n, int64_t T, int dtype, int reaction, int boundary,
                          const rdcnn_tune *tune, void *workspace, size_t workspace_bytes, void *stream) {
    int warn = RDCNN_OK;
    int rc = validate_batch(inst, n, dtype, reaction, boundary, &warn);
    if (rc < 0) return rc;
    if (T < 0) return set_error(RDCNN_EINVAL, "T must be >= 0");
    int k = 0, rows_req = 0;
    rc = resolve_tune(tune, dtype, &k, &rows_req);
    if (rc < 0) return rc;
    if (!workspace || workspace_bytes < table_bytes(n))
        return set_error(RDCNN_ESPACE, "workspace too small (need %zu bytes)", table_bytes(n));
    if (!aligned16(workspace)) return set_error(RDCNN_EINVAL, "workspace must be 16-byte aligned");
    if (T == 0) return warn;
    cudaStream_t s = (cudaStream_t)stream;
    const int V = vec_width(dtype);
    const int H = (k + V - 1) / V;
    const int outw = (32 - 2 * H) * V;
    std::vector<BatchDesc> tab(n);
    long long warps = 0;
    for (int i = 0; i < n; ++i) {
        const rdcnn_instance &x = inst[i];
        BatchDesc &d = tab[i];
        d.u = x.u; d.v = x.v; d.su = x.su; d.sv = x.sv;
        d.nn = (int)x.nn; d.nm = (int)x.nm;
        d.bands = (int)((x.nm + outw - 1) / outw);
        d.rows = rows_req ? rows_req : batch_default_rows(x.nn);
        d.rows = std::max(d.rows, 1);
        const long long strips = (x.nn + d.rows - 1) / d.rows;
        d.warp_begin = warps;
        warps += (long long)d.bands * strips;
        const Coef<double> q = make_coef<double>(x.params, reaction);
        d.dt = q.dt; d.Du = q.Du; d.Dv = q.Dv; d.cm4 = q.cm4;
        d.mthird = q.mthird; d.meps = q.meps; d.ebm4 = q.ebm4; d.mepsa = q.mepsa;
    }
    cudaError_t e = cudaMemcpyAsync(workspace, tab.data(), n * sizeof(BatchDesc),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host table goes out of scope
    if (e != cudaSuccess) return cuda_error(e, "copy batch table");
    const std::vector<int> depths = plan_depths(T, k);
    int flip = 0;
    for (int kk : depths) {
        e = batch_launch(dtype, reaction, boundary, kk, H, (const BatchDesc *)workspace, n, warps, flip, s);
        if (e != cudaSuccess) return cuda_error(e, "batch kernel launch");
        flip ^= 1;
    }
    if (flip) {  // odd launch count (only when every depth is 1): result is in the scratch planes
        for (int i = 0; i < n; ++i) {
            const size_t bytes = (size_t)inst[i].nn * inst[i].nm * elem_size(dtype);
            e = cudaMemcpyAsync(inst[i].u, inst[i].su, bytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(inst[i].v, inst[i].sv, bytes, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_error(e, "batch copy-back");
        }
    }
    return warn;
}

}  // extern "C"
