// summary.cu -- per-instance statistics of a batch of states, computed on
// the device: the measurements a parameter-space search (Sec. III.A: slow
// growth, dynamic patterns or dull homogeneous states over the (Du, Dv)
// plane; Sec. III.B: the (a, b) plane) needs to rank instances without
// copying every grid to the host.
//
// For each instance i (NN x NM torus, planes u, v), out[i * 8 + f] is
//   f = 0 mean(u)        1 var(u)          2 min(u)       3 max(u)
//       4 mean(v)        5 var(v)
//       6 mean over cells of |u(i+1,j) - u(i,j)| + |u(i,j+1) - u(i,j)|
//       7 fraction of cells where that gradient sum exceeds `threshold`
// (population variance; differences wrap around the torus).
//
// Pass 1 (k_summary_partial): each block takes a fixed row range of one
// instance (a warp per row), sums in T (FP32 for FP32 and 16-bit planes,
// FP64 for FP64 planes) within each warp and combines the
// warps in FP64 into one partial record.  Pass 2 (k_summary_final): one block per
// instance sums its partial records in a fixed order.  The result does not
// depend on timing (no atomics).
#include <algorithm>
#include <cfloat>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace rdk {

namespace {

constexpr int kSumBlock = 256;
constexpr int kSumRowsPerBlock = 8;  // one row per warp
constexpr int kFields = 8;

struct SumDesc {
    const void *u, *v;
    int nn, nm;
    long long block_begin;  // first partial-record index of this instance
    int nblocks;
    int dtype;              // RDCNN_F32 / F64 / BF16 / F16: the planes' element type
};

// Element 0 of a plane of the given element type, as a double.
__device__ __forceinline__ double first_value(const void *p, int dtype) {
    switch (dtype) {
        case RDCNN_F64: return load1((const double *)p);
        case RDCNN_BF16: return (double)load1((const __nv_bfloat16 *)p);
        case RDCNN_F16: return (double)load1((const __half *)p);
        default: return (double)load1((const float *)p);
    }
}

// Partial record: sums of (u - u0), (u - u0)^2, (v - v0), (v - v0)^2, |grad u|,
// edge count, and min / max of u (u0, v0: the instance's first cell).
struct Partial {
    double su, suu, sv, svv, sg, se, mn, mx;
};

template <typename T>
__device__ __forceinline__ T warp_red_sum(T x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}
template <typename T>
__device__ __forceinline__ T warp_red_min(T x) {
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(kFull, x, o));
    return x;
}
template <typename T>
__device__ __forceinline__ T warp_red_max(T x) {
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(kFull, x, o));
    return x;
}

// Pass 1: block b covers kSumRowsPerBlock rows of one instance, one warp per
// row, lanes striding the columns (coalesced loads, no index division).  Each
// lane sums in T = CT<S> (S: the plane's storage type); warps reduce in T;
// the block combines its warps in FP64.
template <typename S>
__global__ void __launch_bounds__(kSumBlock)
k_summary_partial(const SumDesc *__restrict__ tab, int n, CT<S> threshold, Partial *__restrict__ part) {
    typedef CT<S> T;
    __shared__ double sh[kSumBlock / 32][kFields];
    const long long b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].block_begin <= b) lo = mid; else hi = mid - 1;
    }
    const SumDesc d = tab[lo];
    const S *u = (const S *)d.u;
    const S *v = (const S *)d.v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = (int)(b - d.block_begin) * kSumRowsPerBlock;
    // Sums of u - u[0] and v - v[0]: with the shift close to the mean, the
    // one-pass variance sum(x^2)/n - mean^2 does not cancel catastrophically.
    const T u0 = load1(u), v0 = load1(v);
    T su = 0, suu = 0, sv = 0, svv = 0, sg = 0, se = 0;
    T mn = T(3.0e38), mx = T(-3.0e38);
    for (int i = r0 + w; i < min(r0 + kSumRowsPerBlock, d.nn); i += kSumBlock / 32) {
        const int ip = (i + 1 == d.nn) ? 0 : i + 1;
        const S *ur = u + (int64_t)i * d.nm;
        const S *un = u + (int64_t)ip * d.nm;
        const S *vr = v + (int64_t)i * d.nm;
        for (int j = lane; j < d.nm; j += 32) {
            const int jp = (j + 1 == d.nm) ? 0 : j + 1;
            const T x = load1(ur + j);
            const T g = fabs(load1(un + j) - x) + fabs(load1(ur + jp) - x);
            const T xs = x - u0, ys = load1(vr + j) - v0;
            su += xs; suu += xs * xs; sv += ys; svv += ys * ys; sg += g;
            se += (g > threshold) ? T(1) : T(0);
            mn = min(mn, x); mx = max(mx, x);
        }
    }
    su = warp_red_sum(su); suu = warp_red_sum(suu); sv = warp_red_sum(sv); svv = warp_red_sum(svv);
    sg = warp_red_sum(sg); se = warp_red_sum(se); mn = warp_red_min(mn); mx = warp_red_max(mx);
    if (lane == 0) {
        sh[w][0] = su; sh[w][1] = suu; sh[w][2] = sv; sh[w][3] = svv;
        sh[w][4] = sg; sh[w][5] = se; sh[w][6] = mn; sh[w][7] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial p{0, 0, 0, 0, 0, 0, DBL_MAX, -DBL_MAX};
        for (int k = 0; k < kSumBlock / 32; ++k) {
            p.su += sh[k][0]; p.suu += sh[k][1]; p.sv += sh[k][2]; p.svv += sh[k][3];
            p.sg += sh[k][4]; p.se += sh[k][5];
            p.mn = fmin(p.mn, sh[k][6]); p.mx = fmax(p.mx, sh[k][7]);
        }
        part[b] = p;
    }
}

__global__ void __launch_bounds__(32)
k_summary_final(const SumDesc *__restrict__ tab, const Partial *__restrict__ part, double *__restrict__ out) {
    const SumDesc d = tab[blockIdx.x];
    if (threadIdx.x != 0) return;
    double su = 0, suu = 0, sv = 0, svv = 0, sg = 0, se = 0, mn = DBL_MAX, mx = -DBL_MAX;
    for (int k = 0; k < d.nblocks; ++k) {
        const Partial p = part[d.block_begin + k];
        su += p.su; suu += p.suu; sv += p.sv; svv += p.svv; sg += p.sg; se += p.se;
        mn = fmin(mn, p.mn); mx = fmax(mx, p.mx);
    }
    const double cnt = (double)d.nn * d.nm;
    const double mu = su / cnt, mv = sv / cnt;  // means of the shifted values
    double *o = out + (int64_t)blockIdx.x * kFields;
    o[0] = mu + first_value(d.u, d.dtype);
    o[4] = mv + first_value(d.v, d.dtype);
    o[1] = fmax(0.0, suu / cnt - mu * mu);
    o[2] = mn;
    o[3] = mx;
    o[5] = fmax(0.0, svv / cnt - mv * mv);
    o[6] = sg / cnt;
    o[7] = se / cnt;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

}  // namespace rdk

using namespace rdk;

extern "C" {

int rdcnn_summary_workspace_bytes(const rdcnn_instance *inst, int n, size_t *bytes) {
    if (!inst || n < 1 || !bytes) return set_error(RDCNN_EINVAL, "bad argument");
    long long blocks = 0;
    for (int i = 0; i < n; ++i) {
        if (inst[i].nn < 1 || inst[i].nm < 1) return set_error(RDCNN_EINVAL, "instance %d: bad grid size", i);
        blocks += (inst[i].nn + kSumRowsPerBlock - 1) / kSumRowsPerBlock;
    }
    *bytes = align256((size_t)n * sizeof(SumDesc)) + align256((size_t)blocks * sizeof(Partial)) +
             align256((size_t)n * kFields * sizeof(double));
    return RDCNN_OK;
}

int rdcnn_batch_summary(const rdcnn_instance *inst, int n, int dtype, double threshold, double *out,
                        void *workspace, size_t workspace_bytes, void *stream) {
    if (!inst || n < 1 || !out || !workspace) return set_error(RDCNN_EINVAL, "bad argument");
    if (dtype != RDCNN_F32 && dtype != RDCNN_F64 && !is_16bit(dtype)) return set_error(RDCNN_EINVAL, "bad dtype");
    size_t need = 0;
    const int rc = rdcnn_summary_workspace_bytes(inst, n, &need);
    if (rc < 0) return rc;
    if (workspace_bytes < need) return set_error(RDCNN_ESPACE, "summary workspace needs %zu bytes", need);
    std::vector<SumDesc> tab(n);
    long long blocks = 0;
    for (int i = 0; i < n; ++i) {
        if (!inst[i].u || !inst[i].v) return set_error(RDCNN_EINVAL, "instance %d: NULL plane", i);
        if (inst[i].nn > 0x7fffffff || inst[i].nm > 0x7fffffff)
            return set_error(RDCNN_EINVAL, "instance %d: grid too large", i);
        tab[i].u = inst[i].u; tab[i].v = inst[i].v;
        tab[i].nn = (int)inst[i].nn; tab[i].nm = (int)inst[i].nm;
        tab[i].nblocks = (int)((inst[i].nn + kSumRowsPerBlock - 1) / kSumRowsPerBlock);
        tab[i].block_begin = blocks;
        tab[i].dtype = dtype;
        blocks += tab[i].nblocks;
    }
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    SumDesc *dtab = (SumDesc *)ws;
    Partial *part = (Partial *)(ws + align256((size_t)n * sizeof(SumDesc)));
    double *dout = (double *)((char *)part + align256((size_t)blocks * sizeof(Partial)));
    cudaError_t e = cudaMemcpyAsync(dtab, tab.data(), n * sizeof(SumDesc), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "copy summary table");
    e = with_dtype(dtype, [&](auto tag) {
        using S = decltype(tag);
        k_summary_partial<S><<<(unsigned)blocks, kSumBlock, 0, s>>>(dtab, n, (CT<S>)threshold, part);
        return cudaGetLastError();
    });
    count_launches(1);
    if (e != cudaSuccess) return cuda_error(e, "summary kernel");
    k_summary_final<<<n, 32, 0, s>>>(dtab, part, dout);
    count_launches(1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, (size_t)n * kFields * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // `out` and the host table are read on return
    if (e != cudaSuccess) return cuda_error(e, "summary results");
    return RDCNN_OK;
}

}  // extern "C"
