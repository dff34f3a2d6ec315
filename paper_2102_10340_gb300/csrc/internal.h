// internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "rdcnn.h"

// The simulation handle behind rdcnn_t (include/rdcnn.h).
struct rdcnn {
    int64_t nn = 0, nm = 0;
    rdcnn_params p{};
    int dtype = RDCNN_F32;
    int reaction = RDCNN_REACTION_FHN;
    int boundary = RDCNN_BC_PERIODIC;
    void *u = nullptr, *v = nullptr, *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    bool bound = false;
    int tune_k = 0, tune_rows = 0;
    cudaStream_t copy_stream = nullptr;  // created on first use by rdcnn_run_snapshots
    // rdcnn_adjoint's second stream (segment rebuilds overlap the reverse
    // sweep) and its events: [0] checkpoints ready, [1..2] rebuild of buffer
    // set 0 / 1 done, [3..4] reverse over set 0 / 1 done.  Created on first use.
    cudaStream_t adj_stream = nullptr;
    cudaEvent_t adj_ev[5] = {};
    // Graph replay of runs of small grids (run_core): a captured sequence of
    // full-depth launches and what it was captured for.
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    struct GraphKey {
        const void *u, *v, *su, *sv;
        int variant, k, rows, dtype, reaction, boundary;
        rdcnn_params p;
    } graph_key{};
};

namespace rdk {

// Launch-shape limits of the vectorised kernels.
constexpr int kMaxK32 = 8;  // temporal depth, FP32
constexpr int kMaxK64 = 4;  // temporal depth, FP64
constexpr int kMaxKWide = 4;  // temporal depth with 8 values per lane

inline int vec_width(int dtype) { return dtype == RDCNN_F64 ? 2 : 4; }
inline size_t elem_size(int dtype) {
    return dtype == RDCNN_F64 ? 8 : (dtype == RDCNN_BF16 || dtype == RDCNN_F16) ? 2 : 4;
}
inline bool is_16bit(int dtype) { return dtype == RDCNN_BF16 || dtype == RDCNN_F16; }
// Alignment the vectorised kernels need: one lane vector of the temporal
// pipeline (16 bytes; 8 bytes = 4 values for 16-bit planes).
inline size_t vec_align(int dtype) { return is_16bit(dtype) ? 8 : 16; }
// Byte offset of the second ping-pong plane in a handle's workspace: the
// plane size rounded up to 256 bytes, so that both planes share the
// workspace's alignment whatever the grid size.
inline size_t plane_stride(size_t plane_bytes) { return (plane_bytes + 255) & ~(size_t)255; }
inline int max_k(int dtype) { return dtype == RDCNN_F64 ? kMaxK64 : kMaxK32; }

// Columns of output a warp of the temporal kernel produces for depth k.
inline int temporal_out_cols(int dtype, int k) {
    const int V = vec_width(dtype);
    const int H = (k + V - 1) / V;
    return (32 - 2 * H) * V;
}

void count_launches(uint64_t n);
void uncount_launches(uint64_t n);  // launches recorded into a graph, not run

// Error reporting (thread-local message, returned code passes through).
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
// Validates a gene for a reaction: RDCNN_OK, RDCNN_WARN_CFL, or a negative
// code.  The CeNN cell takes feedback weights of either sign in Du and c and
// has no diffusion stability bound.
int check_params(const rdcnn_params *p, int reaction = RDCNN_REACTION_FHN);
bool aligned16(const void *p);
inline bool aligned_to(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }
int sm_count();

// Programmatic dependent launch of the stepping kernels: on unless the
// environment sets RDCNN_PDL=0 (read once).
bool pdl_enabled();

// Launch kernel<<<grid, block, smem, s>>>(args...), with the
// programmatic-serialization attribute when pdl_enabled(): the kernel must
// call pdl_wait() (common.cuh) before its first global memory access.
// Returns the launch status.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Read-only view of a handle's configuration (defined in api.cu); the stream
// is the one bound by rdcnn_bind (NULL if unbound).
int handle_view(const rdcnn_t *h, int64_t *nn, int64_t *nm, rdcnn_params *p, int *dtype,
                int *reaction, cudaStream_t *stream, int *boundary = nullptr);

// Callback of run_core: called after the launch that completes step t (a
// multiple of `every`), with the planes that hold the state at that step.
typedef int (*MarkFn)(void *ctx, int64_t t, const void *cu, const void *cv);

// Advance the bound state of h by T steps (the body of rdcnn_run).  With
// every > 0 no launch crosses a multiple of `every`, and mark(ctx, t, ...)
// runs after each such step t.  Result in h->u, h->v.
int run_core(rdcnn_t *h, int64_t T, int variant, int k, int64_t every, MarkFn mark, void *ctx);

// Kernel launchers.  All return the launch status (cudaGetLastError()).
// u/v are read, un/vn written; the two pairs must not overlap.  reaction is
// an RDCNN_REACTION_*, boundary an RDCNN_BC_*.
cudaError_t launch_step1(int dtype, int reaction, int boundary, const void *u, const void *v,
                         void *un, void *vn, int64_t nn, int64_t nm, const rdcnn_params &p, int rows,
                         cudaStream_t s);
cudaError_t launch_temporal(int dtype, int reaction, int boundary, int k, const void *u,
                            const void *v, void *un, void *vn, int64_t nn, int64_t nm,
                            const rdcnn_params &p, int rows, cudaStream_t s);
// The temporal pipeline with 8 values per lane (k = 1..4; F32, BF16, F16;
// NM % 8 == 0 and 16-byte aligned planes, which the caller checks).
cudaError_t launch_temporal_wide(int dtype, int reaction, int boundary, int k, const void *u,
                                 const void *v, void *un, void *vn, int64_t nn, int64_t nm,
                                 const rdcnn_params &p, int rows, cudaStream_t s);
// The temporal pipeline with the K stages split across a warp pair (k >= 2;
// FP32 / FP64 planes, every model).
cudaError_t launch_temporal_split(int dtype, int reaction, int boundary, int k, const void *u, const void *v,
                                  void *un, void *vn, int64_t nn, int64_t nm, const rdcnn_params &p,
                                  int rows, cudaStream_t s);
cudaError_t launch_generic(int dtype, int reaction, int boundary, const void *u, const void *v,
                           void *un, void *vn, int64_t nn, int64_t nm, const rdcnn_params &p,
                           cudaStream_t s);
// One depth of the temporal kernel (temporal_launch.cuh; instantiated for
// float K = 1..8 and double K = 1..4 in the temporal_*.cu units).
template <typename T, int K>
cudaError_t temporal_launch(int reaction, int boundary, const void *u, const void *v, void *un,
                            void *vn, int64_t nn, int64_t nm, const rdcnn_params &p, int rows,
                            cudaStream_t s);
// Rows per warp strip a temporal launch of depth K uses for the requested
// rows (rows <= 0: the launcher's own choice).
template <typename T, int K>
int temporal_rows(int reaction, int boundary, int64_t nn, int64_t nm, int rows);
// The same for every launcher: rows per warp (or per warp pair) of a launch
// of `variant` (an RDCNN_VARIANT_*, already resolved from AUTO) at depth k.
int plan_rows(int dtype, int reaction, int boundary, int variant, int k, int64_t nn, int64_t nm,
              int rows);
// Rows per warp strip of a temporal launch (wave-quantisation model).
int auto_rows_temporal(int K, int64_t nn, int64_t nm, int bands, int blocks_per_sm,
                       int warps_per_block);
// u = v = ka * x; x may alias u.
cudaError_t launch_init(int dtype, const void *x, void *u, void *v, double ka, int64_t n,
                        cudaStream_t s);

// Default launch shapes.  launch_temporal picks its rows per warp strip
// itself when given rows <= 0.
int default_rows_step1(int dtype, int64_t nn, int64_t nm);
int default_k(int dtype, int64_t nn, int64_t nm);

}  // namespace rdk
