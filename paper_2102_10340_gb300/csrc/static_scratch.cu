// static_scratch.cu -- rdcnn_run_static(): rdcnn_run without caller scratch
// and without any device allocation.
//
// Some callers cannot allocate device memory at all: a plug-in running inside
// a host application that owns the whole device memory pool (and forbids or
// cannot afford extra cudaMalloc calls at run time), or a C/Fortran driver
// that only ever receives device pointers from another component.  For them
// the two ping-pong planes the time loop needs live in a fixed, file-scope
// __device__ array instead of caller-provided workspace.
//
// Costs and rules:
//  - every GPU that loads this library reserves RDCNN_STATIC_SCRATCH_BYTES (16 MiB)
//    for the array until the process exits;
//  - one grid may use at most half of it per plane: NN*NM*sizeof(element)
//    <= 8 MiB, i.e. 2,097,152 FP32 cells or 1,048,576 FP64 cells; larger
//    grids are rejected with RDCNN_EINVAL before any GPU work.  The second
//    plane starts at the first one's size rounded up to 256 bytes, as in a
//    handle's workspace, so both planes keep the array's alignment;
//  - the update is the paper's: the toroidal boundary (there is no boundary
//    argument; zero-flux grids need rdcnn_run);
//  - all calls share the one array, so calls whose GPU work overlaps in time
//    (different streams, different host threads on the same device) race on
//    it and corrupt each other: serialise them;
//  - the array keeps the previous call's contents; this entry point never
//    reads scratch before writing it, so nothing needs clearing;
//  - the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress, which may load the module on that device); make
//    that first call before starting any stream capture on the device;
//  - that address is kept for the life of the process: do not use this
//    entry point after a cudaDeviceReset (or any teardown of the device's
//    primary context) in the same process, where it would be stale.
#include <cmath>
#include <mutex>

#include "internal.h"

namespace rdk {

namespace {

constexpr size_t kStaticScratchBytes = RDCNN_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (set up once per device).
int static_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(RDCNN_EINVAL, "device index %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
        if (!p) return set_error(RDCNN_ECUDA, "static scratch has no device address");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RDCNN_OK;
}

}  // namespace

}  // namespace rdk

using namespace rdk;

extern "C" {

int rdcnn_run_static(int64_t nn, int64_t nm, const rdcnn_params *p, int dtype, int reaction,
                     void *u, void *v, int64_t T, int k, void *stream) {
    if (nn < 1 || nm < 1 || nn > 0x7fffffff || nm > 0x7fffffff)
        return set_error(RDCNN_EINVAL, "grid size must be >= 1 (got %lld x %lld)", (long long)nn,
                         (long long)nm);
    if (dtype != RDCNN_F32 && dtype != RDCNN_F64) return set_error(RDCNN_EINVAL, "bad dtype");
    if (reaction != RDCNN_REACTION_FHN && reaction != RDCNN_REACTION_NONE)
        return set_error(RDCNN_EINVAL, "unknown reaction");
    const int pc = check_params(p);
    if (pc < 0) return pc;
    if (!u || !v) return set_error(RDCNN_EINVAL, "state pointers must be non-NULL");
    if (T < 0) return set_error(RDCNN_EINVAL, "T must be >= 0");
    const size_t plane = (size_t)nn * (size_t)nm * elem_size(dtype);
    if (plane > kStaticScratchBytes / 2 || plane_stride(plane) + plane > kStaticScratchBytes)
        return set_error(RDCNN_EINVAL,
                         "grid %lld x %lld needs %zu bytes of scratch; the static scratch holds %zu "
                         "(at most %zu cells of this dtype)",
                         (long long)nn, (long long)nm, 2 * plane, kStaticScratchBytes,
                         kStaticScratchBytes / 2 / elem_size(dtype));
    if (k == 0) k = default_k(dtype, nn, nm);
    if (k < 1 || k > max_k(dtype)) return set_error(RDCNN_EINVAL, "k must be in 1..%d", max_k(dtype));
    if (T == 0) return pc;

    void *scratch = nullptr;
    const int sc = static_scratch(&scratch);
    if (sc < 0) return sc;
    cudaStream_t s = (cudaStream_t)stream;
    void *su = scratch;
    void *sv = (char *)scratch + plane_stride(plane);
    const bool vec = (nm % vec_width(dtype) == 0) && aligned16(u) && aligned16(v) && aligned16(sv);
    const void *cu = u, *cv = v;
    void *nu = su, *nv = sv;
    for (int64_t left = T; left > 0;) {
        const int kk = vec ? (int)(left < k ? left : k) : 1;
        const cudaError_t e =
            vec ? launch_temporal(dtype, reaction, RDCNN_BC_PERIODIC, kk, cu, cv, nu, nv, nn, nm, *p, 0, s)
                : launch_generic(dtype, reaction, RDCNN_BC_PERIODIC, cu, cv, nu, nv, nn, nm, *p, s);
        if (e != cudaSuccess) return cuda_error(e, "static-scratch step launch");
        const void *tu = cu, *tv = cv;
        cu = nu; cv = nv;
        nu = const_cast<void *>(tu); nv = const_cast<void *>(tv);
        left -= kk;
    }
    if (cu != u) {
        cudaError_t e = cudaMemcpyAsync(u, cu, plane, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(v, cv, plane, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_error(e, "copy back from static scratch");
    }
    return pc;
}

}  // extern "C"
