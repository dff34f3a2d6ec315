// snapshots.cu -- rdcnn_run_snapshots(): T steps with the state captured every
// `every` steps, the A_show / B_show arrays of the paper's main loop
// (Sec. II.B: every test_mod iterations the GPU arrays are copied to the host
// into slot 1 + iter / test_mod; slot 0 holds the initial state).
//
// Launches are cut so that one ends exactly at every multiple of `every`;
// after it, the state planes are copied
//  - to device snapshots: straight into the caller's array, on the stream;
//  - to host snapshots: into a caller-provided device staging slot on the
//    compute stream, then to the host on a second stream (created once per
//    handle), so that the transfer overlaps the following steps.  A staging
//    slot is reused only after its previous host copy has finished (events).
#include <algorithm>
#include <vector>

#include "internal.h"

namespace rdk {

namespace {

struct SnapCtx {
    rdcnn_t *h = nullptr;
    int64_t every = 0;
    size_t plane = 0;
    char *u_snap = nullptr, *v_snap = nullptr;
    bool on_device = false;
    char *staging = nullptr;
    int n_stage = 0;
    std::vector<cudaEvent_t> ready, freed;
};

int take_snapshot(SnapCtx &c, int64_t s, const void *cu, const void *cv) {
    rdcnn_t *h = c.h;
    cudaError_t e;
    if (c.on_device) {
        e = cudaMemcpyAsync(c.u_snap + s * c.plane, cu, c.plane, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c.v_snap + s * c.plane, cv, c.plane, cudaMemcpyDeviceToDevice, h->stream);
        return e == cudaSuccess ? RDCNN_OK : cuda_error(e, "snapshot copy");
    }
    const int slot = (int)(s % c.n_stage);
    char *su = c.staging + (size_t)slot * 2 * c.plane;
    char *sv = su + c.plane;
    e = cudaSuccess;
    if (s >= c.n_stage) e = cudaStreamWaitEvent(h->stream, c.freed[slot], 0);  // slot's last host copy done
    if (e == cudaSuccess) e = cudaMemcpyAsync(su, cu, c.plane, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sv, cv, c.plane, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c.ready[slot], h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, c.ready[slot], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.u_snap + s * c.plane, su, c.plane, cudaMemcpyDeviceToHost, h->copy_stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c.v_snap + s * c.plane, sv, c.plane, cudaMemcpyDeviceToHost, h->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(c.freed[slot], h->copy_stream);
    return e == cudaSuccess ? RDCNN_OK : cuda_error(e, "snapshot transfer");
}

int on_mark(void *ctx, int64_t t, const void *cu, const void *cv) {
    SnapCtx &c = *static_cast<SnapCtx *>(ctx);
    return take_snapshot(c, t / c.every, cu, cv);
}

}  // namespace

}  // namespace rdk

using namespace rdk;

extern "C" {

int rdcnn_run_snapshots(rdcnn_t *h, int64_t T, int64_t every, void *u_snap, void *v_snap,
                        int snap_on_device, void *staging, size_t staging_bytes) {
    if (!h) return set_error(RDCNN_EINVAL, "handle is NULL");
    if (!h->bound) return set_error(RDCNN_ESTATE, "handle is not bound");
    if (T < 0 || every < 1) return set_error(RDCNN_EINVAL, "need T >= 0 and every >= 1");
    if (!u_snap || !v_snap) return set_error(RDCNN_EINVAL, "snapshot arrays must be non-NULL");
    SnapCtx c;
    c.h = h;
    c.every = every;
    c.plane = (size_t)h->nn * h->nm * elem_size(h->dtype);
    c.u_snap = (char *)u_snap;
    c.v_snap = (char *)v_snap;
    c.on_device = snap_on_device != 0;
    if (!c.on_device) {
        c.staging = (char *)staging;
        c.n_stage = staging ? (int)std::min<size_t>(staging_bytes / (2 * c.plane), 1 << 16) : 0;
        if (c.n_stage < 1)
            return set_error(RDCNN_ESPACE, "host snapshots need device staging of at least %zu bytes",
                             2 * c.plane);
        cudaError_t e = cudaSuccess;
        if (!h->copy_stream) e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_error(e, "create copy stream");
        c.ready.assign(c.n_stage, nullptr);
        c.freed.assign(c.n_stage, nullptr);
        for (int i = 0; i < c.n_stage && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&c.ready[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.freed[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            for (cudaEvent_t ev : c.ready) if (ev) cudaEventDestroy(ev);
            for (cudaEvent_t ev : c.freed) if (ev) cudaEventDestroy(ev);
            return cuda_error(e, "create snapshot events");
        }
    }
    int rc = take_snapshot(c, 0, h->u, h->v);  // slot 0: the state at the call
    if (rc >= 0) rc = run_core(h, T, RDCNN_VARIANT_AUTO, 0, every, on_mark, &c);
    if (!c.on_device) {
        // host snapshots have landed when the copy stream drains
        const cudaError_t e1 = cudaStreamSynchronize(h->copy_stream);
        const cudaError_t e2 = cudaStreamSynchronize(h->stream);
        for (cudaEvent_t ev : c.ready) cudaEventDestroy(ev);
        for (cudaEvent_t ev : c.freed) cudaEventDestroy(ev);
        if (rc >= 0 && e1 != cudaSuccess) rc = cuda_error(e1, "snapshot copies");
        if (rc >= 0 && e2 != cudaSuccess) rc = cuda_error(e2, "snapshot run");
    }
    return rc;
}

}  // extern "C"
