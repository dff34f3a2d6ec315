// api.cu -- the C ABI of include/rdcnn.h for the single-grid calls:
// handle life cycle, state I/O and the T-step driver (Eq. 1, t = 1..T).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"
#include "rdcnn.h"

namespace rdk {

namespace {
thread_local char g_err[512] = "";
std::atomic<uint64_t> g_launches{0};
}  // namespace

void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char *what) {
    (void)cudaGetLastError();  // a failed call leaves its code pending; clear it for later launch checks
    return set_error(RDCNN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int check_params(const rdcnn_params *p, int reaction) {
    if (!p) return set_error(RDCNN_EINVAL, "params is NULL");
    const double vals[7] = {p->dt, p->a, p->b, p->eps, p->c, p->Du, p->Dv};
    for (double x : vals)
        if (!std::isfinite(x)) return set_error(RDCNN_ENONFINITE, "non-finite gene entry");
    if (reaction == RDCNN_REACTION_CENN) return RDCNN_OK;  // feedback weights: any sign
    if (p->Du < 0 || p->Dv < 0) return set_error(RDCNN_EINVAL, "diffusion coefficients must be >= 0");
    const double dmax = p->Du > p->Dv ? p->Du : p->Dv;
    if (p->dt * dmax > 0.25) {
        set_error(RDCNN_WARN_CFL, "dt*max(Du,Dv) = %g > 1/4: explicit scheme unstable", p->dt * dmax);
        return RDCNN_WARN_CFL;
    }
    return RDCNN_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool pdl_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("RDCNN_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

int handle_view(const rdcnn_t *h, int64_t *nn, int64_t *nm, rdcnn_params *p, int *dtype,
                int *reaction, cudaStream_t *stream, int *boundary) {
    if (!h) return set_error(RDCNN_EINVAL, "handle is NULL");
    *nn = h->nn; *nm = h->nm; *p = h->p; *dtype = h->dtype; *reaction = h->reaction;
    *stream = h->stream;
    if (boundary) *boundary = h->boundary;
    return RDCNN_OK;
}

}  // namespace rdk

using namespace rdk;

extern "C" {

const char *rdcnn_last_error(void) { return g_err; }

uint64_t rdcnn_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char *rdcnn_version(void) { return "rdcnn 0.1 (sm_103a)"; }

int rdcnn_create(rdcnn_t **out, int64_t nn, int64_t nm, const rdcnn_params *p, int boundary,
                 int dtype, int reaction) {
    g_err[0] = '\0';
    if (!out) return set_error(RDCNN_EINVAL, "out is NULL");
    *out = nullptr;
    if (nn < 1 || nm < 1) return set_error(RDCNN_EINVAL, "grid size must be >= 1 (got %lld x %lld)", (long long)nn, (long long)nm);
    // each side below 2^30 (the kernels reflect indices modulo 2 NN and 2 NM in
    // 32-bit arithmetic); plane offsets are 64-bit
    if (nn >= (int64_t(1) << 30) || nm >= (int64_t(1) << 30) || nn * nm > (int64_t(1) << 40))
        return set_error(RDCNN_EINVAL, "grid too large (each side < 2^30, at most 2^40 cells)");
    if (boundary != RDCNN_BC_PERIODIC && boundary != RDCNN_BC_ZEROFLUX)
        return set_error(RDCNN_EINVAL, "boundary must be RDCNN_BC_PERIODIC or RDCNN_BC_ZEROFLUX");
    if (dtype != RDCNN_F32 && dtype != RDCNN_F64 && dtype != RDCNN_BF16 && dtype != RDCNN_F16)
        return set_error(RDCNN_EINVAL, "dtype must be RDCNN_F32, RDCNN_F64, RDCNN_BF16 or RDCNN_F16");
    if (reaction != RDCNN_REACTION_FHN && reaction != RDCNN_REACTION_NONE && reaction != RDCNN_REACTION_CENN)
        return set_error(RDCNN_EINVAL, "unknown reaction");
    const int pc = check_params(p, reaction);
    if (pc < 0) return pc;
    rdcnn_t *h = new (std::nothrow) rdcnn_t();
    if (!h) return set_error(RDCNN_EINVAL, "out of host memory");
    h->nn = nn; h->nm = nm; h->p = *p; h->dtype = dtype; h->reaction = reaction; h->boundary = boundary;
    *out = h;
    return pc;
}

int rdcnn_set_params(rdcnn_t *h, const rdcnn_params *p) {
    if (!h) return set_error(RDCNN_EINVAL, "handle is NULL");
    const int pc = check_params(p, h->reaction);
    if (pc < 0) return pc;
    h->p = *p;
    return pc;
}

int rdcnn_set_tune(rdcnn_t *h, const rdcnn_tune *tune) {
    if (!h) return set_error(RDCNN_EINVAL, "handle is NULL");
    if (!tune) { h->tune_k = 0; h->tune_rows = 0; return RDCNN_OK; }
    if (tune->k < 0 || tune->k > max_k(h->dtype))
        return set_error(RDCNN_EINVAL, "k must be in 0..%d", max_k(h->dtype));
    if (tune->rows < 0 || tune->rows > (1 << 20)) return set_error(RDCNN_EINVAL, "rows out of range");
    h->tune_k = tune->k;
    h->tune_rows = tune->rows;
    return RDCNN_OK;
}

int rdcnn_workspace_bytes(const rdcnn_t *h, size_t *bytes) {
    if (!h || !bytes) return set_error(RDCNN_EINVAL, "NULL argument");
    const size_t plane = (size_t)h->nn * (size_t)h->nm * elem_size(h->dtype);
    *bytes = plane_stride(plane) + plane;
    return RDCNN_OK;
}

int rdcnn_bind(rdcnn_t *h, void *u, void *v, void *workspace, size_t workspace_bytes, void *stream) {
    if (!h) return set_error(RDCNN_EINVAL, "handle is NULL");
    if (!u || !v || !workspace) return set_error(RDCNN_EINVAL, "state and workspace pointers must be non-NULL");
    size_t need = 0;
    rdcnn_workspace_bytes(h, &need);
    if (workspace_bytes < need)
        return set_error(RDCNN_ESPACE, "workspace has %zu bytes, need %zu", workspace_bytes, need);
    h->u = u; h->v = v; h->ws = workspace; h->ws_bytes = workspace_bytes;
    h->stream = (cudaStream_t)stream;
    h->bound = true;
    return RDCNN_OK;
}

int rdcnn_init(rdcnn_t *h, const void *x, double ka, int x_on_device) {
    if (!h) return set_error(RDCNN_EINVAL, "handle is NULL");
    if (!h->bound) return set_error(RDCNN_ESTATE, "handle is not bound");
    if (!x) return set_error(RDCNN_EINVAL, "x is NULL");
    if (!std::isfinite(ka)) return set_error(RDCNN_ENONFINITE, "ka is not finite");
    const int64_t n = h->nn * h->nm;
    const size_t bytes = (size_t)n * elem_size(h->dtype);
    cudaError_t e;
    if (!x_on_device) {
        e = cudaMemcpyAsync(h->u, x, bytes, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_error(e, "copy x to device");
        e = launch_init(h->dtype, h->u, h->u, h->v, ka, n, h->stream);
        if (e != cudaSuccess) return cuda_error(e, "init kernel");
        e = cudaStreamSynchronize(h->stream);  // x (host) may be reused on return
        if (e != cudaSuccess) return cuda_error(e, "init synchronize");
    } else {
        e = launch_init(h->dtype, x, h->u, h->v, ka, n, h->stream);
        if (e != cudaSuccess) return cuda_error(e, "init kernel");
    }
    return RDCNN_OK;
}

int rdcnn_set_state(rdcnn_t *h, const void *u0, const void *v0, int on_device) {
    if (!h) return set_error(RDCNN_EINVAL, "handle is NULL");
    if (!h->bound) return set_error(RDCNN_ESTATE, "handle is not bound");
    if (!u0 || !v0) return set_error(RDCNN_EINVAL, "state pointer is NULL");
    const size_t bytes = (size_t)h->nn * h->nm * elem_size(h->dtype);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(h->u, u0, bytes, kind, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->v, v0, bytes, kind, h->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_error(e, "set_state copy");
    return RDCNN_OK;
}

}  // extern "C"

namespace rdk {

// Resolve AUTO and the default depth for a run of h; vec_ok says whether the
// vectorised variants may run (NM multiple of the vector width, aligned
// buffers).  Returns RDCNN_OK or RDCNN_EINVAL.
static int resolve_variant(const rdcnn_t *h, bool vec_ok, bool wide_ok, int *variant, int *k) {
    if (*variant < RDCNN_VARIANT_AUTO || *variant > RDCNN_VARIANT_TEMPORAL_WIDE)
        return set_error(RDCNN_EINVAL, "unknown variant %d", *variant);
    if (*variant == RDCNN_VARIANT_TEMPORAL_WIDE) {
        if (h->dtype == RDCNN_F64) return set_error(RDCNN_EINVAL, "RDCNN_VARIANT_TEMPORAL_WIDE has no FP64 form");
        if (!wide_ok)
            return set_error(RDCNN_EINVAL, "RDCNN_VARIANT_TEMPORAL_WIDE needs NM %% 8 == 0 and 16-byte aligned buffers");
        if (*k == 0) *k = h->tune_k ? std::min(h->tune_k, kMaxKWide) : kMaxKWide;
        if (*k < 1 || *k > kMaxKWide) return set_error(RDCNN_EINVAL, "k must be in 1..%d for the wide variant", kMaxKWide);
        return RDCNN_OK;
    }
    if (*variant == RDCNN_VARIANT_AUTO) *variant = vec_ok ? RDCNN_VARIANT_TEMPORAL : RDCNN_VARIANT_GENERIC;
    if ((*variant == RDCNN_VARIANT_STEP1 || *variant == RDCNN_VARIANT_TEMPORAL ||
         *variant == RDCNN_VARIANT_TEMPORAL2) && !vec_ok)
        return set_error(RDCNN_EINVAL,
                         "vectorised variants need NM %% %d == 0 and %d-byte aligned buffers",
                         vec_width(h->dtype), (int)vec_align(h->dtype));
    if (*variant == RDCNN_VARIANT_TEMPORAL2 && is_16bit(h->dtype))
        return set_error(RDCNN_EINVAL, "RDCNN_VARIANT_TEMPORAL2 supports FP32 / FP64 planes only");
    if (*variant == RDCNN_VARIANT_TEMPORAL || *variant == RDCNN_VARIANT_TEMPORAL2) {
        if (*k == 0) *k = h->tune_k ? h->tune_k : default_k(h->dtype, h->nn, h->nm);
        if (*k < 1 || *k > max_k(h->dtype))
            return set_error(RDCNN_EINVAL, "k must be in 1..%d", max_k(h->dtype));
    } else {
        *k = 1;
    }
    return RDCNN_OK;
}

// Whether the vectorised kernels may run on h's planes: NM a multiple of
// `width` values and every plane aligned to `align` bytes.
static bool planes_ok(const rdcnn_t *h, int width, size_t align) {
    const bool nm_ok = (h->nm % width == 0);
    if (!h->bound) return nm_ok;
    const size_t plane = (size_t)h->nn * h->nm * elem_size(h->dtype);
    const char *ws = (const char *)h->ws;
    return nm_ok && aligned_to(h->u, align) && aligned_to(h->v, align) && aligned_to(ws, align) &&
           aligned_to(ws + plane_stride(plane), align);
}
static bool vec_ok_for(const rdcnn_t *h) { return planes_ok(h, vec_width(h->dtype), vec_align(h->dtype)); }
static bool wide_ok_for(const rdcnn_t *h) { return planes_ok(h, 8, 16); }

// One launch of the resolved variant: kk steps from (cu, cv) into (nu, nv).
static cudaError_t launch_one(const rdcnn_t *h, int variant, int kk, const void *cu, const void *cv, void *nu,
                              void *nv, cudaStream_t s) {
    if (variant == RDCNN_VARIANT_TEMPORAL_WIDE)
        return launch_temporal_wide(h->dtype, h->reaction, h->boundary, kk, cu, cv, nu, nv, h->nn, h->nm, h->p,
                                    h->tune_rows, s);  // 0 = chosen by the launcher
    if (variant == RDCNN_VARIANT_TEMPORAL2 && kk >= 2)
        return launch_temporal_split(h->dtype, h->reaction, h->boundary, kk, cu, cv, nu, nv, h->nn, h->nm, h->p,
                                     h->tune_rows, s);
    if (variant == RDCNN_VARIANT_TEMPORAL || variant == RDCNN_VARIANT_TEMPORAL2)
        return launch_temporal(h->dtype, h->reaction, h->boundary, kk, cu, cv, nu, nv, h->nn, h->nm, h->p,
                               h->tune_rows, s);
    if (variant == RDCNN_VARIANT_STEP1)
        return launch_step1(h->dtype, h->reaction, h->boundary, cu, cv, nu, nv, h->nn, h->nm, h->p,
                            h->tune_rows ? h->tune_rows : default_rows_step1(h->dtype, h->nn, h->nm), s);
    return launch_generic(h->dtype, h->reaction, h->boundary, cu, cv, nu, nv, h->nn, h->nm, h->p, s);
}

// Graph replay for launch-bound runs: grids whose launches are short
// (cells x k <= 2^23) spend a large share of each launch in launch overhead.
// kGraphLaunches consecutive full-depth launches (an even count, so the state
// is back in the bound planes after them) are captured once per launch
// configuration on a private stream and replayed on the bound stream.  Same
// kernels with the same arguments: the same bits as the plain launches.
constexpr int kGraphLaunches = 32;

static bool same_key(const rdcnn::GraphKey &a, const rdcnn::GraphKey &b) {
    return a.u == b.u && a.v == b.v && a.su == b.su && a.sv == b.sv && a.variant == b.variant && a.k == b.k &&
           a.rows == b.rows && a.dtype == b.dtype && a.reaction == b.reaction && a.boundary == b.boundary &&
           std::memcmp(&a.p, &b.p, sizeof(rdcnn_params)) == 0;
}

static void drop_graph(rdcnn_t *h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
}

// Capture (or reuse) the graph of kGraphLaunches launches of depth k for h's
// current configuration.  Returns false when graphs cannot be used here; the
// caller then launches normally.
static bool ensure_graph(rdcnn_t *h, int variant, int k, void *su, void *sv) {
    const rdcnn::GraphKey key{h->u, h->v, su, sv, variant, k, h->tune_rows, h->dtype, h->reaction, h->boundary, h->p};
    if (h->graph && same_key(key, h->graph_key)) return true;
    drop_graph(h);
    if (!h->capture_stream && cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        h->capture_stream = nullptr;
        return false;
    }
    // launch-shape queries (occupancy) happen here, outside the capture
    (void)plan_rows(h->dtype, h->reaction, h->boundary, variant, k, h->nn, h->nm, h->tune_rows);
    if (cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    const void *cu = h->u, *cv = h->v;
    void *nu = su, *nv = sv;
    cudaError_t e = cudaSuccess;
    int issued = 0;
    for (int i = 0; i < kGraphLaunches && e == cudaSuccess; ++i, ++issued) {
        e = launch_one(h, variant, k, cu, cv, nu, nv, h->capture_stream);
        const void *tu = cu, *tv = cv;
        cu = nu; cv = nv;
        nu = const_cast<void *>(tu); nv = const_cast<void *>(tv);
    }
    uncount_launches((uint64_t)issued);  // recorded, not run (each launcher counted itself)
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->capture_stream, &g);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && ec == cudaSuccess && g) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || ec != cudaSuccess || !exec) {
        (void)cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        return false;
    }
    h->graph = exec;
    h->graph_key = key;
    return true;
}

int run_core(rdcnn_t *h, int64_t T, int variant, int k, int64_t every, MarkFn mark, void *ctx) {
    if (!h) return set_error(RDCNN_EINVAL, "handle is NULL");
    if (!h->bound) return set_error(RDCNN_ESTATE, "handle is not bound");
    if (T < 0) return set_error(RDCNN_EINVAL, "T must be >= 0");
    if (variant < RDCNN_VARIANT_AUTO || variant > RDCNN_VARIANT_TEMPORAL_WIDE)
        return set_error(RDCNN_EINVAL, "unknown variant %d", variant);
    if (T == 0) return RDCNN_OK;
    const size_t plane = (size_t)h->nn * h->nm * elem_size(h->dtype);
    char *ws = (char *)h->ws;
    void *su = ws, *sv = ws + plane_stride(plane);
    const int rv = resolve_variant(h, vec_ok_for(h), wide_ok_for(h), &variant, &k);
    if (rv < 0) return rv;
    const void *cu = h->u, *cv = h->v;
    void *nu = su, *nv = sv;
    int64_t left = T;
    // launch-bound runs: replay whole groups of full-depth launches as a graph
    const int64_t full = T / k;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (every == 0 && !mark && full >= 2 * kGraphLaunches && h->nn * h->nm * (int64_t)k <= (int64_t(1) << 23) &&
        cudaStreamIsCapturing(h->stream, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone &&
        ensure_graph(h, variant, k, su, sv)) {
        const int64_t reps = full / kGraphLaunches;
        for (int64_t r = 0; r < reps; ++r) {
            const cudaError_t e = cudaGraphLaunch(h->graph, h->stream);
            if (e != cudaSuccess) return cuda_error(e, "graph launch");
            count_launches(kGraphLaunches);
        }
        left -= reps * kGraphLaunches * (int64_t)k;  // the state is back in (u, v)
    }
    (void)cudaGetLastError();  // a refused capture query leaves nothing pending
    while (left > 0) {
        int kk = (int)(left < k ? left : k);
        const int64_t done = T - left;
        if (every > 0) kk = (int)std::min<int64_t>(kk, every - done % every);
        const cudaError_t e = launch_one(h, variant, kk, cu, cv, nu, nv, h->stream);
        if (e != cudaSuccess) return cuda_error(e, "step kernel launch");
        const void *tu = cu, *tv = cv;
        cu = nu; cv = nv;
        nu = const_cast<void *>(tu); nv = const_cast<void *>(tv);
        left -= kk;
        if (every > 0 && (T - left) % every == 0 && mark) {
            const int rc = mark(ctx, T - left, cu, cv);
            if (rc < 0) return rc;
        }
    }
    if (cu != h->u) {
        cudaError_t e = cudaMemcpyAsync(h->u, cu, plane, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->v, cv, plane, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return cuda_error(e, "copy back to state");
    }
    return RDCNN_OK;
}

}  // namespace rdk

extern "C" {

int rdcnn_run(rdcnn_t *h, int64_t T, int variant, int k) { return run_core(h, T, variant, k, 0, nullptr, nullptr); }

int rdcnn_plan(const rdcnn_t *h, int *variant, rdcnn_tune *out) {
    if (!h || !variant || !out) return set_error(RDCNN_EINVAL, "NULL argument");
    int v = *variant, k = out->k;
    const int rv = resolve_variant(h, vec_ok_for(h), wide_ok_for(h), &v, &k);
    if (rv < 0) return rv;
    const int rows = v == RDCNN_VARIANT_GENERIC ? 0 : h->tune_rows;
    out->rows = plan_rows(h->dtype, h->reaction, h->boundary, v, k, h->nn, h->nm, rows);
    out->k = k;
    *variant = v;
    return RDCNN_OK;
}

int rdcnn_get_state(rdcnn_t *h, void *u_out, void *v_out, int to_device) {
    if (!h) return set_error(RDCNN_EINVAL, "handle is NULL");
    if (!h->bound) return set_error(RDCNN_ESTATE, "handle is not bound");
    const size_t bytes = (size_t)h->nn * h->nm * elem_size(h->dtype);
    const cudaMemcpyKind kind = to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    if (u_out) e = cudaMemcpyAsync(u_out, h->u, bytes, kind, h->stream);
    if (e == cudaSuccess && v_out) e = cudaMemcpyAsync(v_out, h->v, bytes, kind, h->stream);
    if (e == cudaSuccess && !to_device) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_error(e, "get_state copy");
    return RDCNN_OK;
}

void rdcnn_destroy(rdcnn_t *h) {
    if (!h) return;
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->adj_stream) cudaStreamDestroy(h->adj_stream);
    for (cudaEvent_t ev : h->adj_ev)
        if (ev) cudaEventDestroy(ev);
    delete h;
}

}  // extern "C"
