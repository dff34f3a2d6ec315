// adjoint.cu -- reverse-time (discrete adjoint) sweep of Eq. 1-3.
//
// Not in the paper: it differentiates the update of Sec. II.A exactly.  For
// one step (u+, v+) = F(u, v) and co-state (lu, lv) = dL/d(u+, v+):
//   dL/du = lu + dt [ (c - u^2) lu - eps lv + Du Lap(lu) ]
//   dL/dv = lv + dt [ -lu + eps b lv + Dv Lap(lv) ]
// (the 5-point Laplacian is symmetric, so it is its own transpose: on the
// torus, and under zero flux too, where a missing neighbour adds the cell
// itself, i.e. to the diagonal, and adjacency stays mutual),
// and the gene picks up, per step,
//   dL/dDu += dt sum lu Lap(u)     dL/dDv += dt sum lv Lap(v)
//   dL/dc  += dt sum lu u          dL/da  += dt sum lv (-eps)
//   dL/db  += dt sum lv eps v      dL/deps += dt sum lv (-(u - b v + a))
// with (u, v) the state before the step.  Because the Laplacian is symmetric,
// sum lu Lap(u) = sum u Lap(lu): the Du / Dv terms reuse the co-state
// neighbour sums the update forms anyway, and the state is needed only at
// the centre cell.  Under zero flux the co-state rows and columns beyond an
// edge are mirrored exactly like the state's (the mirrored grid evolves as
// the reflected image of the real one, forward and backward), so the
// pipeline's mirrored halos serve both.
//
// The Chua-Yang cell (u+ = u + dt [-u + c y(u) + Du sum_nbr y(u_n) + v],
// v+ = v) has
//   dL/du = lu + dt [ -lu + y'(u) (c lu + Du sum_nbr lu) ],  dL/dv = lv + dt lu
// with y' = 1 on (-1, 1) and 0 elsewhere (the corners included), and per step
//   dL/dDu += dt sum lu sum_nbr y(u_n) = dt sum y(u) sum_nbr lu
//   dL/dc  += dt sum lu y(u)
// (again by the symmetry of the neighbour relation), so it too reads the
// state at the centre cell only.
//
// Driver: a forward sweep stores n_ck checkpoints (every S = ceil(T/n_ck)
// steps).  Segments are then processed last to first: k_forward_all rebuilds
// the segment's states K per launch (every stage of the temporal pipeline is
// stored), and k_adjoint_pipe walks them backwards K steps per launch with
// the same register pipeline running the co-state update.  With more than
// one segment the rebuilds run on a second stream into two alternating
// buffer sets, so the rebuild of segment s - 1 overlaps the reverse sweep of
// segment s (events order each rebuild after the reverse sweep that last read
// its set, and each reverse sweep after its rebuild).  Each warp owns the
// same cells at every launch and adds its sums to its own FP64 slot, so the
// gradient is deterministic.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "temporal.cuh"
#include "adjoint_kernels.cuh"

// the pipelines compile in adjoint_f32a.cu .. adjoint_f32e.cu and adjoint_f64.cu
RDK_EXTERN_ADJ(float, 1, 1) RDK_EXTERN_ADJ(float, 2, 1) RDK_EXTERN_ADJ(float, 3, 1) RDK_EXTERN_ADJ(float, 4, 1)
RDK_EXTERN_ADJ(float, 1, 2) RDK_EXTERN_ADJ(float, 2, 2) RDK_EXTERN_ADJ(float, 3, 2) RDK_EXTERN_ADJ(float, 4, 2)
RDK_EXTERN_ADJ(float, 5, 2) RDK_EXTERN_ADJ(float, 6, 2) RDK_EXTERN_ADJ(float, 7, 2) RDK_EXTERN_ADJ(float, 8, 2)
RDK_EXTERN_ADJ(double, 1, 1) RDK_EXTERN_ADJ(double, 2, 1)
RDK_EXTERN_ADJ(double, 1, 2) RDK_EXTERN_ADJ(double, 2, 2) RDK_EXTERN_ADJ(double, 3, 2) RDK_EXTERN_ADJ(double, 4, 2)

namespace rdk {

namespace {
// Sum per-warp partials (fixed order), scale by dt: out[q] = dt * sum_w partial[w][q].
__global__ void __launch_bounds__(256)
k_reduce_partials(const double *__restrict__ partial, int nwarps, double dt, double *__restrict__ out) {
    __shared__ double sh[256];
    for (int q = 0; q < 6; ++q) {
        double s = 0.0;
        for (int w = threadIdx.x; w < nwarps; w += 256) s += partial[(int64_t)w * 6 + q];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int h = 128; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = dt * sh[0];
        __syncthreads();
    }
}

// Depth of the recompute / reverse launches (handle tune k, else these), and
// the halo lanes of the call's warp map: one lane while k <= V, else two.
// Default FP32 depth: 4, and 5 when every state is stored (no rebuild runs
// beside the reverse sweep; 512^2, T = 2000, 3-row strips: k = 3 / 4 / 5 / 6
// gave 6.3 / 6.2 / 5.5 / 6.0 ms for the full-tape sweep, 7.8 / 7.8 / 7.8 / 9.5
// ms with sqrt(T) checkpoints).
constexpr int kMaxAdjK32 = 8, kMaxAdjK64 = 4;
inline int adj_depth(int dtype, int tune_k, bool full) {
    const int cap = dtype == RDCNN_F64 ? kMaxAdjK64 : kMaxAdjK32;
    if (tune_k > 0) return std::min(tune_k, cap);
    return dtype == RDCNN_F64 ? 2 : (full ? 5 : 4);
}
inline int adj_halo(int dtype, int k) { return k <= vec_width(dtype) ? 1 : 2; }

// One warp -> cells map for every recompute / reverse launch of a call.
PipeShape pipe_shape(int dtype, int64_t nn, int64_t nm, int H) {
    const int V = vec_width(dtype);
    const int outw = (32 - 2 * H) * V;
    PipeShape s;
    const int64_t cells = nn * nm;
    // strip length by size class (short strips fill more SMs, long ones waste less halo).
    // 512^2, T = 2000, FP32 (ms; own checkpoints / sqrt(T) tape / full tape, k = 4):
    // 1 row 15.6 / 13.0 / 11.9, 2 rows 10.8 / 8.2 / 7.2, 3 rows 10.4 / 7.8 / 6.2,
    // 4 rows 11.0 / 8.3 / 6.7, 6 rows 10.7 / 8.1 / 6.5, 8 rows 11.4 / 8.7 / 7.4
    s.rows = cells < (int64_t(1) << 17) ? 4 : cells < (int64_t(1) << 19) ? 3 : cells < (int64_t(1) << 22) ? 16 : 64;
    s.bands = (int)((nm + outw - 1) / outw);
    s.strips = (int)((nn + s.rows - 1) / s.rows);
    s.nwarps = s.bands * s.strips;
    return s;
}

// Depth and halo dispatch: F32 k = 1..4 (H = 1) or 1..8 (H = 2), F64 1..2 / 1..4.
template <typename T>
cudaError_t reverse_launch(int reaction, int boundary, int k, int H, const void *lu, const void *lv, void *lun,
                           void *lvn, const StagePlanes<T> &st, double *partial, int64_t nn, int64_t nm,
                           const PipeShape &sh, const rdcnn_params &p, cudaStream_t s) {
    return with_depth(k, [&](auto kk) -> cudaError_t {
        constexpr int K = decltype(kk)::value;
        constexpr int V = Vec<T>::N;
        if (H == 1) {
            if constexpr (K <= V) return reverse_launch_kh<T, K, 1>(reaction, boundary, lu, lv, lun, lvn, st, partial, nn, nm, sh, p, s);
        } else {
            if constexpr (K <= 2 * V) return reverse_launch_kh<T, K, 2>(reaction, boundary, lu, lv, lun, lvn, st, partial, nn, nm, sh, p, s);
        }
        return cudaErrorInvalidValue;
    });
}

template <typename T>
cudaError_t forward_all_launch(int reaction, int boundary, int k, int H, const void *u, const void *v,
                               const StagePlanes<T> &pl, int64_t nn, int64_t nm, const PipeShape &sh,
                               const rdcnn_params &p, cudaStream_t s) {
    return with_depth(k, [&](auto kk) -> cudaError_t {
        constexpr int K = decltype(kk)::value;
        constexpr int V = Vec<T>::N;
        if (H == 1) {
            if constexpr (K <= V) return forward_all_launch_kh<T, K, 1>(reaction, boundary, u, v, pl, nn, nm, sh, p, s);
        } else {
            if constexpr (K <= 2 * V) return forward_all_launch_kh<T, K, 2>(reaction, boundary, u, v, pl, nn, nm, sh, p, s);
        }
        return cudaErrorInvalidValue;
    });
}

// Workspace (and tape) layout of one adjoint call.  Checkpoint slot i holds
// the state at step i*S.  With S = 1 (n_checkpoints >= T) every state is a
// checkpoint -- a full tape -- and nothing is rebuilt: the reverse sweep reads
// the slots directly.  own_ck: the checkpoints live in the workspace
// (rdcnn_adjoint) rather than in a caller's tape (rdcnn_adjoint_tape).
struct AdjLayout {
    int64_t S, nseg, nslots, nsets;  // nsets: segment buffer sets (2 when segments can overlap)
    bool full;
    int ka, H;  // depth of the recompute / reverse launches, halo lanes of the warp map
    size_t plane, ck_off, seg_off, lam_off, part_off, out_off, total, tape;
};

AdjLayout adj_layout(int dtype, int64_t nn, int64_t nm, int64_t T, int64_t nck, int tune_k, bool own_ck) {
    AdjLayout L{};
    if (nck <= 0) nck = (int64_t)std::ceil(std::sqrt((double)std::max<int64_t>(T, 1)));
    nck = std::max<int64_t>(1, std::min<int64_t>(nck, std::max<int64_t>(T, 1)));
    L.S = (std::max<int64_t>(T, 1) + nck - 1) / nck;
    L.nseg = (std::max<int64_t>(T, 1) + L.S - 1) / L.S;
    L.full = (L.S == 1 && T > 1);
    L.ka = adj_depth(dtype, tune_k, L.full);
    L.H = adj_halo(dtype, L.ka);
    L.nslots = L.full ? 0 : std::max<int64_t>(L.S, 2);
    L.nsets = L.full ? 0 : (L.nseg > 1 ? 2 : 1);
    L.plane = (((size_t)nn * nm * elem_size(dtype)) + 255) & ~(size_t)255;
    const PipeShape sh = pipe_shape(dtype, nn, nm, L.H);
    L.tape = (size_t)L.nseg * 2 * L.plane;
    L.ck_off = 0;
    L.seg_off = own_ck ? L.tape : 0;
    L.lam_off = L.seg_off + (size_t)L.nsets * L.nslots * 2 * L.plane;
    L.part_off = L.lam_off + 4 * L.plane;
    L.out_off = L.part_off + (((size_t)sh.nwarps * 6 * sizeof(double) + 255) & ~(size_t)255);
    L.total = L.out_off + 256;
    return L;
}

// The second stream and events of the overlapped driver (created once per
// handle); false if they cannot be had, and the driver then runs on one stream.
bool adj_streams(rdcnn_t *h) {
    if (!h->adj_stream && cudaStreamCreateWithFlags(&h->adj_stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        h->adj_stream = nullptr;
        return false;
    }
    for (cudaEvent_t &ev : h->adj_ev) {
        if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            ev = nullptr;
            return false;
        }
    }
    return true;
}

// Forward from the state in `ck` slot 0 (already written): fill checkpoint
// slots 1 .. nseg-1 (the state every S steps), with (tu, tv) as scratch
// planes; with lu_ non-NULL, continue through step T into (lu_, lv_).  The
// launches of a stretch alternate between the scratch pair and the stretch's
// destination and end in the destination, so no launch reads the planes it
// writes.
// Launch shapes: the temporal kernel at the size's default depth between
// checkpoints; for a full tape (S = 1) the store-all pipeline, which writes
// ka consecutive states per launch.  Every variant computes the same bits,
// so the states are those rdcnn_run produces.
template <typename T>
int record_states(int dtype, int reaction, int boundary, int64_t nn, int64_t nm, const rdcnn_params &p,
                  cudaStream_t s, int64_t nsteps, const AdjLayout &L, char *ck, void *tu, void *tv, void *lu_,
                  void *lv_) {
    auto ck_u = [&](int64_t i) { return (T *)(ck + (size_t)(2 * i) * L.plane); };
    auto ck_v = [&](int64_t i) { return (T *)(ck + (size_t)(2 * i + 1) * L.plane); };
    cudaError_t e = cudaSuccess;
    if (L.full) {
        const PipeShape sh = pipe_shape(dtype, nn, nm, L.H);
        for (int64_t q = 0; q + 1 < L.nseg;) {
            const int kk = (int)std::min<int64_t>(L.ka, L.nseg - 1 - q);
            StagePlanes<T> pl{};
            for (int j = 0; j < kk; ++j) { pl.u[j] = ck_u(q + 1 + j); pl.v[j] = ck_v(q + 1 + j); }
            e = forward_all_launch<T>(reaction, boundary, kk, L.H, ck_u(q), ck_v(q), pl, nn, nm, sh, p, s);
            if (e != cudaSuccess) return cuda_error(e, "tape recompute");
            q += kk;
        }
    }
    const int kf = default_k(dtype, nn, nm);
    auto advance = [&](const void *cu, const void *cv, int64_t len, void *ou, void *ov) -> cudaError_t {
        const int64_t nl = (len + kf - 1) / kf;
        for (int64_t j = 0; j < nl; ++j) {
            const int kk = (int)std::min<int64_t>(kf, len - j * kf);
            const bool to_dest = ((nl - 1 - j) % 2) == 0;
            void *nu = to_dest ? ou : tu;
            void *nv = to_dest ? ov : tv;
            const cudaError_t le = launch_temporal(dtype, reaction, boundary, kk, cu, cv, nu, nv, nn, nm, p, 0, s);
            if (le != cudaSuccess) return le;
            cu = nu; cv = nv;
        }
        return cudaSuccess;
    };
    if (!L.full) {
        for (int64_t i = 0; i + 1 < L.nseg && nsteps > 0; ++i) {
            e = advance(ck_u(i), ck_v(i), L.S, ck_u(i + 1), ck_v(i + 1));
            if (e != cudaSuccess) return cuda_error(e, "adjoint forward sweep");
        }
    }
    if (lu_) {
        const int64_t rest = nsteps - (L.nseg - 1) * L.S;
        if (rest > 0) e = advance(ck_u(L.nseg - 1), ck_v(L.nseg - 1), rest, lu_, lv_);
        if (e != cudaSuccess) return cuda_error(e, "forward to the final state");
    }
    return RDCNN_OK;
}

// The reverse sweep given the checkpoints in `ck` (slot i = state at step i*S).
template <typename T>
int reverse_sweep(rdcnn_t *h, int64_t nn, int64_t nm, const rdcnn_params &p, int dtype, int reaction, int boundary,
                  cudaStream_t s, int64_t nsteps, const void *dLdu_T, const void *dLdv_T, const AdjLayout &L,
                  const char *ck, char *ws, void *dLdu0, void *dLdv0, double grad[6]) {
    const size_t bytes = (size_t)nn * nm * sizeof(T);
    auto ck_u = [&](int64_t i) { return (T *)(ck + (size_t)(2 * i) * L.plane); };
    auto ck_v = [&](int64_t i) { return (T *)(ck + (size_t)(2 * i + 1) * L.plane); };
    int set = 0;  // buffer set of the segment being rebuilt / swept
    auto seg_u = [&](int64_t i) { return (T *)(ws + L.seg_off + (size_t)(2 * (set * L.nslots + i)) * L.plane); };
    auto seg_v = [&](int64_t i) { return (T *)(ws + L.seg_off + (size_t)(2 * (set * L.nslots + i) + 1) * L.plane); };
    const bool overlap = L.nsets == 2 && adj_streams(h);
    cudaStream_t rs = overlap ? h->adj_stream : s;  // the rebuild stream
    // an error after work went to the rebuild stream: let it drain before returning
    auto fail = [&](cudaError_t err, const char *what) {
        if (overlap) (void)cudaStreamSynchronize(rs);
        return cuda_error(err, what);
    };
    T *lam_u[2] = {(T *)(ws + L.lam_off), (T *)(ws + L.lam_off + 2 * L.plane)};
    T *lam_v[2] = {(T *)(ws + L.lam_off + L.plane), (T *)(ws + L.lam_off + 3 * L.plane)};
    double *partial = (double *)(ws + L.part_off);
    double *gout = (double *)(ws + L.out_off);
    const PipeShape sh = pipe_shape(dtype, nn, nm, L.H);
    const int ka = L.ka;  // depth of recompute / reverse launches

    cudaError_t e = cudaMemcpyAsync(lam_u[0], dLdu_T, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lam_v[0], dLdv_T, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(partial, 0, (size_t)sh.nwarps * 6 * sizeof(double), s);
    if (e != cudaSuccess) return cuda_error(e, "adjoint setup copies");
    if (overlap) {  // the rebuilds read the checkpoints
        e = cudaEventRecord(h->adj_ev[0], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(rs, h->adj_ev[0], 0);
        if (e != cudaSuccess) return fail(e, "adjoint stream order");
    }
    int cur = 0;
    auto sweep_back = [&](int64_t len, auto state_u, auto state_v) -> cudaError_t {
        for (int64_t qh = len; qh > 0;) {
            const int kk = (int)std::min<int64_t>(ka, qh);
            StagePlanes<T> st{};
            for (int j = 0; j < kk; ++j) { st.u[j] = state_u(qh - 1 - j); st.v[j] = state_v(qh - 1 - j); }
            const cudaError_t le = reverse_launch<T>(reaction, boundary, kk, L.H, lam_u[cur], lam_v[cur], lam_u[cur ^ 1],
                                                     lam_v[cur ^ 1], st, partial, nn, nm, sh, p, s);
            if (le != cudaSuccess) return le;
            cur ^= 1;
            qh -= kk;
        }
        return cudaSuccess;
    };
    if (L.full) {
        // every state is a checkpoint: one sweep over the whole horizon, nothing rebuilt
        if (nsteps > 0) e = sweep_back(nsteps, ck_u, ck_v);
        if (e != cudaSuccess) return fail(e, "adjoint reverse step");
    }
    // segments last to first: rebuild the states, then sweep the co-state back
    for (int64_t sg = L.nseg - 1; !L.full && sg >= 0 && nsteps > 0; --sg) {
        const int64_t len = std::min<int64_t>(L.S, nsteps - sg * L.S);
        set = overlap ? (int)((L.nseg - 1 - sg) & 1) : 0;
        auto state_u = [&](int64_t q) { return q == 0 ? ck_u(sg) : seg_u(q); };
        auto state_v = [&](int64_t q) { return q == 0 ? ck_v(sg) : seg_v(q); };
        if (overlap && sg + 2 <= L.nseg - 1) {  // the reverse sweep two segments back read this set
            e = cudaStreamWaitEvent(rs, h->adj_ev[3 + set], 0);
            if (e != cudaSuccess) return fail(e, "adjoint stream order");
        }
        for (int64_t q = 0; q + 1 < len;) {
            const int kk = (int)std::min<int64_t>(ka, len - 1 - q);
            StagePlanes<T> pl{};
            for (int j = 0; j < kk; ++j) { pl.u[j] = seg_u(q + 1 + j); pl.v[j] = seg_v(q + 1 + j); }
            e = forward_all_launch<T>(reaction, boundary, kk, L.H, state_u(q), state_v(q), pl, nn, nm, sh, p, rs);
            if (e != cudaSuccess) return fail(e, "adjoint recompute");
            q += kk;
        }
        if (overlap) {
            e = cudaEventRecord(h->adj_ev[1 + set], rs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->adj_ev[1 + set], 0);
            if (e != cudaSuccess) return fail(e, "adjoint stream order");
        }
        e = sweep_back(len, state_u, state_v);
        if (e != cudaSuccess) return fail(e, "adjoint reverse step");
        if (overlap) {
            e = cudaEventRecord(h->adj_ev[3 + set], s);
            if (e != cudaSuccess) return fail(e, "adjoint stream order");
        }
    }
    k_reduce_partials<<<1, 256, 0, s>>>(partial, sh.nwarps, p.dt, gout);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "gradient reduction");
    e = cudaMemcpyAsync(dLdu0, lam_u[cur], bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dLdv0, lam_v[cur], bytes, cudaMemcpyDeviceToDevice, s);
    double hg[6];
    if (e == cudaSuccess) e = cudaMemcpyAsync(hg, gout, sizeof(hg), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "adjoint results");
    for (int q = 0; q < 6; ++q) grad[q] = hg[q];
    return RDCNN_OK;
}

// rdcnn_adjoint: checkpoints recorded into the workspace, then the reverse sweep.
template <typename T>
int adjoint_t(rdcnn_t *h, int64_t nn, int64_t nm, const rdcnn_params &p, int dtype, int reaction, int boundary,
              cudaStream_t s, int64_t nsteps, const void *u0, const void *v0, const void *dLdu_T,
              const void *dLdv_T, const AdjLayout &L, char *ws, void *dLdu0, void *dLdv0, double grad[6]) {
    const size_t bytes = (size_t)nn * nm * sizeof(T);
    char *ck = ws + L.ck_off;
    cudaError_t e = cudaMemcpyAsync(ck, u0, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ck + L.plane, v0, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "adjoint setup copies");
    // a co-state plane pair serves as the sweep's scratch until the reverse sweep starts
    char *lam = ws + L.lam_off;
    const int rc = record_states<T>(dtype, reaction, boundary, nn, nm, p, s, nsteps, L, ck, lam, lam + L.plane,
                                    nullptr, nullptr);
    if (rc < 0) return rc;
    return reverse_sweep<T>(h, nn, nm, p, dtype, reaction, boundary, s, nsteps, dLdu_T, dLdv_T, L, ck, ws, dLdu0,
                            dLdv0, grad);
}

// Shared checks of the adjoint entry points.
int adjoint_checks(int64_t T, int dtype, int64_t nm) {
    if (is_16bit(dtype)) return set_error(RDCNN_EINVAL, "the adjoint supports FP32 / FP64 handles only");
    if (T < 0) return set_error(RDCNN_EINVAL, "T must be >= 0");
    const int V = vec_width(dtype);
    if (nm % V != 0) return set_error(RDCNN_EINVAL, "adjoint needs NM %% %d == 0", V);
    return RDCNN_OK;
}

}  // namespace

}  // namespace rdk

using namespace rdk;

extern "C" {

int rdcnn_adjoint_workspace_bytes(const rdcnn_t *h, int64_t T, int64_t n_checkpoints,
                                  size_t *bytes) {
    int64_t nn, nm; rdcnn_params p; int dtype, reaction; cudaStream_t s;
    if (!bytes) return set_error(RDCNN_EINVAL, "bytes is NULL");
    const int rc = handle_view(h, &nn, &nm, &p, &dtype, &reaction, &s);
    if (rc < 0) return rc;
    if (T < 0) return set_error(RDCNN_EINVAL, "T must be >= 0");
    if (is_16bit(dtype)) return set_error(RDCNN_EINVAL, "the adjoint supports FP32 / FP64 handles only");
    *bytes = adj_layout(dtype, nn, nm, T, n_checkpoints, h->tune_k, true).total;
    return RDCNN_OK;
}

int rdcnn_adjoint(rdcnn_t *h, int64_t T, const void *u0, const void *v0, const void *dLdu_T,
                  const void *dLdv_T, int64_t n_checkpoints, void *dLdu0, void *dLdv0,
                  double grad[6], void *workspace, size_t workspace_bytes) {
    int64_t nn, nm; rdcnn_params p; int dtype, reaction, boundary; cudaStream_t s;
    int rc = handle_view(h, &nn, &nm, &p, &dtype, &reaction, &s, &boundary);
    if (rc < 0) return rc;
    rc = adjoint_checks(T, dtype, nm);
    if (rc < 0) return rc;
    if (!u0 || !v0 || !dLdu_T || !dLdv_T || !dLdu0 || !dLdv0 || !grad || !workspace)
        return set_error(RDCNN_EINVAL, "NULL argument");
    const void *ptrs[7] = {u0, v0, dLdu_T, dLdv_T, dLdu0, dLdv0, workspace};
    for (const void *q : ptrs)
        if (!aligned16(q)) return set_error(RDCNN_EINVAL, "adjoint buffers must be 16-byte aligned");
    const AdjLayout L = adj_layout(dtype, nn, nm, T, n_checkpoints, h->tune_k, true);
    if (workspace_bytes < L.total)
        return set_error(RDCNN_ESPACE, "adjoint workspace has %zu bytes, need %zu", workspace_bytes, L.total);
    if (dtype == RDCNN_F64)
        return adjoint_t<double>(h, nn, nm, p, dtype, reaction, boundary, s, T, u0, v0, dLdu_T, dLdv_T, L,
                                 (char *)workspace, dLdu0, dLdv0, grad);
    return adjoint_t<float>(h, nn, nm, p, dtype, reaction, boundary, s, T, u0, v0, dLdu_T, dLdv_T, L,
                            (char *)workspace, dLdu0, dLdv0, grad);
}

int rdcnn_tape_bytes(const rdcnn_t *h, int64_t T, int64_t n_checkpoints, size_t *tape_bytes,
                     size_t *workspace_bytes) {
    int64_t nn, nm; rdcnn_params p; int dtype, reaction; cudaStream_t s;
    if (!tape_bytes || !workspace_bytes) return set_error(RDCNN_EINVAL, "NULL output");
    const int rc = handle_view(h, &nn, &nm, &p, &dtype, &reaction, &s);
    if (rc < 0) return rc;
    if (T < 0) return set_error(RDCNN_EINVAL, "T must be >= 0");
    if (is_16bit(dtype)) return set_error(RDCNN_EINVAL, "the adjoint supports FP32 / FP64 handles only");
    const AdjLayout L = adj_layout(dtype, nn, nm, T, n_checkpoints, h->tune_k, false);
    *tape_bytes = L.tape;
    *workspace_bytes = L.total;
    return RDCNN_OK;
}

int rdcnn_run_record(rdcnn_t *h, int64_t T, int64_t n_checkpoints, void *tape, size_t tape_bytes) {
    int64_t nn, nm; rdcnn_params p; int dtype, reaction, boundary; cudaStream_t s;
    int rc = handle_view(h, &nn, &nm, &p, &dtype, &reaction, &s, &boundary);
    if (rc < 0) return rc;
    if (!h->bound) return set_error(RDCNN_ESTATE, "handle is not bound");
    rc = adjoint_checks(T, dtype, nm);
    if (rc < 0) return rc;
    if (!tape) return set_error(RDCNN_EINVAL, "tape is NULL");
    if (!aligned16(tape) || !aligned16(h->u) || !aligned16(h->v) || !aligned16(h->ws))
        return set_error(RDCNN_EINVAL, "the tape and the bound buffers must be 16-byte aligned");
    const AdjLayout L = adj_layout(dtype, nn, nm, T, n_checkpoints, h->tune_k, false);
    if (tape_bytes < L.tape) return set_error(RDCNN_ESPACE, "tape has %zu bytes, need %zu", tape_bytes, L.tape);
    const size_t bytes = (size_t)nn * nm * elem_size(dtype);
    char *ck = (char *)tape;
    cudaError_t e = cudaMemcpyAsync(ck, h->u, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ck + L.plane, h->v, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "tape slot 0");
    if (T == 0) return RDCNN_OK;
    // scratch: the bound ping-pong planes (second one at the rounded stride)
    char *ws = (char *)h->ws;
    void *su = ws, *sv = ws + plane_stride(bytes);
    if (dtype == RDCNN_F64)
        return record_states<double>(dtype, reaction, boundary, nn, nm, p, s, T, L, ck, su, sv, h->u, h->v);
    return record_states<float>(dtype, reaction, boundary, nn, nm, p, s, T, L, ck, su, sv, h->u, h->v);
}

int rdcnn_adjoint_tape(rdcnn_t *h, int64_t T, int64_t n_checkpoints, const void *tape, size_t tape_bytes,
                       const void *dLdu_T, const void *dLdv_T, void *dLdu0, void *dLdv0, double grad[6],
                       void *workspace, size_t workspace_bytes) {
    int64_t nn, nm; rdcnn_params p; int dtype, reaction, boundary; cudaStream_t s;
    int rc = handle_view(h, &nn, &nm, &p, &dtype, &reaction, &s, &boundary);
    if (rc < 0) return rc;
    rc = adjoint_checks(T, dtype, nm);
    if (rc < 0) return rc;
    if (!tape || !dLdu_T || !dLdv_T || !dLdu0 || !dLdv0 || !grad || !workspace)
        return set_error(RDCNN_EINVAL, "NULL argument");
    const void *ptrs[6] = {tape, dLdu_T, dLdv_T, dLdu0, dLdv0, workspace};
    for (const void *q : ptrs)
        if (!aligned16(q)) return set_error(RDCNN_EINVAL, "adjoint buffers must be 16-byte aligned");
    const AdjLayout L = adj_layout(dtype, nn, nm, T, n_checkpoints, h->tune_k, false);
    if (tape_bytes < L.tape) return set_error(RDCNN_ESPACE, "tape has %zu bytes, need %zu", tape_bytes, L.tape);
    if (workspace_bytes < L.total)
        return set_error(RDCNN_ESPACE, "adjoint workspace has %zu bytes, need %zu", workspace_bytes, L.total);
    if (dtype == RDCNN_F64)
        return reverse_sweep<double>(h, nn, nm, p, dtype, reaction, boundary, s, T, dLdu_T, dLdv_T, L,
                                     (const char *)tape, (char *)workspace, dLdu0, dLdv0, grad);
    return reverse_sweep<float>(h, nn, nm, p, dtype, reaction, boundary, s, T, dLdu_T, dLdv_T, L, (const char *)tape,
                                (char *)workspace, dLdu0, dLdv0, grad);
}

}  // extern "C"
