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
// the same register pipeline running the co-state update.  Each warp owns
// the same cells at every launch and adds its sums to its own FP64 slot, so
// the gradient is deterministic.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "temporal.cuh"

namespace rdk {

namespace {

constexpr int kPipeBlock = 32 * kTemporalWarps;

// Coefficients of the reverse step, arranged like the forward cell update
// (the -4 centre weight folded in): cm4 = c - 4 Du, ebm4 = eps b - 4 Dv;
// with no reaction cm4 = -4 Du, ebm4 = -4 Dv and the rest is unused.
// a, eps (FP64) enter only the final scaling of the gradient sums.
template <typename T> struct AdjCoef {
    T dt, Du, Dv, cm4, meps, ebm4, mb;
    double a, eps;
};

template <typename T>
AdjCoef<T> make_adj_coef(const rdcnn_params &p, int reaction) {
    const bool fhn = (reaction == RDCNN_REACTION_FHN);
    AdjCoef<T> q;
    if (reaction == RDCNN_REACTION_CENN) {  // cm4 = c: the self-feedback weight
        q.dt = T(p.dt); q.Du = T(p.Du); q.Dv = T(0);
        q.cm4 = T(p.c);
        q.meps = q.ebm4 = q.mb = T(0);
        q.a = 0.0; q.eps = 0.0;
        return q;
    }
    q.dt = T(p.dt); q.Du = T(p.Du); q.Dv = T(p.Dv);
    q.cm4 = T((fhn ? p.c : 0.0) - 4.0 * p.Du);
    q.meps = T(fhn ? -p.eps : 0.0);
    q.ebm4 = T((fhn ? p.eps * p.b : 0.0) - 4.0 * p.Dv);
    q.mb = T(-p.b);
    q.a = p.a; q.eps = p.eps;
    return q;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = add_rn(x, __shfl_xor_sync(kFull, x, o));
    return x;
}

// Reverse policy for the K-stage pipeline.  The pipeline streams the
// co-state (Slice.u = lu, Slice.v = lv, time t_hi first); stage s produces
// the co-state at time t_hi - s - 1 from the one at t_hi - s, using the state
// at time t_hi - s - 1 (state.u[s], state.v[s]) at the centre cell.  State
// rows travel through a per-warp shared-memory ring (one per stage) filled by
// cp.async in the same commit groups as the co-state rows, kRing - 1 beats
// ahead of use.  The six gene sums run in T over the owned cells and reach
// FP64 once per warp (FP64 arithmetic is slow here).
template <typename T, int K, int RX, int BC>
struct ReversePolicy {
    // A stage reads only its own ring slot of the beat and sums over owned
    // rows (q >= K, inside the light cone), so the fill may skip stages; the
    // state-row copies are issued per beat for every stage regardless.
    static constexpr bool kLightCone = true;
    typedef typename Vec<T>::type VT;
    const AdjCoef<T> &p;
    const StripGeom &geo;
    const StagePlanes<T> &state;
    T *__restrict__ lun;
    T *__restrict__ lvn;
    int nn, nm;
    VT (*aux)[kRing][2][32];  // [stage][slot][field][lane]
    RowWalk<BC> gw[K];        // next state row to copy, per stage (wrapped / reflected)
    T rg[6];                  // sums: u Lap(lu), v Lap(lv), lv, lv v, lv (u - b v), lu u

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < 6; ++q) rg[q] = T(0);
        // stage s at beat m reads input-row index q = m - s - 1
#pragma unroll
        for (int s = 0; s < K; ++s) gw[s].start((int64_t)geo.r0 - K - s - 1, nn);
    }
    __device__ __forceinline__ void issue(int j) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int s = 0; s < K; ++s) {
            const int64_t off = (int64_t)gw[s].g * nm + geo.lc;
            cp_async16(&aux[s][j % kRing][0][lane], state.u[s] + off);
            cp_async16(&aux[s][j % kRing][1][lane], state.v[s] + off);
            gw[s].next(nn);
        }
    }
    __device__ __forceinline__ void begin_beat(int) {}
    __device__ __forceinline__ void stage(int s, const Slice<T> &A, const Slice<T> &B, const Slice<T> &C,
                                          T wu, T eu, T wv, T ev, int q, Slice<T> &out) {
        constexpr int V = Vec<T>::N;
        const bool own = (q >= K) && (q < K + geo.nout) && geo.st_lane;
        const int lane = threadIdx.x & 31;
        const int slot = (q + s + 1) % kRing;  // beat m = q + s + 1
        const VT su4 = aux[s][slot][0][lane];
        const VT sv4 = aux[s][slot][1][lane];
        const T *stu = reinterpret_cast<const T *>(&su4);
        const T *stv = reinterpret_cast<const T *>(&sv4);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const T luc = B.u[e], lvc = B.v[e];
            const T su = add_rn(add_rn(A.u[e], C.u[e]), add_rn(e == 0 ? wu : B.u[e - 1],
                                                               e == V - 1 ? eu : B.u[e + 1]));
            const T sv = add_rn(add_rn(A.v[e], C.v[e]), add_rn(e == 0 ? wv : B.v[e - 1],
                                                               e == V - 1 ? ev : B.v[e + 1]));
            // a mirrored lane holds its state vector reversed, like its co-state
            const bool flip = (BC == BC_MIRROR) && geo.rev;
            const T uc = flip ? stu[V - 1 - e] : stu[e];
            const T vc = flip ? stv[V - 1 - e] : stv[e];
            // co-state update with the centre term folded in, like the forward:
            //   lu + dt [ Du s(lu) + (c - 4 Du - u^2) lu - eps lv ]
            //   lv + dt [ Dv s(lv) + (eps b - 4 Dv) lv - lu ]
            if constexpr (RX == RX_CENN) {
                // -lu + y'(u) (c lu + Du sum_nbr lu); y' in {0, 1}, so the product is exact
                const T slope = fabs(uc) < T(1) ? T(1) : T(0);
                const T back = fma_rn(p.Du, su, mul_rn(p.cm4, luc));
                out.u[e] = fma_rn(p.dt, fma_rn(slope, back, -luc), luc);
                out.v[e] = fma_rn(p.dt, luc, lvc);
                if (own) {
                    const T yc = clamp1(uc);
                    rg[0] = fma_rn(yc, su, rg[0]);   // y(u) sum_nbr lu  (Du)
                    rg[5] = fma_rn(luc, yc, rg[5]);  // lu y(u)          (c)
                }
                continue;
            }
            T ru, rv;
            if (RX == RX_FHN) {
                ru = fma_rn(fma_rn(-uc, uc, p.cm4), luc, mul_rn(p.meps, lvc));
                rv = fma_rn(p.ebm4, lvc, -luc);
            } else {
                ru = mul_rn(p.cm4, luc);
                rv = mul_rn(p.ebm4, lvc);
            }
            out.u[e] = fma_rn(p.dt, fma_rn(p.Du, su, ru), luc);
            out.v[e] = fma_rn(p.dt, fma_rn(p.Dv, sv, rv), lvc);
            if (own) {
                rg[0] = fma_rn(uc, fma_rn(T(-4), luc, su), rg[0]);     // u Lap(lu)
                rg[1] = fma_rn(vc, fma_rn(T(-4), lvc, sv), rg[1]);     // v Lap(lv)
                if (RX == RX_FHN) {
                    rg[2] = add_rn(rg[2], lvc);                        // lv        (x -eps)
                    rg[3] = fma_rn(lvc, vc, rg[3]);                    // lv v      (x eps)
                    rg[4] = fma_rn(lvc, fma_rn(p.mb, vc, uc), rg[4]);  // lv (u - b v)
                    rg[5] = fma_rn(luc, uc, rg[5]);                    // lu u
                }
            }
        }
    }
    __device__ __forceinline__ void finish(int q, const Slice<T> &out) {
        const int orow = q - K;
        if (orow >= 0 && geo.st_lane) {
            const int64_t off = (int64_t)(geo.r0 + orow) * nm + geo.sc;
            store_vec<T>(lun + off, out.u);
            store_vec<T>(lvn + off, out.v);
        }
    }
    __device__ __forceinline__ void flush(double *__restrict__ slot) {
#pragma unroll
        for (int q = 0; q < 6; ++q) rg[q] = warp_sum_t(rg[q]);
        if ((threadIdx.x & 31) == 0) {
            slot[0] += (double)rg[0];
            if (RX == RX_CENN) {
                slot[5] += (double)rg[5];
                return;
            }
            slot[1] += (double)rg[1];
            if (RX == RX_FHN) {
                slot[2] -= p.eps * (double)rg[2];
                slot[3] += p.eps * (double)rg[3];
                slot[4] -= (double)rg[4] + p.a * (double)rg[2];
                slot[5] += (double)rg[5];
            }
        }
    }
};

// K reverse steps: co-state (lu, lv) at t_hi -> (lun, lvn) at t_hi - K, with
// state.u[s], state.v[s] = state at t_hi - s - 1.  H: halo lanes (fixed per
// call sequence so every launch has the same warp -> cells map).
template <typename T, int K, int H, int RX, int BC>
__global__ void __launch_bounds__(kPipeBlock)
k_adjoint_pipe(const T *__restrict__ lu, const T *__restrict__ lv, T *__restrict__ lun,
               T *__restrict__ lvn, StagePlanes<T> state, double *__restrict__ partial, int nn,
               int nm, int bands, int nwarps, int rows, AdjCoef<T> p) {
    pdl_wait();
    const int wid = blockIdx.x * kTemporalWarps + (threadIdx.x >> 5);
    if (wid >= nwarps) return;
    const StripGeom geo = strip_geom<T, K, H, BC>(wid % bands, wid / bands, nn, nm, rows);
    typedef typename Vec<T>::type VT;
    // state rings in dynamic shared memory: [warp][stage][slot][field][lane]
    extern __shared__ __align__(16) unsigned char adj_dyn_smem[];
    VT(*aux_mem)[K][kRing][2][32] = reinterpret_cast<VT(*)[K][kRing][2][32]>(adj_dyn_smem);
    ReversePolicy<T, K, RX, BC> pol{p, geo, state, lun, lvn, nn, nm, aux_mem[(threadIdx.x >> 5) % kTemporalWarps]};
    pol.init();
    pipeline_strip<T, K, BC>(geo, lu, lv, nn, nm, pol);
    pol.flush(partial + (int64_t)wid * 6);
    pdl_trigger();
}

// K forward steps from (u, v), storing the state after every step s+1 into
// planes.u[s], planes.v[s] (the states a reverse sweep reads).
template <typename T, int K, int H, int RX, int BC>
__global__ void __launch_bounds__(kPipeBlock)
k_forward_all(const T *__restrict__ u, const T *__restrict__ v, StagePlanes<T> planes, int nn,
              int nm, int bands, int nwarps, int rows, Coef<T> p) {
    pdl_wait();
    const int wid = blockIdx.x * kTemporalWarps + (threadIdx.x >> 5);
    if (wid >= nwarps) return;
    const StripGeom geo = strip_geom<T, K, H, BC>(wid % bands, wid / bands, nn, nm, rows);
    ForwardAllPolicy<T, K, RX> pol{p, geo, planes, nm};
    pipeline_strip<T, K, BC>(geo, u, v, nn, nm, pol);
    pdl_trigger();
}

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

// Depth of the recompute / reverse launches: 4 steps with one halo lane for
// FP32, 2 steps (one lane of two doubles) for FP64.
inline int adj_depth(int dtype) { return dtype == RDCNN_F64 ? 2 : 4; }

struct PipeShape {
    int bands, strips, nwarps, rows;
};

// One warp -> cells map for every recompute / reverse launch of a call.
PipeShape pipe_shape(int dtype, int64_t nn, int64_t nm) {
    const int V = vec_width(dtype);
    const int outw = (32 - 2) * V;  // one halo lane per side
    PipeShape s;
    const int64_t cells = nn * nm;
    // strip length by size class; 512^2 measured 2 / 4 / 8 / 16 rows = 19.6 / 16.4 / 17.5 /
    // 22.6 ms for the T = 2000 adjoint (short strips fill more SMs, long ones waste less halo)
    s.rows = cells < (int64_t(1) << 19) ? 4 : cells < (int64_t(1) << 22) ? 16 : 64;
    s.bands = (int)((nm + outw - 1) / outw);
    s.strips = (int)((nn + s.rows - 1) / s.rows);
    s.nwarps = s.bands * s.strips;
    return s;
}

// Dynamic shared memory of k_adjoint_pipe<T, K>: the per-stage state rings.
template <typename T, int K>
constexpr size_t pipe_smem_bytes() {
    return (size_t)kTemporalWarps * K * kRing * 2 * 32 * sizeof(typename Vec<T>::type);
}

// Opt the kernel in to its dynamic shared memory (above the 48 KB default), once.
template <typename T, int K, int RX, int BC>
cudaError_t pipe_smem_optin() {
    static cudaError_t done = cudaErrorNotReady;
    if (done == cudaErrorNotReady)
        done = cudaFuncSetAttribute(k_adjoint_pipe<T, K, 1, RX, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)pipe_smem_bytes<T, K>());
    return done;
}


template <typename T, int K>
cudaError_t reverse_launch_k(int reaction, int boundary, const void *lu, const void *lv, void *lun, void *lvn,
                             const StagePlanes<T> &st, double *partial, int64_t nn, int64_t nm,
                             const PipeShape &sh, const rdcnn_params &p, cudaStream_t s) {
    const unsigned grid = (unsigned)((sh.nwarps + kTemporalWarps - 1) / kTemporalWarps);
    const AdjCoef<T> c = make_adj_coef<T>(p, reaction);
    const size_t smem = pipe_smem_bytes<T, K>();
    return with_model(reaction, boundary, [&](auto rx, auto bc) {
        constexpr int RX = decltype(rx)::value;
        constexpr int BC = decltype(bc)::value;
        const cudaError_t oe = pipe_smem_optin<T, K, RX, BC>();
        if (oe != cudaSuccess) return oe;
        const cudaError_t e = launch_k(k_adjoint_pipe<T, K, 1, RX, BC>, grid, kPipeBlock, smem, s, (const T *)lu,
                                       (const T *)lv, (T *)lun, (T *)lvn, st, partial, (int)nn, (int)nm,
                                       sh.bands, sh.nwarps, sh.rows, c);
        count_launches(1);
        return e;
    });
}

template <typename T, int K>
cudaError_t forward_all_launch_k(int reaction, int boundary, const void *u, const void *v,
                                 const StagePlanes<T> &pl, int64_t nn, int64_t nm, const PipeShape &sh,
                                 const rdcnn_params &p, cudaStream_t s) {
    const unsigned grid = (unsigned)((sh.nwarps + kTemporalWarps - 1) / kTemporalWarps);
    const Coef<T> c = make_coef<T>(p, reaction);
    return with_model(reaction, boundary, [&](auto rx, auto bc) {
        const cudaError_t e = launch_k(k_forward_all<T, K, 1, decltype(rx)::value, decltype(bc)::value>, grid,
                                       kPipeBlock, 0, s, (const T *)u, (const T *)v, pl, (int)nn, (int)nm,
                                       sh.bands, sh.nwarps, sh.rows, c);
        count_launches(1);
        return e;
    });
}

// Depth dispatch (depth <= V keeps one halo lane): F32 1..4, F64 1..2.
template <typename T>
cudaError_t reverse_launch(int reaction, int boundary, int k, const void *lu, const void *lv, void *lun,
                           void *lvn, const StagePlanes<T> &st, double *partial, int64_t nn, int64_t nm,
                           const PipeShape &sh, const rdcnn_params &p, cudaStream_t s) {
    switch (k) {
        case 1: return reverse_launch_k<T, 1>(reaction, boundary, lu, lv, lun, lvn, st, partial, nn, nm, sh, p, s);
        case 2: return reverse_launch_k<T, 2>(reaction, boundary, lu, lv, lun, lvn, st, partial, nn, nm, sh, p, s);
        case 3: if constexpr (Vec<T>::N >= 3) return reverse_launch_k<T, 3>(reaction, boundary, lu, lv, lun, lvn, st, partial, nn, nm, sh, p, s); break;
        case 4: if constexpr (Vec<T>::N >= 4) return reverse_launch_k<T, 4>(reaction, boundary, lu, lv, lun, lvn, st, partial, nn, nm, sh, p, s); break;
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t forward_all_launch(int reaction, int boundary, int k, const void *u, const void *v, const StagePlanes<T> &pl,
                               int64_t nn, int64_t nm, const PipeShape &sh, const rdcnn_params &p,
                               cudaStream_t s) {
    switch (k) {
        case 1: return forward_all_launch_k<T, 1>(reaction, boundary, u, v, pl, nn, nm, sh, p, s);
        case 2: return forward_all_launch_k<T, 2>(reaction, boundary, u, v, pl, nn, nm, sh, p, s);
        case 3: if constexpr (Vec<T>::N >= 3) return forward_all_launch_k<T, 3>(reaction, boundary, u, v, pl, nn, nm, sh, p, s); break;
        case 4: if constexpr (Vec<T>::N >= 4) return forward_all_launch_k<T, 4>(reaction, boundary, u, v, pl, nn, nm, sh, p, s); break;
    }
    return cudaErrorInvalidValue;
}

struct AdjLayout {
    int64_t S, nseg, nslots;
    size_t plane, ck_off, seg_off, lam_off, part_off, out_off, total;
};

AdjLayout adj_layout(int dtype, int64_t nn, int64_t nm, int64_t T, int64_t nck) {
    AdjLayout L{};
    if (nck <= 0) nck = (int64_t)std::ceil(std::sqrt((double)std::max<int64_t>(T, 1)));
    nck = std::max<int64_t>(1, std::min<int64_t>(nck, std::max<int64_t>(T, 1)));
    L.S = (std::max<int64_t>(T, 1) + nck - 1) / nck;
    L.nseg = (std::max<int64_t>(T, 1) + L.S - 1) / L.S;
    L.nslots = std::max<int64_t>(L.S, 2);
    L.plane = (((size_t)nn * nm * elem_size(dtype)) + 255) & ~(size_t)255;
    const PipeShape sh = pipe_shape(dtype, nn, nm);
    L.ck_off = 0;
    L.seg_off = L.ck_off + (size_t)L.nseg * 2 * L.plane;
    L.lam_off = L.seg_off + (size_t)L.nslots * 2 * L.plane;
    L.part_off = L.lam_off + 4 * L.plane;
    L.out_off = L.part_off + (((size_t)sh.nwarps * 6 * sizeof(double) + 255) & ~(size_t)255);
    L.total = L.out_off + 256;
    return L;
}

template <typename T>
int adjoint_t(int64_t nn, int64_t nm, const rdcnn_params &p, int dtype, int reaction, int boundary, cudaStream_t s,
              int64_t nsteps, const void *u0, const void *v0, const void *dLdu_T, const void *dLdv_T,
              const AdjLayout &L, char *ws, void *dLdu0, void *dLdv0, double grad[6]) {
    const size_t bytes = (size_t)nn * nm * sizeof(T);
    auto ck_u = [&](int64_t i) { return (T *)(ws + L.ck_off + (size_t)(2 * i) * L.plane); };
    auto ck_v = [&](int64_t i) { return (T *)(ws + L.ck_off + (size_t)(2 * i + 1) * L.plane); };
    auto seg_u = [&](int64_t i) { return (T *)(ws + L.seg_off + (size_t)(2 * i) * L.plane); };
    auto seg_v = [&](int64_t i) { return (T *)(ws + L.seg_off + (size_t)(2 * i + 1) * L.plane); };
    T *lam_u[2] = {(T *)(ws + L.lam_off), (T *)(ws + L.lam_off + 2 * L.plane)};
    T *lam_v[2] = {(T *)(ws + L.lam_off + L.plane), (T *)(ws + L.lam_off + 3 * L.plane)};
    double *partial = (double *)(ws + L.part_off);
    double *gout = (double *)(ws + L.out_off);
    const PipeShape sh = pipe_shape(dtype, nn, nm);
    const int kf = default_k(dtype, nn, nm);  // depth of the checkpoint sweep
    const int ka = adj_depth(dtype);          // depth of recompute / reverse launches

    cudaError_t e = cudaMemcpyAsync(lam_u[0], dLdu_T, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lam_v[0], dLdv_T, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ck_u(0), u0, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ck_v(0), v0, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(partial, 0, (size_t)sh.nwarps * 6 * sizeof(double), s);
    if (e != cudaSuccess) return cuda_error(e, "adjoint setup copies");

    // forward sweep: checkpoint i = state at step i*S
    for (int64_t i = 0; i + 1 < L.nseg && nsteps > 0; ++i) {
        const int64_t len = L.S;
        const int64_t nl = (len + kf - 1) / kf;
        const void *cu = ck_u(i), *cv = ck_v(i);
        for (int64_t j = 0; j < nl; ++j) {
            const int kk = (int)std::min<int64_t>(kf, len - j * kf);
            void *nu = (j == nl - 1) ? (void *)ck_u(i + 1) : (void *)seg_u(j % 2);
            void *nv = (j == nl - 1) ? (void *)ck_v(i + 1) : (void *)seg_v(j % 2);
            e = launch_temporal(dtype, reaction, boundary, kk, cu, cv, nu, nv, nn, nm, p, 0, s);
            if (e != cudaSuccess) return cuda_error(e, "adjoint forward sweep");
            cu = nu; cv = nv;
        }
    }
    // segments last to first: rebuild the states, then sweep the co-state back
    int cur = 0;
    for (int64_t sg = L.nseg - 1; sg >= 0 && nsteps > 0; --sg) {
        const int64_t len = std::min<int64_t>(L.S, nsteps - sg * L.S);
        auto state_u = [&](int64_t q) { return q == 0 ? ck_u(sg) : seg_u(q); };
        auto state_v = [&](int64_t q) { return q == 0 ? ck_v(sg) : seg_v(q); };
        for (int64_t q = 0; q + 1 < len;) {
            const int kk = (int)std::min<int64_t>(ka, len - 1 - q);
            StagePlanes<T> pl{};
            for (int j = 0; j < kk; ++j) { pl.u[j] = seg_u(q + 1 + j); pl.v[j] = seg_v(q + 1 + j); }
            e = forward_all_launch<T>(reaction, boundary, kk, state_u(q), state_v(q), pl, nn, nm, sh, p, s);
            if (e != cudaSuccess) return cuda_error(e, "adjoint recompute");
            q += kk;
        }
        for (int64_t qh = len; qh > 0;) {
            const int kk = (int)std::min<int64_t>(ka, qh);
            StagePlanes<T> st{};
            for (int j = 0; j < kk; ++j) { st.u[j] = state_u(qh - 1 - j); st.v[j] = state_v(qh - 1 - j); }
            e = reverse_launch<T>(reaction, boundary, kk, lam_u[cur], lam_v[cur], lam_u[cur ^ 1], lam_v[cur ^ 1], st,
                                  partial, nn, nm, sh, p, s);
            if (e != cudaSuccess) return cuda_error(e, "adjoint reverse step");
            cur ^= 1;
            qh -= kk;
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
    *bytes = adj_layout(dtype, nn, nm, T, n_checkpoints).total;
    return RDCNN_OK;
}

int rdcnn_adjoint(rdcnn_t *h, int64_t T, const void *u0, const void *v0, const void *dLdu_T,
                  const void *dLdv_T, int64_t n_checkpoints, void *dLdu0, void *dLdv0,
                  double grad[6], void *workspace, size_t workspace_bytes) {
    int64_t nn, nm; rdcnn_params p; int dtype, reaction, boundary; cudaStream_t s;
    int rc = handle_view(h, &nn, &nm, &p, &dtype, &reaction, &s, &boundary);
    if (rc < 0) return rc;
    if (is_16bit(dtype)) return set_error(RDCNN_EINVAL, "the adjoint supports FP32 / FP64 handles only");
    if (T < 0) return set_error(RDCNN_EINVAL, "T must be >= 0");
    if (!u0 || !v0 || !dLdu_T || !dLdv_T || !dLdu0 || !dLdv0 || !grad || !workspace)
        return set_error(RDCNN_EINVAL, "NULL argument");
    const int V = vec_width(dtype);
    if (nm % V != 0) return set_error(RDCNN_EINVAL, "adjoint needs NM %% %d == 0", V);
    const void *ptrs[7] = {u0, v0, dLdu_T, dLdv_T, dLdu0, dLdv0, workspace};
    for (const void *q : ptrs)
        if (!aligned16(q)) return set_error(RDCNN_EINVAL, "adjoint buffers must be 16-byte aligned");
    const AdjLayout L = adj_layout(dtype, nn, nm, T, n_checkpoints);
    if (workspace_bytes < L.total)
        return set_error(RDCNN_ESPACE, "adjoint workspace has %zu bytes, need %zu", workspace_bytes, L.total);
    if (dtype == RDCNN_F64)
        return adjoint_t<double>(nn, nm, p, dtype, reaction, boundary, s, T, u0, v0, dLdu_T, dLdv_T, L,
                                 (char *)workspace, dLdu0, dLdv0, grad);
    return adjoint_t<float>(nn, nm, p, dtype, reaction, boundary, s, T, u0, v0, dLdu_T, dLdv_T, L,
                            (char *)workspace, dLdu0, dLdv0, grad);
}

}  // extern "C"
