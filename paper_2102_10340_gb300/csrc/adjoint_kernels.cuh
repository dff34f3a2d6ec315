// adjoint_kernels.cuh -- the adjoint's two pipelines (k_forward_all rebuilds
// a segment's states, k_adjoint_pipe runs the co-state backwards; derivation
// in adjoint.cu) and their launchers for one (element type, depth K, halo
// lanes H).  The adjoint_*.cu units instantiate them, so the kernels of every
// model compile in parallel.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "temporal.cuh"

namespace rdk {

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
    __device__ __forceinline__ void finish_main(int q, const Slice<T> &out) { finish(q, out); }
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

// Warp -> cells map shared by every recompute / reverse launch of a call.
struct PipeShape {
    int bands, strips, nwarps, rows;
};

// Dynamic shared memory of k_adjoint_pipe<T, K>: the per-stage state rings.
template <typename T, int K>
constexpr size_t pipe_smem_bytes() {
    return (size_t)kTemporalWarps * K * kRing * 2 * 32 * sizeof(typename Vec<T>::type);
}

// Opt the kernel in to its dynamic shared memory (above the 48 KB default), once.
template <typename T, int K, int H, int RX, int BC>
cudaError_t pipe_smem_optin() {
    static cudaError_t done = cudaErrorNotReady;
    if (done == cudaErrorNotReady)
        done = cudaFuncSetAttribute(k_adjoint_pipe<T, K, H, RX, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)pipe_smem_bytes<T, K>());
    return done;
}

// K reverse steps of the co-state on the call's warp map (halo H lanes).
template <typename T, int K, int H>
cudaError_t reverse_launch_kh(int reaction, int boundary, const void *lu, const void *lv, void *lun, void *lvn,
                              const StagePlanes<T> &st, double *partial, int64_t nn, int64_t nm,
                              const PipeShape &sh, const rdcnn_params &p, cudaStream_t s) {
    const unsigned grid = (unsigned)((sh.nwarps + kTemporalWarps - 1) / kTemporalWarps);
    const AdjCoef<T> c = make_adj_coef<T>(p, reaction);
    const size_t smem = pipe_smem_bytes<T, K>();
    return with_model(reaction, boundary, [&](auto rx, auto bc) {
        constexpr int RX = decltype(rx)::value;
        constexpr int BC = decltype(bc)::value;
        const cudaError_t oe = pipe_smem_optin<T, K, H, RX, BC>();
        if (oe != cudaSuccess) return oe;
        const cudaError_t e = launch_k(k_adjoint_pipe<T, K, H, RX, BC>, grid, kPipeBlock, smem, s, (const T *)lu,
                                       (const T *)lv, (T *)lun, (T *)lvn, st, partial, (int)nn, (int)nm,
                                       sh.bands, sh.nwarps, sh.rows, c);
        count_launches(1);
        return e;
    });
}

// K forward steps storing every step's state, on the call's warp map.
template <typename T, int K, int H>
cudaError_t forward_all_launch_kh(int reaction, int boundary, const void *u, const void *v,
                                  const StagePlanes<T> &pl, int64_t nn, int64_t nm, const PipeShape &sh,
                                  const rdcnn_params &p, cudaStream_t s) {
    const unsigned grid = (unsigned)((sh.nwarps + kTemporalWarps - 1) / kTemporalWarps);
    const Coef<T> c = make_coef<T>(p, reaction);
    return with_model(reaction, boundary, [&](auto rx, auto bc) {
        const cudaError_t e = launch_k(k_forward_all<T, K, H, decltype(rx)::value, decltype(bc)::value>, grid,
                                       kPipeBlock, 0, s, (const T *)u, (const T *)v, pl, (int)nn, (int)nm,
                                       sh.bands, sh.nwarps, sh.rows, c);
        count_launches(1);
        return e;
    });
}

}  // namespace rdk

// Explicit instantiation of the two launchers for (TT, KK, HH) / a
// declaration that another unit instantiates them.
#define RDK_ADJ_REV_SIG(TT, KK, HH)                                                                          \
    cudaError_t rdk::reverse_launch_kh<TT, KK, HH>(int, int, const void *, const void *, void *, void *,       \
                                                   const rdk::StagePlanes<TT> &, double *, int64_t, int64_t,   \
                                                   const rdk::PipeShape &, const rdcnn_params &, cudaStream_t)
#define RDK_ADJ_FWD_SIG(TT, KK, HH)                                                                          \
    cudaError_t rdk::forward_all_launch_kh<TT, KK, HH>(int, int, const void *, const void *,                   \
                                                       const rdk::StagePlanes<TT> &, int64_t, int64_t,         \
                                                       const rdk::PipeShape &, const rdcnn_params &, cudaStream_t)
#define RDK_INSTANTIATE_ADJ(TT, KK, HH) template RDK_ADJ_REV_SIG(TT, KK, HH); template RDK_ADJ_FWD_SIG(TT, KK, HH);
#define RDK_EXTERN_ADJ(TT, KK, HH) extern template RDK_ADJ_REV_SIG(TT, KK, HH); extern template RDK_ADJ_FWD_SIG(TT, KK, HH);
