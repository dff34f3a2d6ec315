// common.cuh -- device-side building blocks shared by the RD-CNN kernels.
//
// The cell update is Eq. 1 of Sec. II.A with the FitzHugh-Nagumo terms of
// Eq. 2-3, or one of the other local models the simulator is a template for
// (Sec. I, Sec. II.A): pure diffusion, and the Chua-Yang cellular neural
// network cell.  Every kernel of the library (single step, temporally
// blocked, batched) computes a cell through cell_update() below, and
// cell_update() spells out each rounding with the *_rn intrinsics, so the
// compiler cannot contract or reorder differently in different kernels: all
// variants give bit-identical states for the same inputs.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "rdcnn.h"

namespace rdk {

constexpr unsigned kFull = 0xffffffffu;

// Local model (values equal to RDCNN_REACTION_*).
enum { RX_FHN = 0, RX_NONE = 1, RX_CENN = 2 };

// Boundary (values equal to RDCNN_BC_*): wrap = torus; mirror = zero flux,
// the ghost cell beyond an edge holds the edge cell's value.
enum { BC_WRAP = 0, BC_MIRROR = 1 };

template <int N> using IntC = std::integral_constant<int, N>;

// Host-side dispatch of a runtime (reaction, boundary) pair to a callable
// taking the two as compile-time tags: f(IntC<RX>{}, IntC<BC>{}).
template <class F>
inline cudaError_t with_model(int reaction, int boundary, F &&f) {
    const bool zf = (boundary == RDCNN_BC_ZEROFLUX);
    switch (reaction) {
        case RDCNN_REACTION_FHN:
            return zf ? f(IntC<RX_FHN>{}, IntC<BC_MIRROR>{}) : f(IntC<RX_FHN>{}, IntC<BC_WRAP>{});
        case RDCNN_REACTION_NONE:
            return zf ? f(IntC<RX_NONE>{}, IntC<BC_MIRROR>{}) : f(IntC<RX_NONE>{}, IntC<BC_WRAP>{});
        case RDCNN_REACTION_CENN:
            return zf ? f(IntC<RX_CENN>{}, IntC<BC_MIRROR>{}) : f(IntC<RX_CENN>{}, IntC<BC_WRAP>{});
        default:
            return cudaErrorInvalidValue;
    }
}

// 16-byte vector of the element type: the unit each lane loads and stores.
template <typename T> struct Vec;
template <> struct Vec<float> {
    typedef float4 type;
    static constexpr int N = 4;
};
template <> struct Vec<double> {
    typedef double2 type;
    static constexpr int N = 2;
};

// Gene in the form the update consumes.  The -4 centre weight of the
// Laplacian is folded into the reaction coefficients (cm4 = c - 4 Du,
// ebm4 = eps b - 4 Dv); the state itself always enters the final FMA
// exactly, so only increment-sized terms carry coefficient rounding.
// With no reaction: cm4 = -4 Du, ebm4 = -4 Dv, mthird = meps = mepsa = 0.
// CeNN cell: cm4 = c (feedback centre), Du = feedback arms, the rest 0.
template <typename T> struct Coef {
    T dt, Du, Dv, cm4, mthird, meps, ebm4, mepsa;
};

__device__ __forceinline__ float add_rn(float x, float y) { return __fadd_rn(x, y); }
__device__ __forceinline__ double add_rn(double x, double y) { return __dadd_rn(x, y); }
__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }
__device__ __forceinline__ float fma_rn(float x, float y, float z) { return __fmaf_rn(x, y, z); }
__device__ __forceinline__ double fma_rn(double x, double y, double z) { return __fma_rn(x, y, z); }

__device__ __forceinline__ float clamp1(float x) { return fminf(fmaxf(x, -1.0f), 1.0f); }
__device__ __forceinline__ double clamp1(double x) { return fmin(fmax(x, -1.0), 1.0); }

// One cell.  c* = centre, n/s = rows i-1/i+1, w/e = columns j-1/j+1.
// FitzHugh-Nagumo (Eq. 1-3) is evaluated as
//   u+ = u + dt [ Du ((n + s) + (w + e)) + u (c - 4 Du - u^2/3) - v ]
//   v+ = v + dt [ Dv ((n + s) + (w + e)) - eps u + (eps b - 4 Dv) v - eps a ]
// i.e. with the -4 Du u (-4 Dv v) term of the Laplacian moved into the
// reaction polynomial: 15 FP instructions per cell instead of 18.  The state
// is the exact addend of the last FMA, so the FP32 accuracy is that of the
// literal form.
// CeNN (Chua-Yang cell, output y(x) = clamp(x, -1, 1), which equals
// (|x + 1| - |x - 1|) / 2; u = state x, v = offset plane w, held constant):
//   u+ = u + dt [ Du ((y_n + y_s) + (y_w + y_e)) + c y(u) + (w - u) ],  v+ = v.
// A NaN state stays NaN (it is the exact addend); a NaN neighbour's output
// saturates to -1 instead of propagating.
template <typename T, int RX>
__device__ __forceinline__ void cell_update(T uc, T un, T us, T uw, T ue,
                                            T vc, T vn, T vs, T vw, T ve,
                                            const Coef<T> &p, T &out_u, T &out_v) {
    if constexpr (RX == RX_CENN) {
        const T sy = add_rn(add_rn(clamp1(un), clamp1(us)), add_rn(clamp1(uw), clamp1(ue)));
        out_u = fma_rn(p.dt, fma_rn(p.Du, sy, fma_rn(p.cm4, clamp1(uc), add_rn(vc, -uc))), uc);
        out_v = vc;
        return;
    }
    const T su = add_rn(add_rn(un, us), add_rn(uw, ue));      // neighbour sum of u
    const T sv = add_rn(add_rn(vn, vs), add_rn(vw, ve));      // neighbour sum of v
    T ru, rv;
    if (RX == RX_FHN) {
        const T cm = fma_rn(mul_rn(uc, uc), p.mthird, p.cm4);  // c - 4 Du - u^2/3
        ru = fma_rn(uc, cm, -vc);                               // Eq. 2 (+ centre term)
        rv = fma_rn(p.meps, uc, fma_rn(p.ebm4, vc, p.mepsa));   // Eq. 3 (+ centre term)
    } else {
        ru = mul_rn(p.cm4, uc);                                 // -4 Du u
        rv = mul_rn(p.ebm4, vc);                                // -4 Dv v
    }
    out_u = fma_rn(p.dt, fma_rn(p.Du, su, ru), uc);
    out_v = fma_rn(p.dt, fma_rn(p.Dv, sv, rv), vc);
}

// A lane's slice of one grid row for both fields: V consecutive columns.
template <typename T> struct Slice {
    T u[Vec<T>::N];
    T v[Vec<T>::N];
};

template <typename T>
__device__ __forceinline__ void load_vec(T (&dst)[Vec<T>::N], const T *__restrict__ src) {
    typedef typename Vec<T>::type VT;
    const VT x = __ldg(reinterpret_cast<const VT *>(src));
    if constexpr (Vec<T>::N == 4) {
        dst[0] = x.x; dst[1] = x.y; dst[2] = x.z; dst[3] = x.w;
    } else {
        dst[0] = x.x; dst[1] = x.y;
    }
}

template <typename T>
__device__ __forceinline__ void store_vec(T *__restrict__ dst, const T (&src)[Vec<T>::N]) {
    typedef typename Vec<T>::type VT;
    VT x;
    if constexpr (Vec<T>::N == 4) {
        x.x = src[0]; x.y = src[1]; x.z = src[2]; x.w = src[3];
    } else {
        x.x = src[0]; x.y = src[1];
    }
    *reinterpret_cast<VT *>(dst) = x;
}

// Stencil over one lane's slice.  cen = row i, nor = row i-1, sou = row i+1.
// The west neighbour of element 0 and the east neighbour of element V-1 come
// from the adjacent lanes (or, for lanes whose neighbour is not in the warp,
// from the caller: west_u/east_u etc.).
template <typename T, int RX>
__device__ __forceinline__ void slice_update(const Slice<T> &nor, const Slice<T> &cen,
                                             const Slice<T> &sou, T west_u, T east_u,
                                             T west_v, T east_v, const Coef<T> &p,
                                             Slice<T> &out) {
    constexpr int V = Vec<T>::N;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const T wu = (e == 0) ? west_u : cen.u[e - 1];
        const T eu = (e == V - 1) ? east_u : cen.u[e + 1];
        const T wv = (e == 0) ? west_v : cen.v[e - 1];
        const T ev = (e == V - 1) ? east_v : cen.v[e + 1];
        cell_update<T, RX>(cen.u[e], nor.u[e], sou.u[e], wu, eu,
                        cen.v[e], nor.v[e], sou.v[e], wv, ev, p, out.u[e], out.v[e]);
    }
}

template <typename T>
inline Coef<T> make_coef(const rdcnn_params &p, int reaction) {
    const bool fhn = (reaction == RDCNN_REACTION_FHN);
    Coef<T> q;
    if (reaction == RDCNN_REACTION_CENN) {
        q.dt = T(p.dt);
        q.Du = T(p.Du);
        q.Dv = T(0);
        q.cm4 = T(p.c);
        q.mthird = q.meps = q.ebm4 = q.mepsa = T(0);
        return q;
    }
    q.dt = T(p.dt);
    q.Du = T(p.Du);
    q.Dv = T(p.Dv);
    q.cm4 = T((fhn ? p.c : 0.0) - 4.0 * p.Du);
    q.mthird = T(fhn ? -1.0 / 3.0 : 0.0);
    q.meps = T(fhn ? -p.eps : 0.0);
    q.ebm4 = T((fhn ? p.eps * p.b : 0.0) - 4.0 * p.Dv);
    q.mepsa = T(fhn ? -p.eps * p.a : 0.0);
    return q;
}

template <typename T>
__device__ __forceinline__ void load_slice(Slice<T> &s, const T *__restrict__ u,
                                           const T *__restrict__ v, int64_t off) {
    load_vec<T>(s.u, u + off);
    load_vec<T>(s.v, v + off);
}

template <typename T>
__device__ __forceinline__ void zero_slice(Slice<T> &s) {
#pragma unroll
    for (int e = 0; e < Vec<T>::N; ++e) {
        s.u[e] = T(0);
        s.v[e] = T(0);
    }
}

__device__ __forceinline__ int wrap_row(int64_t r, int64_t n) {
    int64_t q = r % n;
    return (int)(q < 0 ? q + n : q);
}

// Index that stands in for row/column r under boundary BC: wrapped modulo n
// on the torus; under zero flux, reflected about the edge faces (r = -1 -> 0,
// r = n -> n - 1, and periodically with period 2n beyond that).
template <int BC>
__device__ __forceinline__ int bc_index(int64_t r, int64_t n) {
    if constexpr (BC == BC_MIRROR) {
        const int q = wrap_row(r, 2 * n);
        return q < n ? q : (int)(2 * n - 1 - q);
    } else {
        return wrap_row(r, n);
    }
}

}  // namespace rdk
