// common.cuh -- device-side building blocks shared by the RD-CNN kernels.
//
// The cell update is Eq. 1 of Sec. II.A with the FitzHugh-Nagumo terms of
// Eq. 2-3.  Every kernel of the library (single step, temporally blocked,
// batched) computes a cell through fhn_cell() below, and fhn_cell() spells
// out each rounding with the *_rn intrinsics, so the compiler cannot contract
// or reorder differently in different kernels: all variants give bit-identical
// states for the same inputs.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rdcnn.h"

namespace rdk {

constexpr unsigned kFull = 0xffffffffu;

enum { RX_FHN = 0, RX_NONE = 1 };

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

// Gene in the form the update consumes.  mb = -b, meps = -eps,
// mthird = -1/3 (rounded to T).
template <typename T> struct Coef {
    T dt, a, mb, meps, c, Du, Dv, mthird;
};

__device__ __forceinline__ float add_rn(float x, float y) { return __fadd_rn(x, y); }
__device__ __forceinline__ double add_rn(double x, double y) { return __dadd_rn(x, y); }
__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }
__device__ __forceinline__ float fma_rn(float x, float y, float z) { return __fmaf_rn(x, y, z); }
__device__ __forceinline__ double fma_rn(double x, double y, double z) { return __fma_rn(x, y, z); }

// One cell of Eq. 1.  c* = centre, n/s = rows i-1/i+1, w/e = columns j-1/j+1.
// Laplacian grouped as ((n + s) + (w + e)) - 4 c, so a uniform field gives
// exactly 0 (the sum of the two pairs is exactly 4c).
template <typename T, int RX>
__device__ __forceinline__ void fhn_cell(T uc, T un, T us, T uw, T ue,
                                         T vc, T vn, T vs, T vw, T ve,
                                         const Coef<T> &p, T &out_u, T &out_v) {
    const T lu = fma_rn(T(-4), uc, add_rn(add_rn(un, us), add_rn(uw, ue)));
    const T lv = fma_rn(T(-4), vc, add_rn(add_rn(vn, vs), add_rn(vw, ve)));
    T ru, rv;
    if (RX == RX_FHN) {
        const T uu = mul_rn(uc, uc);
        const T cm = fma_rn(uu, p.mthird, p.c);              // c - u^2/3
        ru = fma_rn(uc, cm, -vc);                             // f1 = u (c - u^2/3) - v   (Eq. 2)
        const T w = add_rn(fma_rn(p.mb, vc, uc), p.a);        // u - b v + a
        rv = mul_rn(p.meps, w);                               // f2 = -eps (u - b v + a)  (Eq. 3)
    } else {
        ru = T(0);
        rv = T(0);
    }
    out_u = fma_rn(p.dt, fma_rn(p.Du, lu, ru), uc);          // u + dt (f1 + Du lap u)
    out_v = fma_rn(p.dt, fma_rn(p.Dv, lv, rv), vc);          // v + dt (f2 + Dv lap v)
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
        fhn_cell<T, RX>(cen.u[e], nor.u[e], sou.u[e], wu, eu,
                        cen.v[e], nor.v[e], sou.v[e], wv, ev, p, out.u[e], out.v[e]);
    }
}

template <typename T>
inline Coef<T> make_coef(const rdcnn_params &p) {
    Coef<T> c;
    c.dt = T(p.dt);
    c.a = T(p.a);
    c.mb = T(-p.b);
    c.meps = T(-p.eps);
    c.c = T(p.c);
    c.Du = T(p.Du);
    c.Dv = T(p.Dv);
    c.mthird = T(-1.0 / 3.0);
    return c;
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

}  // namespace rdk
