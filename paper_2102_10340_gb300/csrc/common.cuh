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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
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

// Programmatic dependent launch.  A stepping kernel launched with the
// programmatic-serialization attribute (launch_k in internal.h) may be
// scheduled while the previous kernel of the stream is still draining.
// pdl_wait() returns when the previous kernel has completed and its writes
// are visible: every kernel launched this way calls it before its first
// global memory access (reads and writes: the ping-pong planes are read by
// one launch and overwritten by the next).  pdl_trigger(), called when a
// thread's work is done, lets the next kernel be scheduled once every block
// of this one has called it or exited, so its launch overlaps this kernel's
// tail.  Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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

// Host-side dispatch of a storage dtype (RDCNN_F32 / F64 / BF16 / F16) to a
// callable taking a value of that type as a tag, and of a temporal depth
// 1..8 to a callable taking IntC<K>.
template <class F>
inline auto with_dtype(int dtype, F &&f) {
    switch (dtype) {
        case RDCNN_F64: return f(double{});
        case RDCNN_BF16: return f(__nv_bfloat16{});
        case RDCNN_F16: return f(__half{});
        default: return f(float{});
    }
}
template <class F>
inline cudaError_t with_depth(int k, F &&f) {
    switch (k) {
        case 1: return f(IntC<1>{});
        case 2: return f(IntC<2>{});
        case 3: return f(IntC<3>{});
        case 4: return f(IntC<4>{});
        case 5: return f(IntC<5>{});
        case 6: return f(IntC<6>{});
        case 7: return f(IntC<7>{});
        case 8: return f(IntC<8>{});
        default: return cudaErrorInvalidValue;
    }
}
// Deepest temporal pipeline per storage type (register budget).
template <typename T> struct MaxDepth : IntC<8> {};
template <> struct MaxDepth<double> : IntC<4> {};

// V values of storage type T held by one lane: 16 bytes (float x 4,
// double x 2) or 8 bytes (16-bit x 4).
template <typename T, int V> struct LaneVec;
template <> struct LaneVec<float, 4> { typedef float4 type; };
template <> struct LaneVec<double, 2> { typedef double2 type; };
template <> struct LaneVec<__nv_bfloat16, 4> { typedef uint2 type; };
template <> struct LaneVec<__half, 4> { typedef uint2 type; };

// A storage type E read 8 values per lane (16 bytes of a 16-bit type, 32 of
// float): the same bits in memory as E, a distinct type so that a pipeline
// instantiated on it takes the wider lane.  The fixed per-row costs of a
// lane (ring copies, addresses, shuffles, loop) then cover twice the cells,
// and one halo lane covers a depth of up to 8 instead of 4.
template <typename E> struct Wide { E x; };
struct __align__(16) Float8 { float4 a, b; };
template <> struct LaneVec<Wide<__nv_bfloat16>, 8> { typedef uint4 type; };
template <> struct LaneVec<Wide<__half>, 8> { typedef uint4 type; };
template <> struct LaneVec<Wide<float>, 8> { typedef Float8 type; };

// The element format behind a storage type (itself for the plain types).
template <typename T> struct Base16 { typedef T type; };
template <typename E> struct Base16<Wide<E>> { typedef E type; };

// Lane width of the register pipelines: 4 values (2 doubles) of every
// storage type, so that 16-bit planes share the FP32 lane layout and
// register budget (8 bytes per lane and field); 8 for Wide.
template <typename T> struct Vec {
    static constexpr int N = std::is_same<T, double>::value ? 2 : 4;
    typedef typename LaneVec<T, N>::type type;
};
template <typename E> struct Vec<Wide<E>> {
    static constexpr int N = 8;
    typedef typename LaneVec<Wide<E>, 8>::type type;
};

// Arithmetic type of a storage type: 16-bit planes are computed in FP32 and
// rounded (to nearest, ties to even) only when stored.
template <typename T> struct Compute { typedef T type; };
template <> struct Compute<__nv_bfloat16> { typedef float type; };
template <> struct Compute<__half> { typedef float type; };
template <typename E> struct Compute<Wide<E>> { typedef float type; };
template <typename T> using CT = typename Compute<T>::type;

// float / double planes: arithmetic in the storage type itself.
template <typename T>
constexpr bool is_f32_f64() { return std::is_same<T, float>::value || std::is_same<T, double>::value; }

// Storage vector <-> compute values.
template <typename T, int V>
__device__ __forceinline__ void unpack_vec(const typename LaneVec<T, V>::type &x, CT<T> (&d)[V]) {
    if constexpr (std::is_same<T, float>::value) {
        d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
    } else if constexpr (std::is_same<T, Wide<float>>::value) {
        d[0] = x.a.x; d[1] = x.a.y; d[2] = x.a.z; d[3] = x.a.w;
        d[4] = x.b.x; d[5] = x.b.y; d[6] = x.b.z; d[7] = x.b.w;
    } else if constexpr (std::is_same<T, double>::value) {
        d[0] = x.x; d[1] = x.y;
    } else {
        const unsigned *w = reinterpret_cast<const unsigned *>(&x);  // two values per word
#pragma unroll
        for (int i = 0; i < V / 2; ++i) {
            float2 f;
            if constexpr (std::is_same<typename Base16<T>::type, __nv_bfloat16>::value)
                f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[i]));
            else
                f = __half22float2(*reinterpret_cast<const __half2 *>(&w[i]));
            d[2 * i] = f.x;
            d[2 * i + 1] = f.y;
        }
    }
}
template <typename T, int V>
__device__ __forceinline__ typename LaneVec<T, V>::type pack_vec(const CT<T> (&s)[V]) {
    if constexpr (std::is_same<T, float>::value) {
        return make_float4(s[0], s[1], s[2], s[3]);
    } else if constexpr (std::is_same<T, Wide<float>>::value) {
        Float8 r;
        r.a = make_float4(s[0], s[1], s[2], s[3]);
        r.b = make_float4(s[4], s[5], s[6], s[7]);
        return r;
    } else if constexpr (std::is_same<T, double>::value) {
        return make_double2(s[0], s[1]);
    } else {
        typename LaneVec<T, V>::type r;
        unsigned *w = reinterpret_cast<unsigned *>(&r);
#pragma unroll
        for (int i = 0; i < V / 2; ++i) {
            if constexpr (std::is_same<typename Base16<T>::type, __nv_bfloat16>::value) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(s[2 * i], s[2 * i + 1]);
                w[i] = *reinterpret_cast<const unsigned *>(&h);
            } else {
                const __half2 h = __floats2half2_rn(s[2 * i], s[2 * i + 1]);
                w[i] = *reinterpret_cast<const unsigned *>(&h);
            }
        }
        return r;
    }
}

// One element: read-only load converted to the compute type / store rounded.
template <typename T>
__device__ __forceinline__ CT<T> load1(const T *p) {
    if constexpr (std::is_same<T, float>::value || std::is_same<T, double>::value) return __ldg(p);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value)
        return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
    else
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p))));
}
template <typename T>
__device__ __forceinline__ CT<T> to_compute(T x) {
    if constexpr (std::is_same<T, float>::value || std::is_same<T, double>::value) return x;
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __bfloat162float(x);
    else return __half2float(x);
}
template <typename T>
__device__ __forceinline__ T to_storage(CT<T> x) {
    if constexpr (std::is_same<T, float>::value || std::is_same<T, double>::value) return x;
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __float2bfloat16_rn(x);
    else return __float2half_rn(x);
}

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
template <typename T, int N = Vec<T>::N> struct Slice {
    T u[N];
    T v[N];
};

template <typename T, int V>
__device__ __forceinline__ void load_vec(CT<T> (&dst)[V], const T *__restrict__ src) {
    typedef typename LaneVec<T, V>::type VT;
    const VT x = __ldg(reinterpret_cast<const VT *>(src));
    unpack_vec<T, V>(x, dst);
}

template <typename T, int V>
__device__ __forceinline__ void store_vec(T *__restrict__ dst, const CT<T> (&src)[V]) {
    typedef typename LaneVec<T, V>::type VT;
    *reinterpret_cast<VT *>(dst) = pack_vec<T, V>(src);
}

// Stencil over one lane's slice.  cen = row i, nor = row i-1, sou = row i+1.
// The west neighbour of element 0 and the east neighbour of element V-1 come
// from the adjacent lanes (or, for lanes whose neighbour is not in the warp,
// from the caller: west_u/east_u etc.).
template <typename T, int RX, int V = Vec<T>::N>
__device__ __forceinline__ void slice_update(const Slice<T, V> &nor, const Slice<T, V> &cen,
                                             const Slice<T, V> &sou, T west_u, T east_u,
                                             T west_v, T east_v, const Coef<T> &p,
                                             Slice<T, V> &out) {
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

template <typename T, int V = Vec<T>::N>
__device__ __forceinline__ void load_slice(Slice<CT<T>, V> &s, const T *__restrict__ u,
                                           const T *__restrict__ v, int64_t off) {
    load_vec<T>(s.u, u + off);
    load_vec<T>(s.v, v + off);
}

template <typename T, int N>
__device__ __forceinline__ void zero_slice(Slice<T, N> &s) {
#pragma unroll
    for (int e = 0; e < N; ++e) {
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
