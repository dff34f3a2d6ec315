// temporal_split.cuh -- the K-stage register pipeline of temporal.cuh split
// across a pair of warps that own the same (band, strip) work item.
//
// The first warp of a pair (producer) streams the input rows through the
// cp.async ring and runs stages 1 .. K/2; at beat m it writes its last
// stage's row into handoff slot m % 2.  The second warp (consumer) reads that
// row one beat later and runs stages K/2 + 1 .. K, storing the owned output
// rows.  Each warp holds half the register windows, so more warps fit on an
// SM.  The pair meets at a named barrier (bar.sync, 64 threads, id 1 + pair)
// once per beat: slot m % 2 is written before the barrier that ends beat m
// and read after it, and rewritten only after the barrier that ends beat
// m + 1, by which time the consumer has read it.  Both warps run exactly
// total + 1 beats, so their barrier counts always match; the only early exit
// (a pair without work) happens before any barrier and for both warps.
//
// Same arithmetic and the same cells as temporal_strip: identical bits, on
// the torus and under zero flux (the producer walks the reflected rows and
// reverses mirrored lane vectors exactly as temporal_strip does).
//
// Light-cone fill (as in temporal.cuh): global stage s first matters at the
// equivalent single-warp beat 2s + 2.  The producer's beat m is that beat;
// the consumer's beat m is beat m - 1.  The first beats of both warps are
// unrolled with compile-time counts of computing stages (ACT); the stage
// just past them only keeps its input row.  Every beat still ends with the
// pair barrier, so the two warps' barrier counts stay equal.
#pragma once

#include "temporal.cuh"

namespace rdk {

constexpr int kSplitPairs = 2;                 // warp pairs per block
constexpr int kSplitBlock = 64 * kSplitPairs;  // threads per block

__device__ __forceinline__ void pair_barrier(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

template <typename T> struct Handoff {
    typedef typename Vec<T>::type VT;
    VT (*slot)[2][32];  // [2 slots][field][lane]
};

// A lane's row in handoff slot `k` -> Slice (same layout as the input ring).
template <typename T>
__device__ __forceinline__ void hand_read(const Handoff<T> &h, int k, Slice<T> &s) {
    RowRing<T> view;
    view.slot = h.slot;  // two slots, indexed like ring slots 0 and 1
    ring_read(view, k, s);
}

// Producer beat: input row m from the ring through stages 1 .. K1; the stage-K1
// row (input-row index m - K1) goes to handoff slot m % 2.
template <typename T, int K1, int RX, int BC, int PH, int ACT = K1>
__device__ __forceinline__ void split_producer_beat(int m, int total, Slice<T> (&W)[3][K1],
                                                    const RowRing<T> &ring, const Handoff<T> &hand,
                                                    RowWalk<BC> &walk, int nn, int nm, int lc, bool rev,
                                                    const T *__restrict__ u, const T *__restrict__ v,
                                                    int bar_id, const Coef<T> &p) {
    constexpr int V = Vec<T>::N;
    typedef typename Vec<T>::type VT;
    if (m > total) return;  // beyond the last beat: no work and no barrier (same m for both warps)
    if (m < total) {
        if (m + kRing - 1 < total) {
            ring_issue(ring, m + kRing - 1, walk.g, nm, lc, u, v);
            walk.next(nn);
        }
        cp_async_commit();
        cp_async_wait<kRing - 1>();
        const int lane = threadIdx.x & 31;
        Slice<T> cur;
        ring_read_bc<T, BC>(ring, m % kRing, rev, cur);
#pragma unroll
        for (int s = 0; s < K1; ++s) {
            if (s < ACT) {
                Slice<T> &A = W[PH][s];
                Slice<T> &B = W[(PH + 1) % 3][s];
                const T wu = __shfl_up_sync(kFull, B.u[V - 1], 1);
                const T eu = __shfl_down_sync(kFull, B.u[0], 1);
                const T wv = __shfl_up_sync(kFull, B.v[V - 1], 1);
                const T ev = __shfl_down_sync(kFull, B.v[0], 1);
                Slice<T> out;
                slice_update<T, RX>(A, B, cur, wu, eu, wv, ev, p, out);
                W[(PH + 2) % 3][s] = cur;
                cur = out;
            } else if (s == ACT) {
                W[(PH + 2) % 3][s] = cur;
            }
        }
        VT a, b;
        if constexpr (V == 4) {
            a = make_float4(cur.u[0], cur.u[1], cur.u[2], cur.u[3]);
            b = make_float4(cur.v[0], cur.v[1], cur.v[2], cur.v[3]);
        } else {
            a = make_double2(cur.u[0], cur.u[1]);
            b = make_double2(cur.v[0], cur.v[1]);
        }
        hand.slot[m % 2][0][lane] = a;
        hand.slot[m % 2][1][lane] = b;
    }
    pair_barrier(bar_id);
}

// Consumer beat: the producer's row of beat m - 1 through stages K1+1 .. K; the
// final row (input-row index m - 1 - K) is stored when the strip owns it.
template <typename T, int K, int K2, int RX, int PH, int ACT = K2, bool KEEP = false>
__device__ __forceinline__ void split_consumer_beat(int m, int total, Slice<T> (&W)[3][K2],
                                                    const Handoff<T> &hand, const StripGeom &geo,
                                                    T *__restrict__ un, T *__restrict__ vn, int nm,
                                                    int bar_id, const Coef<T> &p) {
    constexpr int V = Vec<T>::N;
    if (m > total) return;
    if (m >= 1) {
        Slice<T> cur;
        hand_read(hand, (m - 1) % 2, cur);
#pragma unroll
        for (int s = 0; s < K2; ++s) {
            if (s < ACT) {
                Slice<T> &A = W[PH][s];
                Slice<T> &B = W[(PH + 1) % 3][s];
                const T wu = __shfl_up_sync(kFull, B.u[V - 1], 1);
                const T eu = __shfl_down_sync(kFull, B.u[0], 1);
                const T wv = __shfl_up_sync(kFull, B.v[V - 1], 1);
                const T ev = __shfl_down_sync(kFull, B.v[0], 1);
                Slice<T> out;
                slice_update<T, RX>(A, B, cur, wu, eu, wv, ev, p, out);
                W[(PH + 2) % 3][s] = cur;
                cur = out;
            } else if (KEEP && s == ACT) {
                W[(PH + 2) % 3][s] = cur;
            }
        }
        const int orow = m - 1 - 2 * K;  // negative throughout the fill
        if (orow >= 0 && geo.st_lane) {
            const int64_t off = (int64_t)(geo.r0 + orow) * nm + geo.sc;
            store_vec<T>(un + off, cur.u);
            store_vec<T>(vn + off, cur.v);
        }
    }
    pair_barrier(bar_id);
}

// Fill beats 0 .. F-1 of the producer: ACT = min(M / 2, K1).
template <typename T, int K1, int RX, int BC, int M, int F>
__device__ __forceinline__ void split_producer_fill(int total, Slice<T> (&W)[3][K1], const RowRing<T> &ring,
                                                    const Handoff<T> &hand, RowWalk<BC> &walk, int nn, int nm,
                                                    int lc, bool rev, const T *__restrict__ u,
                                                    const T *__restrict__ v, int bar_id, const Coef<T> &p) {
    split_producer_beat<T, K1, RX, BC, M % 3, (M / 2 < K1 ? M / 2 : K1)>(M, total, W, ring, hand, walk, nn, nm,
                                                                         lc, rev, u, v, bar_id, p);
    if constexpr (M + 1 < F)
        split_producer_fill<T, K1, RX, BC, M + 1, F>(total, W, ring, hand, walk, nn, nm, lc, rev, u, v, bar_id, p);
}

// Fill beats 0 .. F-1 of the consumer (equivalent beat M - 1): local stage j
// computes when M - 1 >= 2 (K1 + j) + 2; the next one keeps its input once
// the handoff row is valid (M - 1 >= 2 K1).
template <typename T, int K, int K2, int RX, int M, int F>
__device__ __forceinline__ void split_consumer_fill(int total, Slice<T> (&W)[3][K2], const Handoff<T> &hand,
                                                    const StripGeom &geo, T *__restrict__ un,
                                                    T *__restrict__ vn, int nm, int bar_id, const Coef<T> &p) {
    constexpr int K1 = K - K2;
    constexpr int D = (M >= 1 ? (M - 1) / 2 : -1) - K1;  // computing stages, before clamping
    constexpr int ACT = D < 0 ? 0 : (D > K2 ? K2 : D);
    split_consumer_beat<T, K, K2, RX, M % 3, ACT, (D >= 0)>(M, total, W, hand, geo, un, vn, nm, bar_id, p);
    if constexpr (M + 1 < F)
        split_consumer_fill<T, K, K2, RX, M + 1, F>(total, W, hand, geo, un, vn, nm, bar_id, p);
}

// One work item per warp pair; `item` is the same for both warps of a pair.
template <typename T, int K, int RX, int BC>
__device__ __forceinline__ void temporal_split_item(int item, int bands, const T *__restrict__ u,
                                                    const T *__restrict__ v, T *__restrict__ un,
                                                    T *__restrict__ vn, int nn, int nm, int rows,
                                                    const Coef<T> &p) {
    constexpr int K1 = K / 2;
    constexpr int K2 = K - K1;
    constexpr int H = (K + Vec<T>::N - 1) / Vec<T>::N;
    // fill beats: the consumer's last stage starts computing at beat 2K + 1;
    // whole 3-beat groups keep the window rotation's phase
    constexpr int kFill = 3 * ((2 * K + 4) / 3);
    typedef typename Vec<T>::type VT;
    __shared__ __align__(16) VT ring_mem[kSplitPairs][kRing][2][32];
    __shared__ __align__(16) VT hand_mem[kSplitPairs][2][2][32];
    const int warp = threadIdx.x >> 5;
    const int pair = warp >> 1;
    const int bar_id = 1 + pair;
    const StripGeom geo = strip_geom<T, K, H, BC>(item % bands, item / bands, nn, nm, rows);
    Handoff<T> hand;
    hand.slot = hand_mem[pair];
    if ((warp & 1) == 0) {
        Slice<T> W[3][K1];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int s = 0; s < K1; ++s) zero_slice(W[a][s]);
        RowRing<T> ring;
        ring.slot = ring_mem[pair];
        RowWalk<BC> walk;
        walk.start((int64_t)geo.r0 - K, nn);
#pragma unroll
        for (int j = 0; j < kRing - 1; ++j) {
            if (j < geo.total) {
                ring_issue(ring, j, walk.g, nm, geo.lc, u, v);
                walk.next(nn);
            }
            cp_async_commit();
        }
        split_producer_fill<T, K1, RX, BC, 0, kFill>(geo.total, W, ring, hand, walk, nn, nm, geo.lc, geo.rev, u, v,
                                                     bar_id, p);
        for (int m = kFill; m <= geo.total; m += 3) {
            split_producer_beat<T, K1, RX, BC, kFill % 3>(m, geo.total, W, ring, hand, walk, nn, nm, geo.lc, geo.rev,
                                                          u, v, bar_id, p);
            split_producer_beat<T, K1, RX, BC, (kFill + 1) % 3>(m + 1, geo.total, W, ring, hand, walk, nn, nm, geo.lc,
                                                                geo.rev, u, v, bar_id, p);
            split_producer_beat<T, K1, RX, BC, (kFill + 2) % 3>(m + 2, geo.total, W, ring, hand, walk, nn, nm, geo.lc,
                                                                geo.rev, u, v, bar_id, p);
        }
        cp_async_wait<0>();
    } else {
        Slice<T> W[3][K2];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int s = 0; s < K2; ++s) zero_slice(W[a][s]);
        split_consumer_fill<T, K, K2, RX, 0, kFill>(geo.total, W, hand, geo, un, vn, nm, bar_id, p);
        for (int m = kFill; m <= geo.total; m += 3) {
            split_consumer_beat<T, K, K2, RX, kFill % 3>(m, geo.total, W, hand, geo, un, vn, nm, bar_id, p);
            split_consumer_beat<T, K, K2, RX, (kFill + 1) % 3>(m + 1, geo.total, W, hand, geo, un, vn, nm, bar_id, p);
            split_consumer_beat<T, K, K2, RX, (kFill + 2) % 3>(m + 2, geo.total, W, hand, geo, un, vn, nm, bar_id, p);
        }
    }
}

}  // namespace rdk
