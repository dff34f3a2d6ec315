// temporal.cuh -- the K-step register pipeline shared by the single-grid and
// batched temporally blocked kernels (Eq. 1 applied K times per HBM pass).
//
// A warp owns one (band, strip) work item: output columns
// [band*OUTW, band*OUTW + OUTW) and output rows [strip*rows, strip*rows + rows)
// of an NN x NM torus.  It loads 32*V columns starting H*V columns to the left
// of its band (H = ceil(K/V) halo lanes per side, indices wrapped modulo NM)
// and input rows r0-K .. r0+rows+K-1 (wrapped modulo NN).  Input rows are
// staged through a per-warp shared-memory ring by cp.async, kRing - 1 rows
// ahead of use.  Each input row passes through K stages held in registers;
// stage s turns rows (q-1, q, q+1)
// of stage s-1 into row q of stage s.  After K stages the K outermost columns
// on each side are stale, which is why only lanes H .. 31-H store.
//
// Zero-flux boundary (BC_MIRROR): the halo rows and columns beyond a grid
// edge are loaded as the mirror image of the rows and columns inside it
// (row -1 <- row 0, row -2 <- row 1, ...; a lane whose 16-byte vector lies
// beyond an edge loads the mirrored vector and reverses its elements).  The
// 2N x 2M torus holding that mirror image evolves exactly like the zero-flux
// grid (the edge faces are mirror planes and the update keeps a mirrored
// state mirrored), so every stage sees the edge cell as its own outside
// neighbour with no per-stage test; only the input indexing differs.  Sums
// of mirrored pairs are formed in swapped order, which IEEE addition does not
// notice: the results are the bits the single-step kernel computes.
#pragma once

#include "common.cuh"

namespace rdk {

// Warps per block of every kernel built on temporal_strip.  One: the same
// resident warps per SM issue faster as one-warp blocks (K = 8 at 4096^2:
// 1436 against 1278 Gcell-updates/s with four-warp blocks and 1270 with
// two; ncu shows the dispatch stalls per issued instruction falling from
// 0.44 to 0.18 and issue-active rising from 63 % to 72 % at the same 8
// warps per SM and the same instructions).
constexpr int kTemporalWarps = 1;
// Input rows staged per warp (prefetch distance kRing - 1 = 2 beats, about
// 1.5 us of the K = 8 pipeline, above the HBM latency).  Three slots match
// the 3-beat window rotation, so a beat's slots are compile-time constants.
constexpr int kRing = 3;

// Per-lane 16-byte asynchronous global -> shared copy (cp.async, L2 only).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// 8-byte variant (16-bit storage: 4 values per lane); cp.async.cg takes 16 only.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory ring of one warp: kRing rows x {u, v} x 32 lanes x 16 bytes.
// Each lane copies and later reads back only its own 16 bytes, so the lane's
// own cp.async.wait_group is the only synchronisation needed.
template <typename T> struct RowRing {
    typedef typename Vec<T>::type VT;
    VT (*slot)[2][32];  // [kRing][field][lane]
};

template <typename T>
__device__ __forceinline__ void ring_issue_at(const RowRing<T> &r, int slot, int g, int nm, int lc,
                                              const T *__restrict__ u, const T *__restrict__ v) {
    const int lane = threadIdx.x & 31;
    const int64_t off = (int64_t)g * nm + lc;
    if constexpr (sizeof(typename Vec<T>::type) == 32) {  // two 16-byte halves per field
        char *su = reinterpret_cast<char *>(&r.slot[slot][0][lane]);
        char *sv = reinterpret_cast<char *>(&r.slot[slot][1][lane]);
        cp_async16(su, u + off);
        cp_async16(su + 16, reinterpret_cast<const char *>(u + off) + 16);
        cp_async16(sv, v + off);
        cp_async16(sv + 16, reinterpret_cast<const char *>(v + off) + 16);
    } else if constexpr (sizeof(typename Vec<T>::type) == 16) {
        cp_async16(&r.slot[slot][0][lane], u + off);
        cp_async16(&r.slot[slot][1][lane], v + off);
    } else {
        cp_async8(&r.slot[slot][0][lane], u + off);
        cp_async8(&r.slot[slot][1][lane], v + off);
    }
}

// Input row m goes to slot m % kRing.
template <typename T>
__device__ __forceinline__ void ring_issue(const RowRing<T> &r, int m, int g, int nm, int lc,
                                           const T *__restrict__ u, const T *__restrict__ v) {
    ring_issue_at(r, m % kRing, g, nm, lc, u, v);
}

template <typename T>
__device__ __forceinline__ void ring_read_at(const RowRing<T> &r, int slot, Slice<CT<T>, Vec<T>::N> &s) {
    typedef typename Vec<T>::type VT;
    const int lane = threadIdx.x & 31;
    const VT a = r.slot[slot][0][lane];
    const VT b = r.slot[slot][1][lane];
    unpack_vec<T, Vec<T>::N>(a, s.u);
    unpack_vec<T, Vec<T>::N>(b, s.v);
}

template <typename T>
__device__ __forceinline__ void ring_read(const RowRing<T> &r, int m, Slice<CT<T>, Vec<T>::N> &s) {
    ring_read_at(r, m % kRing, s);
}

// ring_read for boundary BC; under BC_MIRROR a lane whose columns lie beyond
// an edge (rev) reverses the element order of the mirrored vector it loaded.
template <typename T, int BC>
__device__ __forceinline__ void ring_read_bc(const RowRing<T> &r, int slot, bool rev, Slice<CT<T>, Vec<T>::N> &s) {
    ring_read_at(r, slot, s);
    if constexpr (BC == BC_MIRROR) {
        constexpr int V = Vec<T>::N;
        Slice<CT<T>, Vec<T>::N> t = s;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            s.u[e] = rev ? t.u[V - 1 - e] : t.u[e];
            s.v[e] = rev ? t.v[V - 1 - e] : t.v[e];
        }
    }
}

// Source row of the strip's input rows, advanced one row per beat: wrapped
// on the torus; under zero flux the reflected sequence (..., 1, 0, 0, 1, ...
// at the top edge, ..., n-2, n-1, n-1, n-2, ... at the bottom).
template <int BC> struct RowWalk {
    int g = 0, dir = 1;
    __device__ __forceinline__ void start(int64_t r, int n) {
        if constexpr (BC == BC_MIRROR) {
            const int q = wrap_row(r, 2 * (int64_t)n);
            g = q < n ? q : 2 * n - 1 - q;
            dir = q < n ? 1 : -1;
        } else {
            g = wrap_row(r, n);
        }
    }
    __device__ __forceinline__ void next(int n) {
        if constexpr (BC == BC_MIRROR) {
            if (dir > 0) {
                if (g == n - 1) dir = -1; else ++g;
            } else {
                if (g == 0) dir = 1; else --g;
            }
        } else {
            g = (g + 1 == n) ? 0 : g + 1;
        }
    }
};

// One pipeline beat: take input row m of the strip from the ring (issuing the
// copy of row m + kRing - 1 first), advance every stage by one row, and hand
// the finished row (stage K) to the policy.  W[PH], W[PH+1] hold the two older
// rows of each stage, W[PH+2] receives the newest, so a 3-beat unroll rotates
// the windows without register moves.
//
// The policy P supplies the per-stage arithmetic and the stores:
//   P::issue(j)                          extra cp.async copies for beat j,
//                                        committed with input row j
//   P::begin_beat(m)                     before the stages of beat m
//   P::stage<s>(A, B, C, wu, eu, wv, ev, q, out)
//        stage s maps rows q-1 (A), q (B), q+1 (C) of its input to row q of
//        its output (q = input-row index within the strip, see temporal_strip)
//   P::finish(q, out)                    the row q leaving the last stage
//   P::finish_main(q, out)               the same for a beat of the main loop,
//                                        where q >= K holds: the owned row
//                                        check may be dropped
//
// CHECK = false: a beat of the main loop's whole triplets (m + 2 < total),
// which needs neither the end-of-strip test nor the last-copy test (measured
// at K = 8, 4096^2: 1427 -> 1448 Gcell-updates/s).
//
// ACTIVE < K (the first 2K beats of a strip with a policy that allows it):
// only stages s < ACTIVE compute; stage ACTIVE just keeps its input row for
// the next beats.  Row q of the last stage needs stage s's rows from
// q - (K - 1 - s) on, and the stored rows have q >= K, so stage s's rows
// 0 .. s feed nothing that is stored.  Beat m computes stage s's row
// m - s - 1, so stage s first matters at beat 2s + 2: ACTIVE = m / 2.
template <typename T, int K, int PH, int BC, int ACTIVE = K, bool CHECK = true, class P>
__device__ __forceinline__ void pipeline_beat(int m, int total, Slice<CT<T>, Vec<T>::N> (&W)[3][K],
                                              const RowRing<T> &ring, RowWalk<BC> &walk, int nn, int nm,
                                              int lc, bool rev, const T *__restrict__ u,
                                              const T *__restrict__ v, P &pol) {
    constexpr int V = Vec<T>::N;
    if (CHECK && m >= total) return;
    // The slot written here was read in the previous beat, whose stage
    // computations (issued before this point) consumed that value.
    static_assert(kRing == 3, "slots follow the 3-beat phase: row m sits in slot m % 3 == PH");
    if (!CHECK || m + kRing - 1 < total) {
        ring_issue_at(ring, (PH + kRing - 1) % kRing, walk.g, nm, lc, u, v);
        walk.next(nn);
        pol.issue(m + kRing - 1);
    }
    cp_async_commit();
    cp_async_wait<kRing - 1>();  // the group holding row m is complete
    Slice<CT<T>, Vec<T>::N> cur;
    ring_read_bc<T, BC>(ring, PH, rev, cur);
    pol.begin_beat(m);
#pragma unroll
    for (int s = 0; s < K; ++s) {
        if (s < ACTIVE) {
            Slice<CT<T>, Vec<T>::N> &A = W[PH][s];
            Slice<CT<T>, Vec<T>::N> &B = W[(PH + 1) % 3][s];
            const CT<T> wu = __shfl_up_sync(kFull, B.u[V - 1], 1);
            const CT<T> eu = __shfl_down_sync(kFull, B.u[0], 1);
            const CT<T> wv = __shfl_up_sync(kFull, B.v[V - 1], 1);
            const CT<T> ev = __shfl_down_sync(kFull, B.v[0], 1);
            Slice<CT<T>, Vec<T>::N> out;
            pol.stage(s, A, B, cur, wu, eu, wv, ev, m - s - 1, out);
            W[(PH + 2) % 3][s] = cur;
            cur = out;
        } else if (s == ACTIVE) {
            W[(PH + 2) % 3][s] = cur;  // stage s - 1's row, needed from the next beat on
        }
    }
    if constexpr (ACTIVE == K) {
        if constexpr (CHECK) pol.finish(m - K, cur);
        else pol.finish_main(m - K, cur);
    }
}

// The first 2K beats of a strip (ACTIVE = M / 2), unrolled at compile time.
template <typename T, int K, int BC, int M, class P>
__device__ __forceinline__ void pipeline_fill(int total, Slice<CT<T>, Vec<T>::N> (&W)[3][K],
                                              const RowRing<T> &ring, RowWalk<BC> &walk, int nn, int nm,
                                              int lc, bool rev, const T *__restrict__ u,
                                              const T *__restrict__ v, P &pol) {
    pipeline_beat<T, K, M % 3, BC, (M / 2 < K ? M / 2 : K)>(M, total, W, ring, walk, nn, nm, lc, rev, u, v, pol);
    if constexpr (M + 1 < 2 * K)
        pipeline_fill<T, K, BC, M + 1>(total, W, ring, walk, nn, nm, lc, rev, u, v, pol);
}

// Geometry of one (band, strip) work item for depth K and halo H.
// Input-row index q in 0 .. nout + 2K - 1 is global row r0 - K + q (wrapped,
// or reflected under zero flux); the strip owns rows q in [K, K + nout) and
// lanes H .. 31-H whose column sc = c0 + (lane - H) V is below NM.  lc is the
// first column the lane loads; rev marks a mirrored (reversed) vector.
struct StripGeom {
    int lc, sc, r0, nout, total;
    bool st_lane, rev;
};

template <typename T, int K, int H, int BC = BC_WRAP>
__device__ __forceinline__ StripGeom strip_geom(int band, int strip, int nn, int nm, int rows) {
    constexpr int V = Vec<T>::N;
    static_assert(H * V >= K, "halo narrower than the temporal depth");
    static_assert(2 * H < 32, "halo wider than the warp");
    constexpr int OUTW = (32 - 2 * H) * V;
    const int lane = threadIdx.x & 31;
    StripGeom g;
    const int c0 = band * OUTW;
    const int64_t c = (int64_t)c0 - H * V + lane * V;
    g.rev = false;
    if constexpr (BC == BC_MIRROR) {
        // columns c .. c+V-1 of the 2NM-periodic mirror image: inside the
        // grid, or the reversed vector starting at 2NM - V - q (V-aligned)
        const int q = wrap_row(c, 2 * (int64_t)nm);
        g.rev = q >= nm;
        g.lc = g.rev ? 2 * nm - V - q : q;
    } else {
        g.lc = wrap_row(c, nm);  // V-aligned since nm % V == 0
    }
    g.sc = c0 + (lane - H) * V;
    g.st_lane = (lane >= H) && (lane < 32 - H) && (g.sc < nm);
    g.r0 = strip * rows;
    g.nout = min(rows, nn - g.r0);
    g.total = g.nout + 2 * K;
    return g;
}

// Run one work item through the K-stage pipeline: input rows of (u, v) pass
// through the stages; the policy decides what each stage computes and stores.
template <typename T, int K, int BC = BC_WRAP, class P>
__device__ __forceinline__ void pipeline_strip(const StripGeom &geo, const T *__restrict__ u,
                                               const T *__restrict__ v, int nn, int nm, P &pol) {
    Slice<CT<T>, Vec<T>::N> W[3][K];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int s = 0; s < K; ++s) zero_slice(W[a][s]);

    typedef typename Vec<T>::type VT;
    __shared__ __align__(16) VT ring_mem[kTemporalWarps][kRing][2][32];
    RowRing<T> ring;
    ring.slot = ring_mem[(threadIdx.x >> 5) % kTemporalWarps];

    // prologue: rows 0 .. kRing-2 in flight, one commit group each
    RowWalk<BC> walk;
    walk.start((int64_t)geo.r0 - K, nn);
#pragma unroll
    for (int j = 0; j < kRing - 1; ++j) {
        if (j < geo.total) {
            ring_issue(ring, j, walk.g, nm, geo.lc, u, v);
            walk.next(nn);
            pol.issue(j);
        }
        cp_async_commit();
    }
    // a strip has total = nout + 2K > 2K beats, so the fill always completes
    constexpr int M0 = P::kLightCone ? 2 * K : 0;
    if constexpr (P::kLightCone)
        pipeline_fill<T, K, BC, 0>(geo.total, W, ring, walk, nn, nm, geo.lc, geo.rev, u, v, pol);
    int m = M0;
    for (; m + 2 < geo.total; m += 3) {  // whole triplets: no per-beat bounds tests
        pipeline_beat<T, K, M0 % 3, BC, K, false>(m, geo.total, W, ring, walk, nn, nm, geo.lc, geo.rev, u, v, pol);
        pipeline_beat<T, K, (M0 + 1) % 3, BC, K, false>(m + 1, geo.total, W, ring, walk, nn, nm, geo.lc, geo.rev, u, v,
                                                         pol);
        pipeline_beat<T, K, (M0 + 2) % 3, BC, K, false>(m + 2, geo.total, W, ring, walk, nn, nm, geo.lc, geo.rev, u, v,
                                                         pol);
    }
    // the last 0 .. 2 beats
    pipeline_beat<T, K, M0 % 3>(m, geo.total, W, ring, walk, nn, nm, geo.lc, geo.rev, u, v, pol);
    pipeline_beat<T, K, (M0 + 1) % 3>(m + 1, geo.total, W, ring, walk, nn, nm, geo.lc, geo.rev, u, v, pol);
    cp_async_wait<0>();
}

// Forward policy: Eq. 1 at every stage; the last stage's owned rows are stored.
// Only owned rows are stored, so the fill may skip the stages outside their
// light cone (kLightCone).
template <typename T, int K, int RX>
struct ForwardPolicy {
    static constexpr bool kLightCone = true;
    const Coef<CT<T>> &p;
    const StripGeom &geo;
    T *__restrict__ un;
    T *__restrict__ vn;
    int nm;
    __device__ __forceinline__ void issue(int) {}
    __device__ __forceinline__ void begin_beat(int) {}
    __device__ __forceinline__ void stage(int, const Slice<CT<T>, Vec<T>::N> &A, const Slice<CT<T>, Vec<T>::N> &B, const Slice<CT<T>, Vec<T>::N> &C,
                                          CT<T> wu, CT<T> eu, CT<T> wv, CT<T> ev, int, Slice<CT<T>, Vec<T>::N> &out) {
        slice_update<CT<T>, RX, Vec<T>::N>(A, B, C, wu, eu, wv, ev, p, out);
    }
    __device__ __forceinline__ void finish(int q, const Slice<CT<T>, Vec<T>::N> &out) {
        const int orow = q - K;
        if (orow >= 0) {  // the same for the whole warp
            const int64_t off = (int64_t)(geo.r0 + orow) * nm + geo.sc;
            if (geo.st_lane) {
                store_vec<T>(un + off, out.u);
                store_vec<T>(vn + off, out.v);
            }
        }
    }
    __device__ __forceinline__ void finish_main(int q, const Slice<CT<T>, Vec<T>::N> &out) {
        const int64_t off = (int64_t)(geo.r0 + q - K) * nm + geo.sc;
        if (geo.st_lane) {
            store_vec<T>(un + off, out.u);
            store_vec<T>(vn + off, out.v);
        }
    }
};

// Planes of the K intermediate states written by ForwardAllPolicy.
template <typename T> struct StagePlanes {
    T *u[8];
    T *v[8];
};

// Forward policy that also stores the owned rows of every stage s (the state
// s+1 steps ahead) into planes.u[s], planes.v[s]: the states a reverse sweep
// needs, K per launch.
template <typename T, int K, int RX>
struct ForwardAllPolicy {
    static constexpr bool kLightCone = true;  // stores owned rows only (q >= K)
    const Coef<CT<T>> &p;
    const StripGeom &geo;
    const StagePlanes<T> &planes;
    int nm;
    __device__ __forceinline__ void issue(int) {}
    __device__ __forceinline__ void begin_beat(int) {}
    __device__ __forceinline__ void stage(int s, const Slice<CT<T>, Vec<T>::N> &A, const Slice<CT<T>, Vec<T>::N> &B, const Slice<CT<T>, Vec<T>::N> &C,
                                          CT<T> wu, CT<T> eu, CT<T> wv, CT<T> ev, int q, Slice<CT<T>, Vec<T>::N> &out) {
        slice_update<CT<T>, RX, Vec<T>::N>(A, B, C, wu, eu, wv, ev, p, out);
        const int orow = q - K;
        if (orow >= 0 && orow < geo.nout && geo.st_lane) {
            const int64_t off = (int64_t)(geo.r0 + orow) * nm + geo.sc;
            store_vec<T>(planes.u[s] + off, out.u);
            store_vec<T>(planes.v[s] + off, out.v);
        }
    }
    __device__ __forceinline__ void finish(int, const Slice<CT<T>, Vec<T>::N> &) {}
    __device__ __forceinline__ void finish_main(int, const Slice<CT<T>, Vec<T>::N> &) {}
};

// H = halo lanes per side; any H >= ceil(K/V) is correct (a larger H than
// needed only narrows the band), which lets a batched launch use one band
// layout for launches of different depth.
template <typename T, int K, int H, int RX, int BC = BC_WRAP>
__device__ __forceinline__ void temporal_strip(int band, int strip, const T *__restrict__ u,
                                               const T *__restrict__ v, T *__restrict__ un,
                                               T *__restrict__ vn, int nn, int nm, int rows,
                                               const Coef<CT<T>> &p) {
    const StripGeom geo = strip_geom<T, K, H, BC>(band, strip, nn, nm, rows);
    ForwardPolicy<T, K, RX> pol{p, geo, un, vn, nm};
    pipeline_strip<T, K, BC>(geo, u, v, nn, nm, pol);
}

constexpr int kTemporalBlock = 32 * kTemporalWarps;

// The single-grid temporally blocked kernel: warp w of the launch owns work
// item (band w % bands, strip w / bands).
template <typename T, int K, int RX, int BC>
__global__ void __launch_bounds__(kTemporalBlock)
k_temporal(const T *__restrict__ u, const T *__restrict__ v, T *__restrict__ un,
           T *__restrict__ vn, int nn, int nm, int bands, int nwarps, int rows, Coef<CT<T>> p) {
    pdl_wait();
    const int wid = blockIdx.x * (kTemporalBlock / 32) + (threadIdx.x >> 5);
    if (wid >= nwarps) return;  // whole warps only
    constexpr int H = (K + Vec<T>::N - 1) / Vec<T>::N;
    temporal_strip<T, K, H, RX, BC>(wid % bands, wid / bands, u, v, un, vn, nn, nm, rows, p);
    pdl_trigger();
}

}  // namespace rdk
