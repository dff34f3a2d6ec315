// adjoint.cu -- reverse-time (discrete adjoint) sweep of Eq. 1-3.
//
// Not in the paper: it differentiates the update of Sec. II.A exactly.  For
// one step (u+, v+) = F(u, v) and co-state (lu, lv) = dL/d(u+, v+):
//   dL/du = lu + dt [ (c - u^2) lu - eps lv + Du Lap(lu) ]
//   dL/dv = lv + dt [ -lu + eps b lv + Dv Lap(lv) ]
// (the periodic 5-point Laplacian is symmetric, so it is its own transpose),
// and the gene picks up, per step,
//   dL/dDu += dt sum lu Lap(u)     dL/dDv += dt sum lv Lap(v)
//   dL/dc  += dt sum lu u          dL/da  += dt sum lv (-eps)
//   dL/db  += dt sum lv eps v      dL/deps += dt sum lv (-(u - b v + a))
// with (u, v) the state before the step.
//
// Driver: forward sweep storing n_ck checkpoints (every S = ceil(T/n_ck)
// steps), then segments in reverse: rebuild the S states of the segment with
// single-step launches, then walk them backwards with k_adjoint_step.  Each
// warp of k_adjoint_step owns the same cells at every step and adds its FP64
// partial sums to its own slot, so the gradient is deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace rdk {

namespace {

constexpr int kAdjBlock = 256;

// Coefficients of the reverse step, arranged like the forward cell update
// (the -4 centre weight folded in): cm4 = c - 4 Du, ebm4 = eps b - 4 Dv;
// with no reaction cm4 = -4 Du, ebm4 = -4 Dv and the rest is unused.
// a, b, eps (FP64) enter only the gradient sums.
template <typename T> struct AdjCoef {
    T dt, Du, Dv, cm4, meps, ebm4;
    double a, b, eps;
};

template <typename T>
AdjCoef<T> make_adj_coef(const rdcnn_params &p, int reaction) {
    const bool fhn = (reaction == RDCNN_REACTION_FHN);
    AdjCoef<T> q;
    q.dt = T(p.dt); q.Du = T(p.Du); q.Dv = T(p.Dv);
    q.cm4 = T((fhn ? p.c : 0.0) - 4.0 * p.Du);
    q.meps = T(fhn ? -p.eps : 0.0);
    q.ebm4 = T((fhn ? p.eps * p.b : 0.0) - 4.0 * p.Dv);
    q.a = p.a; q.b = p.b; q.eps = p.eps;
    return q;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// One reverse step for a (band, strip) of rows.  The co-state (lu, lv) is
// streamed with a 3-row window plus one prefetched row (Slice<T>.u = lu,
// .v = lv); the state (u, v) at the same time level is needed only at the
// centre cell.  The Du / Dv gradient terms use the symmetry of the periodic
// Laplacian, sum_k lu_k Lap(u)_k = sum_k u_k Lap(lu)_k, so they reuse the
// co-state neighbour sums the update forms anyway.  Per-row sums of the six
// gene terms are formed in T and accumulated in FP64.
template <typename T, int RX>
__global__ void __launch_bounds__(kAdjBlock)
k_adjoint_step(const T *__restrict__ u, const T *__restrict__ v, const T *__restrict__ lu,
               const T *__restrict__ lv, T *__restrict__ lun, T *__restrict__ lvn,
               double *__restrict__ partial, int nn, int nm, int bands, int nwarps, int rows,
               AdjCoef<T> p) {
    constexpr int V = Vec<T>::N;
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * (kAdjBlock / 32) + (threadIdx.x >> 5);
    if (wid >= nwarps) return;
    const int band = wid % bands;
    const int strip = wid / bands;
    const int col = band * 32 * V + lane * V;
    const bool active = col < nm;
    const int colw = (col == 0) ? nm - 1 : col - 1;
    const int cole = (col + V >= nm) ? 0 : col + V;
    const bool edge_w = (lane == 0);
    const bool edge_e = active && (lane == 31 || col + V >= nm);
    const int r0 = strip * rows;
    const int r1 = min(r0 + rows, nn);

    Slice<T> nor, cen, sou, pre, st, st_pre;  // co-state rows r-1, r, r+1, r+2; state rows r, r+1
    zero_slice(nor); zero_slice(cen); zero_slice(sou); zero_slice(pre); zero_slice(st); zero_slice(st_pre);
    T cw_u = 0, ce_u = 0, cw_v = 0, ce_v = 0, sw_u = 0, se_u = 0, sw_v = 0, se_v = 0;
    T pw_u = 0, pe_u = 0, pw_v = 0, pe_v = 0;
    const int rn = (r0 == 0) ? nn - 1 : r0 - 1;
    int rs = (r0 + 1 == nn) ? 0 : r0 + 1;
    if (active) {
        load_slice(nor, lu, lv, (int64_t)rn * nm + col);
        load_slice(cen, lu, lv, (int64_t)r0 * nm + col);
        load_slice(sou, lu, lv, (int64_t)rs * nm + col);
        load_slice(st, u, v, (int64_t)r0 * nm + col);
    }
    if (edge_w) {
        cw_u = __ldg(lu + (int64_t)r0 * nm + colw); cw_v = __ldg(lv + (int64_t)r0 * nm + colw);
        sw_u = __ldg(lu + (int64_t)rs * nm + colw); sw_v = __ldg(lv + (int64_t)rs * nm + colw);
    }
    if (edge_e) {
        ce_u = __ldg(lu + (int64_t)r0 * nm + cole); ce_v = __ldg(lv + (int64_t)r0 * nm + cole);
        se_u = __ldg(lu + (int64_t)rs * nm + cole); se_v = __ldg(lv + (int64_t)rs * nm + cole);
    }
    double g[6] = {0, 0, 0, 0, 0, 0};
    for (int r = r0; r < r1; ++r) {
        const bool more = (r + 1 < r1);
        const int rp = (rs + 1 == nn) ? 0 : rs + 1;
        if (more) {
            if (active) {
                load_slice(pre, lu, lv, (int64_t)rp * nm + col);
                load_slice(st_pre, u, v, (int64_t)rs * nm + col);
            }
            if (edge_w) { pw_u = __ldg(lu + (int64_t)rp * nm + colw); pw_v = __ldg(lv + (int64_t)rp * nm + colw); }
            if (edge_e) { pe_u = __ldg(lu + (int64_t)rp * nm + cole); pe_v = __ldg(lv + (int64_t)rp * nm + cole); }
        }
        T wu = __shfl_up_sync(kFull, cen.u[V - 1], 1);
        T eu = __shfl_down_sync(kFull, cen.u[0], 1);
        T wv = __shfl_up_sync(kFull, cen.v[V - 1], 1);
        T ev = __shfl_down_sync(kFull, cen.v[0], 1);
        if (edge_w) { wu = cw_u; wv = cw_v; }
        if (edge_e) { eu = ce_u; ev = ce_v; }
        T ou[V], ov[V];
        T rg[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const T luc = cen.u[e], lvc = cen.v[e];
            const T su = add_rn(add_rn(nor.u[e], sou.u[e]), add_rn(e == 0 ? wu : cen.u[e - 1],
                                                                   e == V - 1 ? eu : cen.u[e + 1]));
            const T sv = add_rn(add_rn(nor.v[e], sou.v[e]), add_rn(e == 0 ? wv : cen.v[e - 1],
                                                                   e == V - 1 ? ev : cen.v[e + 1]));
            const T uc = st.u[e], vc = st.v[e];
            // co-state update with the centre term folded in, like the forward:
            //   lu + dt [ Du s(lu) + (c - 4 Du - u^2) lu - eps lv ]
            //   lv + dt [ Dv s(lv) + (eps b - 4 Dv) lv - lu ]
            T ru, rv;
            if (RX == RX_FHN) {
                ru = fma_rn(fma_rn(-uc, uc, p.cm4), luc, mul_rn(p.meps, lvc));
                rv = fma_rn(p.ebm4, lvc, -luc);
            } else {
                ru = mul_rn(p.cm4, luc);
                rv = mul_rn(p.ebm4, lvc);
            }
            ou[e] = fma_rn(p.dt, fma_rn(p.Du, su, ru), luc);
            ov[e] = fma_rn(p.dt, fma_rn(p.Dv, sv, rv), lvc);
            rg[0] = fma_rn(uc, fma_rn(T(-4), luc, su), rg[0]);     // u Lap(lu)
            rg[1] = fma_rn(vc, fma_rn(T(-4), lvc, sv), rg[1]);     // v Lap(lv)
            if (RX == RX_FHN) {
                rg[2] = add_rn(rg[2], lvc);                        // lv        (x -eps)
                rg[3] = fma_rn(lvc, vc, rg[3]);                    // lv v      (x eps)
                rg[4] = fma_rn(lvc, fma_rn(T(-p.b), vc, uc), rg[4]);  // lv (u - b v)
                rg[5] = fma_rn(luc, uc, rg[5]);                    // lu u
            }
        }
        if (active) {
            const int64_t off = (int64_t)r * nm + col;
            store_vec<T>(lun + off, ou);
            store_vec<T>(lvn + off, ov);
            g[0] += (double)rg[0];
            g[1] += (double)rg[1];
            if (RX == RX_FHN) {
                g[2] -= p.eps * (double)rg[2];
                g[3] += p.eps * (double)rg[3];
                g[4] -= (double)rg[4] + p.a * (double)rg[2];
                g[5] += (double)rg[5];
            }
        }
        nor = cen; cen = sou; sou = pre; st = st_pre;
        cw_u = sw_u; ce_u = se_u; cw_v = sw_v; ce_v = se_v;
        sw_u = pw_u; se_u = pe_u; sw_v = pw_v; se_v = pe_v;
        rs = rp;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const double s = warp_sum(g[q]);
        if (lane == 0) partial[(int64_t)wid * 6 + q] += s;
    }
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

// Rows per warp: enough warps to fill the GPU (~2048), at most 16 rows.
int adj_rows(int64_t nn, int bands) {
    const int64_t r = nn * bands / 2048;
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, r));
}

struct AdjShape {
    int bands, strips, nwarps, rows;
};

AdjShape adj_shape(int dtype, int64_t nn, int64_t nm) {
    AdjShape s;
    const int V = vec_width(dtype);
    s.bands = (int)((nm + 32 * V - 1) / (32 * V));
    s.rows = adj_rows(nn, s.bands);
    s.strips = (int)((nn + s.rows - 1) / s.rows);
    s.nwarps = s.bands * s.strips;
    return s;
}

template <typename T>
cudaError_t adjoint_step_t(int reaction, const void *u, const void *v, const void *lu,
                           const void *lv, void *lun, void *lvn, double *partial, int64_t nn,
                           int64_t nm, const rdcnn_params &p, const AdjShape &sh, cudaStream_t s) {
    const int wpb = kAdjBlock / 32;
    const unsigned grid = (unsigned)((sh.nwarps + wpb - 1) / wpb);
    const AdjCoef<T> c = make_adj_coef<T>(p, reaction);
    if (reaction == RDCNN_REACTION_FHN)
        k_adjoint_step<T, RX_FHN><<<grid, kAdjBlock, 0, s>>>(
            (const T *)u, (const T *)v, (const T *)lu, (const T *)lv, (T *)lun, (T *)lvn, partial,
            (int)nn, (int)nm, sh.bands, sh.nwarps, sh.rows, c);
    else
        k_adjoint_step<T, RX_NONE><<<grid, kAdjBlock, 0, s>>>(
            (const T *)u, (const T *)v, (const T *)lu, (const T *)lv, (T *)lun, (T *)lvn, partial,
            (int)nn, (int)nm, sh.bands, sh.nwarps, sh.rows, c);
    count_launches(1);
    return cudaGetLastError();
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
    const AdjShape sh = adj_shape(dtype, nn, nm);
    L.ck_off = 0;
    L.seg_off = L.ck_off + (size_t)L.nseg * 2 * L.plane;
    L.lam_off = L.seg_off + (size_t)L.nslots * 2 * L.plane;
    L.part_off = L.lam_off + 4 * L.plane;
    L.out_off = L.part_off + (((size_t)sh.nwarps * 6 * sizeof(double) + 255) & ~(size_t)255);
    L.total = L.out_off + 256;
    return L;
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
    *bytes = adj_layout(dtype, nn, nm, T, n_checkpoints).total;
    return RDCNN_OK;
}

int rdcnn_adjoint(rdcnn_t *h, int64_t T, const void *u0, const void *v0, const void *dLdu_T,
                  const void *dLdv_T, int64_t n_checkpoints, void *dLdu0, void *dLdv0,
                  double grad[6], void *workspace, size_t workspace_bytes) {
    int64_t nn, nm; rdcnn_params p; int dtype, reaction; cudaStream_t s;
    int rc = handle_view(h, &nn, &nm, &p, &dtype, &reaction, &s);
    if (rc < 0) return rc;
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
    const size_t bytes = (size_t)nn * nm * elem_size(dtype);
    char *ws = (char *)workspace;
    auto ck_u = [&](int64_t i) { return (void *)(ws + L.ck_off + (size_t)(2 * i) * L.plane); };
    auto ck_v = [&](int64_t i) { return (void *)(ws + L.ck_off + (size_t)(2 * i + 1) * L.plane); };
    auto seg_u = [&](int64_t i) { return (void *)(ws + L.seg_off + (size_t)(2 * i) * L.plane); };
    auto seg_v = [&](int64_t i) { return (void *)(ws + L.seg_off + (size_t)(2 * i + 1) * L.plane); };
    void *lam_u[2] = {ws + L.lam_off, ws + L.lam_off + 2 * L.plane};
    void *lam_v[2] = {ws + L.lam_off + L.plane, ws + L.lam_off + 3 * L.plane};
    double *partial = (double *)(ws + L.part_off);
    double *gout = (double *)(ws + L.out_off);
    const AdjShape sh = adj_shape(dtype, nn, nm);
    const int k = default_k(dtype, nn, nm);
    const int rows_t = 0;  // chosen by the launcher
    const int rows_1 = default_rows_step1(dtype, nn, nm);

    cudaError_t e = cudaMemcpyAsync(lam_u[0], dLdu_T, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lam_v[0], dLdv_T, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ck_u(0), u0, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ck_v(0), v0, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(partial, 0, (size_t)sh.nwarps * 6 * sizeof(double), s);
    if (e != cudaSuccess) return cuda_error(e, "adjoint setup copies");

    // forward sweep: checkpoint i = state at step i*S
    for (int64_t i = 0; i + 1 < L.nseg && T > 0; ++i) {
        const int64_t len = L.S;
        const int64_t nl = (len + k - 1) / k;
        const void *cu = ck_u(i), *cv = ck_v(i);
        for (int64_t j = 0; j < nl; ++j) {
            const int kk = (int)std::min<int64_t>(k, len - j * k);
            void *nu = (j == nl - 1) ? ck_u(i + 1) : seg_u(j % 2);
            void *nv = (j == nl - 1) ? ck_v(i + 1) : seg_v(j % 2);
            e = launch_temporal(dtype, reaction, kk, cu, cv, nu, nv, nn, nm, p, rows_t, s);
            if (e != cudaSuccess) return cuda_error(e, "adjoint forward sweep");
            cu = nu; cv = nv;
        }
    }
    // reverse sweep over segments
    int cur = 0;
    for (int64_t sg = L.nseg - 1; sg >= 0 && T > 0; --sg) {
        const int64_t t0 = sg * L.S;
        const int64_t len = std::min<int64_t>(L.S, T - t0);
        for (int64_t q = 1; q < len; ++q) {
            const void *pu = (q == 1) ? ck_u(sg) : seg_u(q - 1);
            const void *pv = (q == 1) ? ck_v(sg) : seg_v(q - 1);
            e = launch_step1(dtype, reaction, pu, pv, seg_u(q), seg_v(q), nn, nm, p, rows_1, s);
            if (e != cudaSuccess) return cuda_error(e, "adjoint recompute");
        }
        for (int64_t q = len - 1; q >= 0; --q) {
            const void *su = (q == 0) ? ck_u(sg) : seg_u(q);
            const void *sv = (q == 0) ? ck_v(sg) : seg_v(q);
            if (dtype == RDCNN_F64)
                e = adjoint_step_t<double>(reaction, su, sv, lam_u[cur], lam_v[cur], lam_u[cur ^ 1],
                                           lam_v[cur ^ 1], partial, nn, nm, p, sh, s);
            else
                e = adjoint_step_t<float>(reaction, su, sv, lam_u[cur], lam_v[cur], lam_u[cur ^ 1],
                                          lam_v[cur ^ 1], partial, nn, nm, p, sh, s);
            if (e != cudaSuccess) return cuda_error(e, "adjoint step");
            cur ^= 1;
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

}  // extern "C"
