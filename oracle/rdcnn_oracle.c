/*
 * rdcnn_oracle.c -- plain, slow, FP64 CPU oracle for the RD-CNN
 * FitzHugh-Nagumo explicit-Euler update (Dogaru & Dogaru, arXiv 2102.10340).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * What it computes (Sec. II.A, Eq. 1-3):
 *   u_ij <- u_ij + dt [ f1(u_ij, v_ij) + Du (u_{i+1,j} + u_{i-1,j} + u_{i,j-1} + u_{i,j+1} - 4 u_ij) ]
 *   v_ij <- v_ij + dt [ f2(u_ij, v_ij) + Dv (same stencil on v) ]
 *   f1(u,v) = c u - u^3 / 3 - v                    (Eq. 2)
 *   f2(u,v) = -eps (u - b v + a)                   (Eq. 3)
 * Both "+" values are formed from the OLD state before either is assigned
 * (the bracket of Eq. 1 assigns u = u+, v = v+ only after both are formed),
 * i.e. a Jacobi sweep.  Neighbour indices wrap around both axes (toroidal
 * boundary, Sec. II.B kernel description and Sec. II.C "modulo" remark).
 *
 * Readings where the paper is silent (all recorded in the design notes):
 *  - precision: FP64 here; compile with -ffp-contract=off so that every
 *    product and sum is rounded as written;
 *  - the four-neighbour sum is grouped as (vertical pair) + (horizontal pair):
 *    ((u_{i+1,j} + u_{i-1,j}) + (u_{i,j-1} + u_{i,j+1})) - 4 u_ij, so that a
 *    uniform field has a Laplacian of exactly zero;
 *  - layout: row-major [NN][NM], i = row in 0..NN-1, j = column in 0..NM-1.
 *
 * Parameter vector p[7] = {dt, a, b, eps, c, Du, Dv} (the order the paper's
 * "Pars" vector is indexed in, Sec. II.B).
 *
 * Model variants (Sec. I and Sec. II.A say the framework is a template for
 * other cellular nonlinear / FDTD models, naming the Chua-Yang cellular
 * neural network; no second model is specified, so these are readings):
 *  - boundary ZEROFLUX: no flux across the grid edge, i.e. the ghost cell
 *    beyond an edge holds the value of the edge cell itself (the neighbour
 *    index is clamped into the grid instead of wrapped);
 *  - reaction CENN: the Chua-Yang cell with the piecewise-linear output
 *    y(x) = (|x + 1| - |x - 1|) / 2, a cross-shaped feedback template
 *    (centre c, the four arms Du, corners 0) and a constant offset plane w
 *    carried in v (the control template's response to the input image plus
 *    the bias):
 *      x_ij <- x_ij + dt [ -x_ij + c y(x_ij) + Du (y_N + y_S + y_W + y_E) + w_ij ],
 *      w_ij <- w_ij.
 *    a, b, eps and Dv are unused.
 *
 * The adjoint (oracle_adjoint) is not in the paper.  It is the exact discrete
 * adjoint (reverse-mode derivative) of the map above, derived by
 * differentiating Eq. 1-3 with respect to u_ij, v_ij and the gene; the
 * derivation is written out above that function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define P_DT 0
#define P_A 1
#define P_B 2
#define P_EPS 3
#define P_C 4
#define P_DU 5
#define P_DV 6

/* reaction selector: 0 = FitzHugh-Nagumo (Eq. 2-3); 1 = none (f1 = f2 = 0,
 * pure diffusion, used only to pin the stencil against closed forms);
 * 2 = Chua-Yang cellular neural network cell (see the header). */
#define ORACLE_FHN 0
#define ORACLE_NONE 1
#define ORACLE_CENN 2

/* boundary selector: 0 = toroidal wrap; 1 = zero flux (ghost = edge cell) */
#define ORACLE_PERIODIC 0
#define ORACLE_ZEROFLUX 1

static int64_t wrap_index(int64_t i, int64_t n) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

/* Index of the cell that stands in for neighbour index i (i may be -1 or n). */
static int64_t neighbour_index(int64_t i, int64_t n, int boundary) {
    if (boundary == ORACLE_ZEROFLUX) return i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
    return wrap_index(i, n);
}

/* Chua-Yang output function: linear on [-1, 1], saturated outside. */
static double cenn_output(double x) {
    return 0.5 * (fabs(x + 1.0) - fabs(x - 1.0));
}

/* Eq. 2 */
static double reaction_f1(double u, double v, const double *p) {
    return p[P_C] * u - (u * u * u) / 3.0 - v;
}

/* Eq. 3 */
static double reaction_f2(double u, double v, const double *p) {
    return -p[P_EPS] * (u - p[P_B] * v + p[P_A]);
}

/* Discrete 5-point Laplacian of plane f at (i, j) (Eq. 1); the neighbours
 * beyond the edge follow the boundary selector. */
static double laplacian_bc(const double *f, int64_t nn, int64_t nm, int64_t i, int64_t j,
                           int boundary) {
    int64_t ip = neighbour_index(i + 1, nn, boundary), im = neighbour_index(i - 1, nn, boundary);
    int64_t jp = neighbour_index(j + 1, nm, boundary), jm = neighbour_index(j - 1, nm, boundary);
    double vert = f[ip * nm + j] + f[im * nm + j];
    double horz = f[i * nm + jm] + f[i * nm + jp];
    return (vert + horz) - 4.0 * f[i * nm + j];
}

/* Slope of the output function: 1 on (-1, 1), 0 outside; at the corners
 * x = +-1, where the function has no derivative, the saturated side's 0. */
static double cenn_slope(double x) {
    return fabs(x) < 1.0 ? 1.0 : 0.0;
}

/* Sum of the four neighbour values of (i, j) (the stand-ins the boundary
 * selects beyond an edge). */
static double neighbour_sum(const double *f, int64_t nn, int64_t nm, int64_t i, int64_t j, int boundary) {
    int64_t ip = neighbour_index(i + 1, nn, boundary), im = neighbour_index(i - 1, nn, boundary);
    int64_t jp = neighbour_index(j + 1, nm, boundary), jm = neighbour_index(j - 1, nm, boundary);
    return (f[im * nm + j] + f[ip * nm + j]) + (f[i * nm + jm] + f[i * nm + jp]);
}

/* Sum of the CeNN outputs y of the four neighbours of (i, j). */
static double neighbour_output_sum(const double *x, int64_t nn, int64_t nm, int64_t i, int64_t j,
                                   int boundary) {
    int64_t ip = neighbour_index(i + 1, nn, boundary), im = neighbour_index(i - 1, nn, boundary);
    int64_t jp = neighbour_index(j + 1, nm, boundary), jm = neighbour_index(j - 1, nm, boundary);
    double vert = cenn_output(x[im * nm + j]) + cenn_output(x[ip * nm + j]);
    double horz = cenn_output(x[i * nm + jm]) + cenn_output(x[i * nm + jp]);
    return vert + horz;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * One application of the update to the whole grid: (u, v) -> (un, vn), with
 * the given reaction and boundary.  The four buffers must be distinct.  Rows
 * are independent, so the row loop may be split across threads without
 * changing any result.
 */
void oracle_step_bc(int64_t nn, int64_t nm, const double *u, const double *v,
                    double *un, double *vn, const double *p, int reaction, int boundary,
                    int nthreads) {
    set_threads(nthreads);
    const double dt = p[P_DT], Du = p[P_DU], Dv = p[P_DV];
#pragma omp parallel for schedule(static) if (nthreads != 1)
    for (int64_t i = 0; i < nn; ++i) {
        for (int64_t j = 0; j < nm; ++j) {
            const int64_t c = i * nm + j;
            const double uc = u[c], vc = v[c];
            if (reaction == ORACLE_CENN) {
                /* state x = u, offset w = v (constant) */
                const double feedback = p[P_C] * cenn_output(uc)
                                        + Du * neighbour_output_sum(u, nn, nm, i, j, boundary);
                un[c] = uc + dt * ((-uc + feedback) + vc);
                vn[c] = vc;
                continue;
            }
            const double lu = laplacian_bc(u, nn, nm, i, j, boundary);
            const double lv = laplacian_bc(v, nn, nm, i, j, boundary);
            double r1 = 0.0, r2 = 0.0;
            if (reaction == ORACLE_FHN) {
                r1 = reaction_f1(uc, vc, p);
                r2 = reaction_f2(uc, vc, p);
            }
            un[c] = uc + dt * (r1 + Du * lu);
            vn[c] = vc + dt * (r2 + Dv * lv);
        }
    }
}

/* One application of Eq. 1 on the torus (the paper's model). */
void oracle_step(int64_t nn, int64_t nm, const double *u, const double *v,
                 double *un, double *vn, const double *p, int reaction, int nthreads) {
    oracle_step_bc(nn, nm, u, v, un, vn, p, reaction, ORACLE_PERIODIC, nthreads);
}

/*
 * T applications of the update (t = 1..T), in place on (u, v).  Allocates
 * two scratch planes; returns 0, or -1 when allocation fails or sizes are bad.
 */
int oracle_run_bc(int64_t nn, int64_t nm, double *u, double *v, const double *p,
                  int reaction, int boundary, int64_t T, int nthreads) {
    if (nn <= 0 || nm <= 0 || T < 0) return -1;
    const size_t n = (size_t)nn * (size_t)nm;
    double *un = (double *)malloc(n * sizeof(double));
    double *vn = (double *)malloc(n * sizeof(double));
    if (!un || !vn) { free(un); free(vn); return -1; }
    double *a = u, *b = v, *an = un, *bn = vn;
    for (int64_t t = 0; t < T; ++t) {
        oracle_step_bc(nn, nm, a, b, an, bn, p, reaction, boundary, nthreads);
        double *ta = a, *tb = b;
        a = an; b = bn; an = ta; bn = tb;
    }
    if (a != u) {
        memcpy(u, a, n * sizeof(double));
        memcpy(v, b, n * sizeof(double));
    }
    free(un); free(vn);
    return 0;
}

/* T applications of Eq. 1 on the torus, in place. */
int oracle_run(int64_t nn, int64_t nm, double *u, double *v, const double *p,
               int reaction, int64_t T, int nthreads) {
    return oracle_run_bc(nn, nm, u, v, p, reaction, ORACLE_PERIODIC, T, nthreads);
}

/*
 * Local dynamics of one isolated cell: Eq. 1 with the diffusion terms absent,
 * T steps from (u0, v0).  Writes the trajectory (T + 1 entries, entry 0 = the
 * start) when traj_u / traj_v are non-null, and the end state to *u_out, *v_out.
 */
void oracle_scalar_map(double u0, double v0, const double *p, int64_t T,
                       double *traj_u, double *traj_v, double *u_out, double *v_out) {
    double u = u0, v = v0;
    if (traj_u) traj_u[0] = u;
    if (traj_v) traj_v[0] = v;
    for (int64_t t = 0; t < T; ++t) {
        const double r1 = reaction_f1(u, v, p);
        const double r2 = reaction_f2(u, v, p);
        const double un = u + p[P_DT] * r1;
        const double vn = v + p[P_DT] * r2;
        u = un; v = vn;
        if (traj_u) traj_u[t + 1] = u;
        if (traj_v) traj_v[t + 1] = v;
    }
    *u_out = u; *v_out = v;
}

/*
 * Discrete adjoint of T steps of Eq. 1 (not in the paper).
 *
 * Write one step as (u+, v+) = F(u, v; theta).  For a loss L of the final
 * state, let (lu, lv) = dL/d(u+, v+) (the co-state after the step).  Then
 *   dL/du_k = lu_k + dt [ (c - u_k^2) lu_k + Du (Lap lu)_k - eps lv_k ]
 *   dL/dv_k = lv_k + dt [ -lu_k + eps b lv_k + Dv (Lap lv)_k ]
 * because d f1/du = c - u^2, d f1/dv = -1, d f2/du = -eps, d f2/dv = eps b,
 * and the periodic 5-point Laplacian is a symmetric operator (cell k is a
 * neighbour of m exactly as often as m is a neighbour of k), so its transpose
 * is itself.  The gene enters each step additively, giving per-step terms
 *   dL/dDu  += dt sum_k lu_k (Lap u)_k        dL/dDv  += dt sum_k lv_k (Lap v)_k
 *   dL/dc   += dt sum_k lu_k u_k              dL/da   += dt sum_k lv_k (-eps)
 *   dL/db   += dt sum_k lv_k eps v_k          dL/deps += dt sum_k lv_k (-(u_k - b v_k + a))
 * with (u, v) the state BEFORE the step and (lu, lv) the co-state AFTER it.
 * With reaction NONE the f-terms and the c, a, b, eps gradients vanish.
 *
 * Inputs: start state (u0, v0), T, the co-state of the final state
 * (lu_T, lv_T) = dL/d(u_T, v_T).  Outputs: dL/du0, dL/dv0 and
 * grad[6] = dL/d{Du, Dv, a, b, eps, c}.
 * Forward states are rebuilt from checkpoints taken every S steps
 * (S = ceil(T / n_checkpoints), n_checkpoints <= 0 meaning ceil(sqrt(T))).
 * CeNN cell (reaction ORACLE_CENN; u = state x, v = offset w):
 *   u+ = u + dt [ -u + c y(u) + Du sum_nbr y(u_n) + v ],  v+ = v,
 * so with y' the slope of the output function (cenn_slope),
 *   dL/du_k = lu_k + dt [ -lu_k + y'(u_k) (c lu_k + Du sum_{m: k nbr of m} lu_m) ]
 *   dL/dv_k = lv_k + dt lu_k
 * where the sum over the cells m that have k as a neighbour equals the
 * neighbour sum of lu at k (adjacency is mutual, and under zero flux a
 * missing neighbour stands for the cell itself on both sides).  Per step
 *   dL/dDu += dt sum_k lu_k sum_nbr y(u_n)     dL/dc += dt sum_k lu_k y(u_k)
 * and the other gene entries do not enter.  The output function has no
 * derivative at +-1; the slope there is taken as 0.
 *
 * Returns 0, or -1 on bad sizes, an unknown reaction, a bad boundary, or
 * allocation failure.
 *
 * Zero flux (oracle_adjoint_bc with ORACLE_ZEROFLUX): the forward map uses
 * the Laplacian whose missing neighbours are replaced by the cell itself.
 * As a matrix, its off-diagonal entry (k, m) counts how often m is a
 * neighbour of k, which is mutual, and the replaced neighbours only add to
 * the diagonal, so it is symmetric as well.  The derivation above therefore
 * holds word for word with Lap the zero-flux Laplacian, in the co-state
 * update and in the Du / Dv sums.
 */
int oracle_adjoint_bc(int64_t nn, int64_t nm, const double *u0, const double *v0,
                      const double *p, int reaction, int boundary, int64_t T,
                      const double *lu_T, const double *lv_T, int64_t n_checkpoints,
                      double *lu0_out, double *lv0_out, double *grad, int nthreads) {
    if (nn <= 0 || nm <= 0 || T < 0) return -1;
    if (reaction != ORACLE_FHN && reaction != ORACLE_NONE && reaction != ORACLE_CENN) return -1;
    if (boundary != ORACLE_PERIODIC && boundary != ORACLE_ZEROFLUX) return -1;
    const size_t n = (size_t)nn * (size_t)nm;
    for (int g = 0; g < 6; ++g) grad[g] = 0.0;
    memcpy(lu0_out, lu_T, n * sizeof(double));
    memcpy(lv0_out, lv_T, n * sizeof(double));
    if (T == 0) return 0;
    if (n_checkpoints <= 0) n_checkpoints = (int64_t)ceil(sqrt((double)T));
    if (n_checkpoints > T) n_checkpoints = T;
    const int64_t S = (T + n_checkpoints - 1) / n_checkpoints;
    const int64_t nseg = (T + S - 1) / S;

    double *ck = (double *)malloc((size_t)nseg * 2 * n * sizeof(double));
    double *seg = (double *)malloc((size_t)S * 2 * n * sizeof(double));
    double *tmp_u = (double *)malloc(n * sizeof(double));
    double *tmp_v = (double *)malloc(n * sizeof(double));
    double *lu = (double *)malloc(n * sizeof(double));
    double *lv = (double *)malloc(n * sizeof(double));
    double *lun = (double *)malloc(n * sizeof(double));
    double *lvn = (double *)malloc(n * sizeof(double));
    if (!ck || !seg || !tmp_u || !tmp_v || !lu || !lv || !lun || !lvn) {
        free(ck); free(seg); free(tmp_u); free(tmp_v); free(lu); free(lv); free(lun); free(lvn);
        return -1;
    }

    /* forward sweep, keeping the state at the start of every segment */
    memcpy(tmp_u, u0, n * sizeof(double));
    memcpy(tmp_v, v0, n * sizeof(double));
    for (int64_t s = 0; s < nseg; ++s) {
        memcpy(ck + (size_t)s * 2 * n, tmp_u, n * sizeof(double));
        memcpy(ck + (size_t)s * 2 * n + n, tmp_v, n * sizeof(double));
        const int64_t len = (s + 1) * S <= T ? S : T - s * S;
        if (s + 1 < nseg) oracle_run_bc(nn, nm, tmp_u, tmp_v, p, reaction, boundary, len, nthreads);
    }

    memcpy(lu, lu_T, n * sizeof(double));
    memcpy(lv, lv_T, n * sizeof(double));
    const double dt = p[P_DT], Du = p[P_DU], Dv = p[P_DV];
    const double a = p[P_A], b = p[P_B], eps = p[P_EPS], c = p[P_C];
    const int fhn = (reaction == ORACLE_FHN), cenn = (reaction == ORACLE_CENN);

    for (int64_t s = nseg - 1; s >= 0; --s) {
        const int64_t t0 = s * S;
        const int64_t len = (s + 1) * S <= T ? S : T - t0;
        /* rebuild the states t0 .. t0+len-1 of this segment */
        memcpy(seg, ck + (size_t)s * 2 * n, 2 * n * sizeof(double));
        for (int64_t q = 1; q < len; ++q) {
            const double *pu = seg + (size_t)(q - 1) * 2 * n;
            double *qu = seg + (size_t)q * 2 * n;
            oracle_step_bc(nn, nm, pu, pu + n, qu, qu + n, p, reaction, boundary, nthreads);
        }
        for (int64_t q = len - 1; q >= 0; --q) {
            const double *u = seg + (size_t)q * 2 * n;
            const double *v = u + n;
            double g[6] = {0, 0, 0, 0, 0, 0};
            for (int64_t i = 0; i < nn; ++i) {
                for (int64_t j = 0; j < nm; ++j) {
                    const int64_t k = i * nm + j;
                    const double uk = u[k], vk = v[k], luk = lu[k], lvk = lv[k];
                    if (cenn) {
                        g[0] += luk * neighbour_output_sum(u, nn, nm, i, j, boundary);
                        g[5] += luk * cenn_output(uk);
                        continue;
                    }
                    g[0] += luk * laplacian_bc(u, nn, nm, i, j, boundary);
                    g[1] += lvk * laplacian_bc(v, nn, nm, i, j, boundary);
                    if (fhn) {
                        g[2] += lvk * (-eps);
                        g[3] += lvk * (eps * vk);
                        g[4] += lvk * (-(uk - b * vk + a));
                        g[5] += luk * uk;
                    }
                }
            }
            for (int gi = 0; gi < 6; ++gi) grad[gi] += dt * g[gi];
            set_threads(nthreads);
#pragma omp parallel for schedule(static) if (nthreads != 1)
            for (int64_t i = 0; i < nn; ++i) {
                for (int64_t j = 0; j < nm; ++j) {
                    const int64_t k = i * nm + j;
                    const double uk = u[k], luk = lu[k], lvk = lv[k];
                    if (cenn) {
                        const double back = c * luk + Du * neighbour_sum(lu, nn, nm, i, j, boundary);
                        lun[k] = luk + dt * (-luk + cenn_slope(uk) * back);
                        lvn[k] = lvk + dt * luk;
                        continue;
                    }
                    double ru = 0.0, rv = 0.0;
                    if (fhn) {
                        ru = (c - uk * uk) * luk - eps * lvk;
                        rv = -luk + eps * b * lvk;
                    }
                    lun[k] = luk + dt * (ru + Du * laplacian_bc(lu, nn, nm, i, j, boundary));
                    lvn[k] = lvk + dt * (rv + Dv * laplacian_bc(lv, nn, nm, i, j, boundary));
                }
            }
            double *t1 = lu, *t2 = lv;
            lu = lun; lv = lvn; lun = t1; lvn = t2;
        }
    }
    memcpy(lu0_out, lu, n * sizeof(double));
    memcpy(lv0_out, lv, n * sizeof(double));
    free(ck); free(seg); free(tmp_u); free(tmp_v); free(lu); free(lv); free(lun); free(lvn);
    return 0;
}

/* The toroidal adjoint (the paper's boundary). */
int oracle_adjoint(int64_t nn, int64_t nm, const double *u0, const double *v0,
                   const double *p, int reaction, int64_t T,
                   const double *lu_T, const double *lv_T, int64_t n_checkpoints,
                   double *lu0_out, double *lv0_out, double *grad, int nthreads) {
    return oracle_adjoint_bc(nn, nm, u0, v0, p, reaction, ORACLE_PERIODIC, T, lu_T, lv_T, n_checkpoints,
                             lu0_out, lv0_out, grad, nthreads);
}
