/*
 * rdcnn.h -- C ABI of the GB300 (sm_103a) RD-CNN FitzHugh-Nagumo stepper.
 *
 * The library advances the two-layer reaction-diffusion cellular nonlinear
 * network of Dogaru & Dogaru (arXiv 2102.10340), Sec. II.A, Eq. 1-3:
 *
 *   u+_ij = u_ij + dt [ f1(u_ij, v_ij) + Du (u_{i+1,j} + u_{i-1,j} + u_{i,j-1} + u_{i,j+1} - 4 u_ij) ]
 *   v+_ij = v_ij + dt [ f2(u_ij, v_ij) + Dv (v_{i+1,j} + v_{i-1,j} + v_{i,j-1} + v_{i,j+1} - 4 v_ij) ]
 *   f1(u, v) = c u - u^3 / 3 - v          (Eq. 2)
 *   f2(u, v) = -eps (u - b v + a)         (Eq. 3)
 *
 * for every cell at once (both "+" values from the old state), T times, on
 * an NN x NM torus (indices wrap on both axes, the only boundary of the
 * paper, Sec. II.B-II.C).
 *
 * The paper presents the simulator as a template for other cellular
 * nonlinear / FDTD models and names the Chua-Yang cellular neural network
 * (Sec. I, Sec. II.A) without fixing a second model.  Two such variants are
 * provided, and every entry point supports them (single-grid runs, the
 * batched sweep, snapshots and the adjoint) except rdcnn_run_static, which
 * takes neither:
 *  - RDCNN_BC_ZEROFLUX: no flux across the grid edge; the ghost cell beyond
 *    an edge holds the value of the edge cell itself;
 *  - RDCNN_REACTION_CENN: the Chua-Yang cell with output
 *    y(x) = (|x + 1| - |x - 1|) / 2, a cross-shaped feedback template
 *    (centre c, arms Du, corners 0) and a constant offset plane w held in v
 *    (the control template's response to an input image plus the bias):
 *      u+_ij = u_ij + dt [ -u_ij + c y(u_ij) + Du (y_{i+1,j} + y_{i-1,j} + y_{i,j-1} + y_{i,j+1}) + v_ij ]
 *      v+_ij = v_ij
 *    a, b, eps and Dv are ignored (they must still be finite).
 *
 * Reduced-precision storage (not in the paper): a handle of dtype RDCNN_BF16
 * or RDCNN_F16 keeps u, v and the workspace in 16-bit planes (bfloat16 /
 * IEEE half, element type uint16_t-sized) and computes every step in FP32;
 * a launch loads 16-bit values, advances them its k steps in FP32 registers
 * and rounds the result to nearest (ties to even) when it stores it.  This
 * halves the bytes per cell-step of the single-step kernel (8 B instead of
 * 16) at the cost of one 16-bit rounding per launch.  Supported by
 * rdcnn_init / set_state / run / get_state / run_snapshots / plan and by
 * the batched sweep (rdcnn_batch_run*, rdcnn_batch_summary); the adjoint,
 * static-scratch and TEMPORAL2 paths return RDCNN_EINVAL.
 *
 * Conventions shared by every entry point
 *  - Layout: one plane per field, row-major [NN][NM], element (i, j) at
 *    offset i * NM + j; i is the row (NN rows), j the column (NM columns).
 *  - Element type: float (RDCNN_F32), double (RDCNN_F64), bfloat16
 *    (RDCNN_BF16) or IEEE half (RDCNN_F16), fixed per handle.
 *  - Memory ownership: the CALLER owns every buffer, host or device.  The
 *    library allocates no device buffers; scratch space is passed in by the
 *    caller, sized by the matching *_workspace_bytes query.  A handle creates
 *    only CUDA objects of its own (streams for snapshot copies, graph
 *    capture and the adjoint's segment rebuilds, a few events, one graph
 *    executable), released by rdcnn_destroy.
 *  - Streams: work is enqueued on the caller's CUDA stream (cudaStream_t
 *    passed as void*; NULL = legacy default stream).  Calls that return data
 *    to host memory synchronise that stream before returning; all other calls
 *    are asynchronous.
 *  - Errors: every int-returning call returns RDCNN_OK (0), a positive
 *    warning, or a negative error code; rdcnn_last_error() then describes the
 *    last failure on the calling thread.  Invalid arguments are rejected on
 *    the host before any GPU work is enqueued.
 *  - Threads: a handle may be used by one host thread at a time.
 */
#ifndef RDCNN_H
#define RDCNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The gene plus the time step (Sec. II.A "Pars": dt, a, b, eps, c, Du, Dv).
 * Paper defaults (Sec. II.A, get_init_state): dt=0.1, a=-0.3, b=1.3,
 * eps=-0.1, c=1, Du=0.06, Dv=1. */
typedef struct rdcnn_params {
    double dt, a, b, eps, c, Du, Dv;
} rdcnn_params;

enum rdcnn_status {
    RDCNN_OK = 0,
    RDCNN_WARN_CFL = 1,     /* accepted, but dt * max(Du, Dv) > 1/4: the explicit
                               5-point scheme is then not von Neumann stable */
    RDCNN_EINVAL = -1,      /* bad argument: size, pointer, alignment, enum, non-finite param */
    RDCNN_ECUDA = -2,       /* a CUDA runtime call or kernel launch failed */
    RDCNN_ETIMEOUT = -3,    /* a bounded device-side wait gave up */
    RDCNN_ENONFINITE = -4,  /* a NaN or Inf was found where a finite value is required */
    RDCNN_ESTATE = -5,      /* handle not bound to state buffers */
    RDCNN_ESPACE = -6       /* caller-provided workspace is too small */
};

enum { RDCNN_BC_PERIODIC = 0,                    /* toroidal wrap, Sec. II.B-II.C */
       RDCNN_BC_ZEROFLUX = 1 };                   /* ghost cell = edge cell (see above) */
enum { RDCNN_F32 = 0, RDCNN_F64 = 1,
       RDCNN_BF16 = 2,                            /* bf16 planes, FP32 arithmetic (see below) */
       RDCNN_F16 = 3 };                           /* IEEE half planes, FP32 arithmetic */
enum { RDCNN_REACTION_FHN = 0,                    /* Eq. 2-3 */
       RDCNN_REACTION_NONE = 1,                   /* f1 = f2 = 0: pure diffusion (testing) */
       RDCNN_REACTION_CENN = 2 };                 /* Chua-Yang cell (see above) */
enum { RDCNN_VARIANT_AUTO = 0,                    /* library's choice (temporal when possible) */
       RDCNN_VARIANT_STEP1 = 1,                   /* one launch per time step, float4/double2 rows */
       RDCNN_VARIANT_TEMPORAL = 2,                /* k time steps fused per launch */
       RDCNN_VARIANT_GENERIC = 3,                 /* scalar path: any size, any alignment */
       RDCNN_VARIANT_TEMPORAL2 = 4,               /* temporal, the k stages split over two warps */
       RDCNN_VARIANT_TEMPORAL_WIDE = 5 };         /* temporal, 8 values per lane (k <= 4; not F64) */

/* Launch shape: k = time steps fused per launch of the temporal kernels
 * (1..8 F32 / BF16 / F16, 1..4 F64, at most 4 for RDCNN_VARIANT_TEMPORAL_WIDE;
 * 0 = library default), rows = grid rows each warp walks (0 = library
 * default).  For F32 / F64 neither changes results, only speed; for 16-bit
 * planes k is also the rounding interval (see above). */
typedef struct rdcnn_tune {
    int k;
    int rows;
} rdcnn_tune;

typedef struct rdcnn rdcnn_t;                     /* opaque simulation handle */

/* ------------------------------------------------------------------ single grid */

/* Create a handle for an NN x NM grid (Sec. II.A: "NNxNM" array of cells).
 * 1 <= nn, nm < 2^30 and nn * nm <= 2^40 (plane offsets are 64-bit; grids
 * beyond 2^31 cells are supported); p finite; boundary RDCNN_BC_PERIODIC/ZEROFLUX; dtype
 * RDCNN_F32/F64/BF16/F16; reaction RDCNN_REACTION_FHN/NONE/CENN.  Du, Dv >= 0 except
 * for CENN, whose feedback weights c and Du may have either sign (and which
 * gets no RDCNN_WARN_CFL check).  Pure host call (no CUDA work).
 * Returns RDCNN_OK, RDCNN_WARN_CFL (handle still created) or RDCNN_EINVAL.
 * A ZEROFLUX or CENN handle supports every entry point and variant. */
int rdcnn_create(rdcnn_t **out, int64_t nn, int64_t nm, const rdcnn_params *p,
                 int boundary, int dtype, int reaction);

/* Replace the gene of an existing handle (same validation as create). */
int rdcnn_set_params(rdcnn_t *h, const rdcnn_params *p);

/* Set the handle's launch shape (see rdcnn_tune); NULL restores defaults.
 * rdcnn_run uses tune->k when its own k argument is 0, and tune->rows for
 * the rows per warp of every vectorised variant.  rdcnn_adjoint uses tune->k
 * (capped at 8 for F32, 4 for F64; default 4 / 2, and 5 for F32 when every
 * state is stored) as the depth of its
 * recompute and reverse launches, and sizes its workspace for it: set the
 * tune before rdcnn_adjoint_workspace_bytes.  Errors: RDCNN_EINVAL. */
int rdcnn_set_tune(rdcnn_t *h, const rdcnn_tune *tune);

/* Bytes of device scratch rdcnn_run needs: two planes (the "Anew"/"Bnew"
 * ping-pong partners of Sec. II.B) of NN * NM * sizeof(element) bytes each,
 * the second starting at the first one's size rounded up to 256 bytes. */
int rdcnn_workspace_bytes(const rdcnn_t *h, size_t *bytes);

/* Attach caller-owned device buffers: u and v planes (the state, updated in
 * place by rdcnn_run), scratch of at least rdcnn_workspace_bytes, and the
 * stream all later work is enqueued on.  Pointers must be device pointers;
 * 16-byte alignment enables the vectorised kernels (otherwise the generic
 * path is used).  Errors: RDCNN_EINVAL (null pointer), RDCNN_ESPACE. */
int rdcnn_bind(rdcnn_t *h, void *u, void *v, void *workspace, size_t workspace_bytes,
               void *stream);

/* Initial state u = v = ka * x (Eq. 1, first line; Sec. II.A "scaling factor
 * k_a").  x is an NN x NM plane of the handle's dtype, in host memory
 * (x_on_device = 0; copied in, the call returns when x may be reused) or
 * device memory (x_on_device = 1; asynchronous).  Errors: RDCNN_ESTATE,
 * RDCNN_EINVAL, RDCNN_ECUDA. */
int rdcnn_init(rdcnn_t *h, const void *x, double ka, int x_on_device);

/* Load an arbitrary state (u0, v0) (checkpoint restore).  Same memory rules
 * as rdcnn_init. */
int rdcnn_set_state(rdcnn_t *h, const void *u0, const void *v0, int on_device);

/* Apply Eq. 1 T times (t = 1..T, Sec. II.A) to the bound state, in place.
 * variant: RDCNN_VARIANT_*; k: time steps fused per launch for the temporal
 * variants (0 = library default; 1..8 for F32 / BF16 / F16, 1..4 for F64).
 * For F32 and F64 all variants give bit-identical results; they differ only
 * in speed.  For BF16 / F16 every launch rounds the state once when it
 * stores it, so results depend on the steps per launch (k for TEMPORAL, 1
 * for STEP1 and GENERIC); variants with the same k agree bit for bit.
 * T = 0 is a no-op.  Asynchronous on the bound stream.  Runs of small grids
 * (cells x k <= 2^23) with at least 64 full-depth launches replay a CUDA
 * graph of 32 captured launches (captured once per launch configuration on a
 * stream the handle owns; not while the bound stream is being captured):
 * the same kernels, the same bits, less launch overhead.  The stepping
 * kernels of every entry point are launched with programmatic dependent
 * launch (each may be scheduled while the previous one drains, and reads
 * nothing before it has completed); the environment variable RDCNN_PDL=0,
 * read once per process, launches them plainly.  The vectorised
 * variants need NM to be a multiple of 4 (F32, BF16, F16) or 2 (F64) and
 * 16-byte (8-byte for BF16 / F16) aligned buffers;
 * AUTO falls back to GENERIC otherwise, an explicit request returns
 * RDCNN_EINVAL.  The handle's reaction and boundary apply to every
 * variant; RDCNN_VARIANT_TEMPORAL2 takes FP32 / FP64 handles only.
 * Errors: RDCNN_ESTATE, RDCNN_EINVAL, RDCNN_ECUDA. */
int rdcnn_run(rdcnn_t *h, int64_t T, int variant, int k);

/* RDCNN_VARIANT_TEMPORAL_WIDE: the temporal pipeline with 8 values per lane
 * (32 bytes of float, 16 of a 16-bit type) instead of 4, so one halo lane per
 * side serves every depth and the per-row costs of a lane cover twice the
 * cells; the register windows double, so k is limited to 1..4.  Needs NM % 8
 * == 0 and 16-byte aligned buffers (RDCNN_EINVAL otherwise, as for the other
 * explicit vectorised variants); not for RDCNN_F64.  Same bits as TEMPORAL at
 * the same k. */

/* The launch shape rdcnn_run(h, T, *variant, out->k) would use, without
 * running anything.  In: *variant (RDCNN_VARIANT_*, AUTO allowed) and
 * out->k (0 = the handle's tuned or default depth).  Out: *variant resolved
 * from AUTO, out->k = time steps per full launch (1 for STEP1 / GENERIC),
 * out->rows = rows per warp strip (the tuned rows, else the launcher's own
 * choice; 0 for GENERIC).  Queries the current device's SM count and kernel
 * occupancy.  Errors: RDCNN_EINVAL (as rdcnn_run would return). */
int rdcnn_plan(const rdcnn_t *h, int *variant, rdcnn_tune *out);

/* Copy the current state out (the "lastA, lastB" the paper's display
 * function returns, Sec. II.A).  to_device = 0: host buffers, the call
 * synchronises the stream; to_device = 1: device buffers, asynchronous.
 * Either output pointer may be NULL to skip that field. */
int rdcnn_get_state(rdcnn_t *h, void *u_out, void *v_out, int to_device);

/* T steps of Eq. 1 with the state captured every `every` steps: the A_show /
 * B_show arrays of the paper's main loop (Sec. II.B, every test_mod
 * iterations the state is copied to the host; slot 0 is the initial state).
 * Snapshot s (s = 0 .. T/every, integer division) is the state after
 * s * every steps, written to u_snap + s*NN*NM and v_snap + s*NN*NM
 * (elements of the handle's dtype).  snap_on_device = 1: device arrays,
 * copied on the bound stream, asynchronous.  snap_on_device = 0: host arrays
 * (pinned memory lets the copies overlap the steps); each snapshot passes
 * through a device staging slot of 2 planes taken from `staging`
 * (staging_bytes / (2 * plane bytes) slots, at least one) and is copied on a
 * second stream while the run continues; the call returns when every
 * snapshot has landed.  The final state is left in the bound u, v, as after
 * rdcnn_run(h, T, AUTO, 0); the results are bit-identical to it.
 * Errors: RDCNN_ESTATE, RDCNN_EINVAL, RDCNN_ESPACE (no staging for host
 * snapshots), RDCNN_ECUDA. */
int rdcnn_run_snapshots(rdcnn_t *h, int64_t T, int64_t every, void *u_snap, void *v_snap,
                        int snap_on_device, void *staging, size_t staging_bytes);

/* Release the handle (not the caller's buffers).  NULL is ignored. */
void rdcnn_destroy(rdcnn_t *h);

/* ------------------------------------------------------------------ batched sweep */

/* One instance of a parameter sweep (Sec. III.A explores the (Du, Dv) plane
 * and Sec. III.B the (a, b) plane by running many simulations).  Each
 * instance has its own grid size and its own gene, dt included.
 * u, v: the instance's state planes (device, updated in place);
 * su, sv: two scratch planes of the same size (device). */
typedef struct rdcnn_instance {
    int64_t nn, nm;
    rdcnn_params params;
    void *u, *v;
    void *su, *sv;
} rdcnn_instance;

/* Bytes of device workspace rdcnn_batch_run needs for its work table. */
int rdcnn_batch_workspace_bytes(const rdcnn_instance *inst, int n, int dtype,
                                const rdcnn_tune *tune, size_t *bytes);

/* Run T steps of Eq. 1 on all n instances with the same reaction and dtype
 * (RDCNN_F32, F64, BF16 or F16; 16-bit planes compute in FP32 and round the
 * state once per launch, as rdcnn_run's TEMPORAL variant does).
 * All instances advance together: each launch covers every instance for k
 * steps, so small grids do not pay one launch per step each.  Vectorised
 * layout rules as for rdcnn_run apply to every instance (NM a multiple of 4,
 * or 2 for F64; 16-byte aligned pointers, 8-byte for BF16 / F16), else
 * RDCNN_EINVAL.  tune may be NULL.
 * Asynchronous on `stream`, except that the work table is copied to the
 * device first (host-synchronous copy into `workspace`). */
int rdcnn_batch_run(const rdcnn_instance *inst, int n, int64_t T, int dtype, int reaction,
                    const rdcnn_tune *tune, void *workspace, size_t workspace_bytes,
                    void *stream);

/* rdcnn_batch_run with the model variants: boundary RDCNN_BC_PERIODIC or
 * RDCNN_BC_ZEROFLUX, reaction FHN / NONE / CENN (the CeNN gene may carry
 * feedback weights of either sign), shared by all instances; every dtype
 * supports every combination.  rdcnn_batch_run(...) ==
 * rdcnn_batch_run_model(..., RDCNN_BC_PERIODIC, ...). */
int rdcnn_batch_run_model(const rdcnn_instance *inst, int n, int64_t T, int dtype, int reaction,
                          int boundary, const rdcnn_tune *tune, void *workspace, size_t workspace_bytes,
                          void *stream);

/* Statistics of every instance's state, computed on the device for ranking
 * the instances of a parameter search (Sec. III.A sorts (Du, Dv) into slow
 * growth, dynamic patterns and dull homogeneous states; Sec. III.B searches
 * (a, b) for edge-detecting behaviour).  Only nn, nm, u, v of each instance
 * are used.  out (host, n x 8 doubles), per instance:
 *   mean(u), var(u), min(u), max(u), mean(v), var(v),
 *   mean of |u(i+1,j) - u(i,j)| + |u(i,j+1) - u(i,j)| (wrapping), and the
 *   fraction of cells where that sum exceeds `threshold`.
 * Variances are population variances.  dtype: any RDCNN_* plane type (16-bit
 * planes are read into FP32).  Work runs on `stream`; the call
 * returns when `out` is filled.  workspace: device, at least
 * rdcnn_summary_workspace_bytes.  Errors: RDCNN_EINVAL, RDCNN_ESPACE,
 * RDCNN_ECUDA. */
int rdcnn_summary_workspace_bytes(const rdcnn_instance *inst, int n, size_t *bytes);
int rdcnn_batch_summary(const rdcnn_instance *inst, int n, int dtype, double threshold, double *out,
                        void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ adjoint */

/* Bytes of device workspace rdcnn_adjoint needs for T steps with
 * n_checkpoints stored states (0 = ceil(sqrt(T))). */
int rdcnn_adjoint_workspace_bytes(const rdcnn_t *h, int64_t T, int64_t n_checkpoints,
                                  size_t *bytes);

/* Reverse-mode derivative of T steps of Eq. 1-3 (not in the paper: the
 * exact discrete adjoint of the update, for gradient-based fitting of the
 * gene the paper searches for in Sec. III).  Given the start state (u0, v0)
 * and the co-state dL/du_T, dL/dv_T of a loss L of the final state, writes
 * dL/du0, dL/dv0 (device planes) and grad[6] = dL/d{Du, Dv, a, b, eps, c}
 * (host array, FP64).  Forward states are rebuilt from n_checkpoints stored
 * states (0 = ceil(sqrt(T)); n_checkpoints >= T stores every state, T plane
 * pairs of workspace, and rebuilds nothing).  All planes are device planes of the handle's
 * size and dtype; the bound u/v/workspace of the handle are not touched.
 * The handle's boundary applies (the zero-flux Laplacian, like the periodic
 * one, is symmetric, so the co-state diffuses under the same operator), and
 * its reaction: for CENN handles grad holds dL/dDu (the neighbour feedback
 * weight) and dL/dc (the self-feedback weight), the other entries are 0, and
 * the output function's slope is taken as 1 on (-1, 1) and 0 elsewhere.
 * With more than one checkpoint segment the segment rebuilds run on a
 * stream the handle owns (created on first use, released by rdcnn_destroy),
 * ordered against the bound stream by events, and the workspace holds two
 * sets of segment states.  Synchronises the handle's stream (grad is a host
 * result). */
int rdcnn_adjoint(rdcnn_t *h, int64_t T, const void *u0, const void *v0,
                  const void *dLdu_T, const void *dLdv_T, int64_t n_checkpoints,
                  void *dLdu0, void *dLdv0, double grad[6],
                  void *workspace, size_t workspace_bytes);

/* ------------------------------------------------------------------ recorded forward + adjoint */

/* For training loops, where the forward run that produces the loss happens
 * anyway: rdcnn_run_record records the states the adjoint needs while it
 * runs, and rdcnn_adjoint_tape then skips rdcnn_adjoint's own forward sweep.
 * Not in the paper, like the adjoint.
 *
 * Tape layout (device memory, caller-owned, 16-byte aligned): slot i
 * (i = 0 .. nseg - 1) holds the state at step i*S as two planes, u then v,
 * each padded to a multiple of 256 bytes, where S = ceil(T / n) and
 * nseg = ceil(T / S) for n = n_checkpoints (0 = ceil(sqrt(T)); n >= T keeps
 * every state 0 .. T-1, and the adjoint then recomputes nothing).
 * rdcnn_tape_bytes gives the tape size and the workspace rdcnn_adjoint_tape
 * needs for that n (both depend on the handle's tune k, as for
 * rdcnn_adjoint: set the tune first).  FP32 / FP64 handles, NM a multiple of
 * 4 (F32) or 2 (F64).  Errors: RDCNN_EINVAL. */
int rdcnn_tape_bytes(const rdcnn_t *h, int64_t T, int64_t n_checkpoints, size_t *tape_bytes,
                     size_t *workspace_bytes);

/* rdcnn_run(h, T, RDCNN_VARIANT_AUTO, 0) that also writes the tape: the bound
 * state advances by T steps (the same bits as rdcnn_run) and slot i of the
 * tape receives the state at step i*S of this run (slot 0: the state at the
 * call).  Uses the bound workspace as scratch; asynchronous on the bound
 * stream.  The bound buffers and the tape must be 16-byte aligned.
 * Errors: RDCNN_ESTATE, RDCNN_EINVAL, RDCNN_ESPACE (tape too small),
 * RDCNN_ECUDA. */
int rdcnn_run_record(rdcnn_t *h, int64_t T, int64_t n_checkpoints, void *tape, size_t tape_bytes);

/* rdcnn_adjoint with the forward states read from a tape that
 * rdcnn_run_record wrote for the same T, n_checkpoints, gene, tune and
 * boundary (the start state is the tape's slot 0, so u0 and v0 are not
 * passed).  The tape is only read.  Outputs, synchronisation and errors as
 * for rdcnn_adjoint (RDCNN_ESPACE also for a short tape); the results are
 * those rdcnn_adjoint returns for that start state and n_checkpoints, bit
 * for bit.  workspace: at least the *workspace_bytes rdcnn_tape_bytes
 * reports. */
int rdcnn_adjoint_tape(rdcnn_t *h, int64_t T, int64_t n_checkpoints, const void *tape, size_t tape_bytes,
                       const void *dLdu_T, const void *dLdv_T, void *dLdu0, void *dLdv0, double grad[6],
                       void *workspace, size_t workspace_bytes);

/* ------------------------------------------------------------------ no-allocation run */

/* Bytes of the fixed device array rdcnn_run_static uses as scratch. */
#define RDCNN_STATIC_SCRATCH_BYTES (16u << 20)

/* rdcnn_run for callers that cannot allocate device memory.  The paper has no
 * counterpart: it exists for hosts that own the whole device memory pool
 * (plug-ins inside another framework, which forbids or cannot budget extra
 * cudaMalloc calls) and for C/Fortran drivers that only receive device
 * pointers from another component, and so cannot supply the scratch
 * workspace rdcnn_bind asks for.
 *
 * Advances the caller's state planes u, v (device, NN x NM, dtype RDCNN_F32
 * or RDCNN_F64, updated in place) by T steps of the same update as rdcnn_run
 * on a periodic (toroidal) handle -- this entry point has no boundary
 * argument and always uses the paper's torus -- with the FHN or NONE
 * reaction (temporal kernel when NM is a multiple of 4 / 2 and u, v are
 * 16-byte aligned, generic otherwise; k = steps per launch, 0 = default;
 * the same bits as rdcnn_run), asynchronously on `stream`.  The two
 * ping-pong planes live in one file-scope __device__ array of
 * RDCNN_STATIC_SCRATCH_BYTES (16 MiB) that every GPU loading this library
 * holds until the process exits, so NN * NM * sizeof(element) may be at most
 * 8 MiB (2,097,152 FP32 or 1,048,576 FP64 cells; the second plane starts at
 * the first one's size rounded up to 256 bytes); larger grids return
 * RDCNN_EINVAL before any GPU work.  The call allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).
 * All calls share that one array and it keeps the last call's contents
 * (nothing in it needs to start at zero): calls whose GPU work overlaps in
 * time -- other streams or other host threads on the same device -- race on
 * it and must be serialised by the caller.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress, which may load
 * the library's module on that device); make that first call before any
 * stream capture begins on the device.  The address is kept for the life of
 * the process, so the entry point must not be used after a cudaDeviceReset
 * (or another teardown of the device's primary context) in that process.
 * Errors: RDCNN_EINVAL, RDCNN_ENONFINITE, RDCNN_ECUDA; RDCNN_WARN_CFL as for
 * rdcnn_create. */
int rdcnn_run_static(int64_t nn, int64_t nm, const rdcnn_params *p, int dtype, int reaction,
                     void *u, void *v, int64_t T, int k, void *stream);

/* ------------------------------------------------------------------ diagnostics */

/* Description of the last error on the calling thread ("" if none). */
const char *rdcnn_last_error(void);

/* Number of kernels this library has launched in this process (all devices,
 * all handles).  Used by benchmarks to report launch counts. */
uint64_t rdcnn_launch_count(void);

/* Library version string. */
const char *rdcnn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RDCNN_H */
