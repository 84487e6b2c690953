/*
 * pc.h -- C ABI of the GB300 (sm_103a) batched Picard-Chebyshev propagator.
 *
 * Method: augmented Picard-Chebyshev (PC) integration of Masat, Colombo &
 * Boutonnet, "GPU-based high-precision orbital propagation of large sets of
 * initial conditions through Picard-Chebyshev augmentation" (arXiv
 * 2301.03989).  Many non-interacting, massless trajectories are propagated at
 * once under the Newtonian gravity of a central body and B perturbing bodies
 * whose positions come from a Chebyshev ephemeris table.  Each trajectory is
 * split into segments; on each segment the Picard iteration (Eq. 2) is run in
 * the matrix form of Section "Matrix form for vectorized and parallel
 * computation" until the sweep-to-sweep change drops below a tolerance.  The
 * trajectories are stacked column-wise (Section "One-level augmentation") in
 * the component-planar layout of Section "Dynamics model, array sorting, and
 * CUDA kernel".
 *
 * Units: km, s, km^3/s^2.  All floating-point arguments are IEEE FP64.
 *
 * Layouts: a batch of M states is "planar": x[c * M + m] for component c in
 * 0..5 = (x, y, z, vx, vy, vz) and trajectory m -- component-stacked columns
 * as in the paper.
 *
 * Ownership: the caller owns every buffer it passes (device or host, as each
 * argument states).  The plan owns its operator, its copy of the force model
 * and ephemeris, and its device workspace.
 *
 * Errors: every entry point returns a pc_status; nothing aborts, prints or
 * traps.  Per-trajectory outcomes go to the optional status[] array.
 *
 * Streams: work is ordered on the CUDA stream passed in (NULL = legacy default
 * stream): it starts after the stream's earlier work and the stream's later
 * work waits for it.  A propagation called on a default stream (legacy or
 * per-thread) runs on a stream the plan owns, forked from and joined back to
 * the caller's by events, because a default stream cannot be captured into
 * the CUDA graphs the round loop replays.  In mixed precision each round also
 * uses a second stream of the plan for its new-segment branch.  Use one plan
 * per concurrently used stream: a plan's workspace and streams are shared by
 * all its calls.
 */
#ifndef PC_H_
#define PC_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pc_plan pc_plan; /* opaque, owned by the library */

typedef enum {
  PC_OK = 0,          /* success */
  PC_EINVAL = 1,      /* bad argument (sizes, NULL pointers, options, arc outside the table) */
  PC_ENOMEM = 2,      /* device or host allocation failed */
  PC_ECUDA = 3,       /* a CUDA runtime call failed */
  PC_ENOTCONV = 4,    /* finished, but at least one trajectory stopped early (status bit 4 or 8) */
  PC_ENONFINITE = 5   /* reserved: a non-finite value where a finite one is required */
} pc_status;

/* Per-trajectory status bits written to status[] (0 = converged everywhere). */
#define PC_IC_STALLED 1        /* a segment was accepted by the stall rule (change stopped falling near tol) */
#define PC_IC_UNRESOLVED 2     /* a segment at the deepest halving still failed the resolution test */
#define PC_IC_NOT_CONVERGED 4  /* stopped: a segment did not converge even at the deepest halving */
#define PC_IC_NONFINITE 8      /* stopped: non-finite input, or the iteration blew up at the deepest halving */
#define PC_IC_OUT_OF_RANGE 16  /* refused: the arc leaves the ephemeris table, or a bad per-trajectory arc */

/* Force model: a(r, t) = -mu_c r/|r|^3 - sum_b mu_b [(r - r_b)/|r - r_b|^3 + r_b/|r_b|^3]
 * (heliocentric Newtonian point masses; the bracket's second term, the
 * indirect term, only when `indirect` != 0).  The paper's own force is the
 * relativistic EIH model (Section "Dynamics model"); this library evaluates
 * the Newtonian one. */
typedef struct {
  int n_bodies;        /* B >= 0 perturbing bodies */
  double mu_central;   /* GM of the central body, > 0 */
  const double *mu;    /* host [n_bodies], copied at plan creation */
  int indirect;        /* 1: include the indirect term */
  double c_light;      /* speed of light in km/s: > 0 adds the relativistic terms of the
                          Einstein-Infeld-Hoffmann equations (the paper's model, Section
                          "Dynamics model"): for the particle among the central body and the
                          table's bodies, velocities taken in the barycentric frame, each body's
                          Newtonian acceleration and potential from the others; 0: Newtonian.
                          The FP32 sweeps of mixed precision keep the Newtonian terms (the FP64
                          sweeps and their residual carry the relativistic ones); reverse mode
                          (tape, adjoint) refuses such a plan with PC_EINVAL. */
} pc_force_model;

/* Ephemeris: granule g covers [t_begin + g*granule_s, t_begin + (g+1)*granule_s)
 * (a time on a boundary uses the later granule; times outside the table use
 * the nearest granule); inside it sigma = 2 (t - t_g)/granule_s - 1 and
 * r_b(t) = sum_k coef[b][g][axis][k] T_k(sigma) (degree at most 63).  The paper evaluates the
 * planetary data once per set of node times, before the iterations (Section
 * "Dynamics model"); so does this library, once per segment. */
typedef struct {
  int n_bodies;         /* must equal the force model's */
  double t_begin;       /* s */
  double granule_s;     /* > 0 */
  int degree;           /* >= 0 */
  int n_granules;       /* >= 1 */
  const double *coef;   /* host [n_bodies][n_granules][3][degree+1], copied at plan creation */
} pc_ephemeris;

#define PC_PREC_FP64 0   /* every sweep in FP64 */
#define PC_PREC_MIXED 1  /* each segment first runs FP32 sweeps on the deviation from its warm start
                            until the change is below switch_tol or stops falling, then FP64 sweeps
                            to tol, with FP32 correction solves between them (refine32); not in
                            the paper: an extension; needs N <= 287 */

#define PC_CONTRACT_DMMA 0   /* FP64 operator contraction on the FP64 tensor cores (mma.sync .f64) */
#define PC_CONTRACT_SPLIT 1  /* the same contraction as exact products of 8-bit digits on the bf16
                                tensor cores: each operand is cut into 7 signed digits (55 bits) against
                                its row's or column's largest exponent, the digit products of one
                                anti-diagonal are summed exactly in FP32, and the sums are combined in
                                64-bit integers and FP64; error below that of an FP64 dot product
                                (N <= 255; larger N use the FP64 tensor cores).  Not in the paper. */

typedef struct {
  double tol;          /* stopping tolerance on the sweep-to-sweep change (overridden per call) */
  int relative;        /* 1: change relative to |r| and |v| of the new iterate; 0: absolute */
  int max_iters;       /* sweeps per segment attempt (>= 1) */
  int max_depth;       /* times a segment may be halved, 0..30 */
  int warm_start;      /* 1: Keplerian two-body guess (central body only); 0: all nodes = x0 */
  int seg_mode;        /* 0: `segments` equal segments per arc; 1: per osculating period of x0 */
  int truncated;       /* 1: drop the degree-(N+1) term of the integral (the paper's N+1-row B) */
  int stall_sweeps;    /* accept a segment when the change has not improved for this many sweeps ... */
  double stall_factor; /* ... and the best change is below stall_factor * tol */
  double div_limit;    /* a change above this, or non-finite, fails the attempt */
  double trunc_tol;    /* resolution test on the Chebyshev tail of the force fit (<= 0 disables) */
  int precision;       /* PC_PREC_FP64 or PC_PREC_MIXED */
  double switch_tol;   /* mixed precision: FP32 sweeps until the change is below this (0: until the
                          FP32 change stops falling) */
  long long max_rounds;/* safety cap on sweep rounds per call (0 = 10,000,000) */
  int refine32;        /* mixed precision: 1 lets an FP64 sweep whose change is below 1e-3 be
                          followed by an FP32 solve for the correction to its iterate (up to
                          two per segment attempt) instead of further FP64 sweeps */
  int contraction;     /* PC_CONTRACT_DMMA or PC_CONTRACT_SPLIT: how FP64 sweeps apply the operator */
  int order;           /* 1: the paper's sweep, y' = x0 + omega2 K f(y); 2: its second-order form
                          (the paper's Introduction and Conclusion name it as a further gain):
                          V' = v0 + omega2 K a(R), then R' = r0 + omega2 K V' -- the same fixed point
                          in about half the sweeps; in FP32 sweeps too; needs PC_CONTRACT_SPLIT
                          and N <= 255 */
  int fp32_mma;        /* mixed precision: 1 runs the FP32 sweeps' operator contraction on the
                          tensor cores as three TF32 products per term (K_hi G_lo + K_lo G_hi +
                          K_hi G_hi, each operand split into TF32 high and low parts; about 2^-22
                          per term, FP32 accumulation), 0 as FP32 multiply-adds.  Not in the
                          paper.  It fixes the FP32 kernel to the tiled shape with 4 rows per
                          thread and node records read from global memory (launch tuning
                          then varies only slots and CTAs per SM): faster on large
                          synchronised batches with few bodies, slower on short lists with
                          many bodies, where one trajectory per CTA wins */
} pc_options;

/* Fills *o with the defaults: tol 1e-13, relative 1, max_iters 60, max_depth 8,
 * warm_start 1, seg_mode 0, truncated 0, stall_sweeps 5, stall_factor 1e3,
 * div_limit 1e3, trunc_tol 1e-13, precision FP64, switch_tol 0, max_rounds 0, refine32 1,
 * contraction PC_CONTRACT_SPLIT, order 1, fp32_mma 0.
 * Returns PC_EINVAL if o is NULL. */
pc_status pc_options_default(pc_options *o);

/* Creates a plan for degree-N segments (N + 1 Chebyshev-Gauss-Lobatto nodes,
 * Eq. chnodes1/2 with tau_0 = -1 at the segment start), `segments` base
 * segments (per arc, or per osculating period with seg_mode 1; Section
 * "Matrix form", piecewise integration).  Builds the PC operator K (the
 * paper's C [S A; A], Eq. for B and y = C B) in extended precision, uploads
 * it with the force model and ephemeris to the current CUDA device.
 * N in [2, 512]; segments >= 1; opt may be NULL (defaults).
 * Errors: PC_EINVAL, PC_ENOMEM, PC_ECUDA.  *out is NULL on failure. */
pc_status pc_plan_create(int N, int segments, const pc_force_model *force, const pc_ephemeris *ephem,
                         const pc_options *opt, pc_plan **out);

/* Propagates n_ic trajectories from t0 to tf (tf < t0 integrates backward).
 *   x0      device, planar [6][n_ic], read only
 *   tol     stopping tolerance for this call (<= 0: the plan's)
 *   xf      device, planar [6][n_ic], written: state at tf, or at the last
 *           accepted segment boundary of a trajectory that stopped early
 *   status  device [n_ic] PC_IC_* bits, or NULL
 *   iters   device [n_ic] sweeps spent (all attempts), or NULL
 *   stream  cudaStream_t or NULL
 * Each trajectory runs its own segment schedule (equal base segments, halved
 * on failure, grown back after success) so trajectories never wait on each
 * other.  Work is queued on `stream`; the call returns once every trajectory
 * has finished (it polls a device counter).  The arc must lie inside the
 * ephemeris table when n_bodies > 0.  n_ic = 0 is a no-op.
 * Returns PC_OK, PC_ENOTCONV (some trajectory stopped early), PC_EINVAL,
 * PC_ENOMEM or PC_ECUDA. */
pc_status pc_propagate(pc_plan *plan, long long n_ic, const double *x0, double t0, double tf, double tol,
                       double *xf, int *status, int *iters, void *stream);

/* Same as pc_propagate, with optional extra outputs (NULL = not wanted):
 *   nseg    device [n_ic]: accepted segments
 *   ckpt    device [n_ic][max_ckpt][7]: (t_a, x(t_a)) at the start of each of the
 *           first max_ckpt accepted segments -- the segment-boundary checkpoints
 *   rounds  host: number of sweep rounds the call ran */
pc_status pc_propagate_ex(pc_plan *plan, long long n_ic, const double *x0, double t0, double tf, double tol,
                          double *xf, int *status, int *iters, int *nseg, int max_ckpt, double *ckpt,
                          long long *rounds, void *stream);

/* ---- Kernel-level entry points -------------------------------------------
 * Each runs one of the device kernels the sweep uses, on caller buffers, so a
 * step can be checked on its own.  All pointers are device pointers; the calls
 * are asynchronous on `stream` and use the plan's workspace (same rule as
 * pc_propagate: one plan per concurrently used stream). */

/* Ephemeris (the table's Chebyshev series) at n_pts times t [n_pts]: rb planar
 * [n_bodies][3][n_pts]. */
pc_status pc_eval_ephemeris(pc_plan *plan, long long n_pts, const double *t, double *rb, void *stream);

/* Dynamics f(y, t) = (v, a(r, t)) of Eq. (ibvp) with the plan's force model at
 * n_pts states y (planar [6][n_pts]) and times t [n_pts]: f planar [6][n_pts]. */
pc_status pc_eval_dynamics(pc_plan *plan, long long n_pts, const double *t, const double *y, double *f,
                           void *stream);

/* Keplerian warm start (central body only): x = two-body propagation of x0 by
 * dt, planar [6][n_pts]; states that are not bound ellipses are copied
 * unchanged (the cold start). */
pc_status pc_eval_warm_start(pc_plan *plan, long long n_pts, const double *x0, const double *dt, double *x,
                             void *stream);

/* The operator contraction of one sweep, y_j = x0 + sum_k K_jk g_k (the
 * paper's B = [S A F + 2 y0; A F], y = C B with F = omega2 f already scaled),
 * for n_ic trajectories: x0 planar [6][n_ic]; g and y node-major planar
 * [N+1][6][n_ic]. */
pc_status pc_apply_operator(pc_plan *plan, long long n_ic, const double *x0, const double *g, double *y,
                            void *stream);

/* Allocation-free variant of pc_apply_operator (the paper has no counterpart:
 * it is an addition of this library for callers that cannot allocate device
 * memory at call time -- for example a caller whose GPU memory is owned by
 * another allocator with a fixed budget, or a latency-sensitive caller that
 * must not risk the implicit device synchronisation of cudaMalloc/cudaFree).
 * Same arguments and result as pc_apply_operator, but the operands are staged
 * in a fixed 32 MiB device array that is part of the library image (every GPU
 * that loads the library holds it until the process exits) instead of the
 * plan's workspace; the call makes no cudaMalloc, cudaFree or other allocating
 * call.
 *   Limit: (4*ceil((N+1)/4) + N + 2) * 6 * 8 * ceil(n_ic/8)*8 bytes must fit in
 *   32 MiB (N = 128: up to 2,664 trajectories); larger n_ic returns PC_EINVAL.
 *   The plan must belong to the current device (else PC_EINVAL).
 *   Every call looks up the array's device address on the current device (a
 *   lookup, not an allocation); the first call on a device also loads the
 *   library's device code there, so make that first call before any stream
 *   capture.
 *   All calls share the one array and it keeps the last call's contents: calls
 *   whose work overlaps on the GPU (different streams, or different host
 *   threads) race on it and must be serialised by the caller. */
pc_status pc_apply_operator_static(pc_plan *plan, long long n_ic, const double *x0, const double *g, double *y,
                                   void *stream);

/* ---- Per-kernel timing ----------------------------------------------------
 * With profiling on, pc_propagate / pc_propagate_ex record a CUDA event
 * between consecutive kernels of every sweep round on the call's stream; the
 * elapsed times are summed when pc_plan_kernel_times is called (not during the
 * propagation, so the host adds no gap to the timed work). */
#define PC_KERNEL_SETUP 0     /* new segments: node times, ephemeris, warm start */
#define PC_KERNEL_FP32 1      /* mixed precision: the FP32 sweeps of new segments */
#define PC_KERNEL_FORCE 2     /* FP64 sweeps: F = omega2 f(Y, t) */
#define PC_KERNEL_CONTRACT 3  /* FP64 sweeps: Y' = x0 + K F and the per-trajectory change */
#define PC_KERNEL_CONTROL 4   /* stop tests, segment accept / halve / advance */
#define PC_KERNEL_KINDS 5
typedef struct {
  long long launches[PC_KERNEL_KINDS];
  double ms[PC_KERNEL_KINDS]; /* summed device time */
  long long sweeps64;         /* trajectory-sweeps done in FP64 */
  long long sweeps32;         /* trajectory-sweeps done in FP32 (mixed precision) */
  long long kernel_launches;  /* device kernels the library launched */
} pc_kernel_times;

/* on != 0 turns per-kernel event recording on for later calls. */
pc_status pc_plan_set_profiling(pc_plan *plan, int on);

/* Sums the recorded intervals into *out (after synchronizing the recorded
 * events) and clears them.  The sweep and launch counts cover every call since
 * the previous pc_plan_kernel_times, whether profiling was on or not. */
pc_status pc_plan_kernel_times(pc_plan *plan, pc_kernel_times *out);

/* ---- Launch tuning and CUDA graphs ------------------------------------------
 * Launch shapes of the sweep kernels and the host's round loop.  None of them
 * changes any arithmetic: results are bitwise the same for every setting.
 *   setup_ctas_per_sm     CTAs per SM of the new-segment set-up kernel (1..16)
 *   fp32_ctas_per_sm      CTAs per SM of the FP32 kernels (1..16)
 *   contract_ctas_per_sm  persistent CTAs per SM of the FP64 contraction (1..16)
 *   rounds_per_batch      sweep rounds queued between two looks at the device's
 *                         done counter (1..64)
 *   repack_div            compact the working set when at least 1/repack_div of
 *                         its slots have finished (2..64)
 *   graphs                1: each batch of rounds is captured once per working-set
 *                         shape as a CUDA graph and replayed (0: direct launches)
 *   side_priority         mixed precision: 1 runs the new-segment branch of each
 *                         round (set-up, FP32 phase) on a stream of the device's
 *                         highest priority beside the FP64 branch, 0 at default
 *                         priority
 *   fp32_rows             FP32 kernels: output rows per thread of the tiled
 *                         kernel (4 or 8), or 0 for one trajectory per CTA
 *   fp32_slots            FP32 kernels: trajectories per CTA of the tiled kernel
 *                         (8..64, a multiple of 8; fewer when N is large or
 *                         shared memory is short).  The slots' node records are
 *                         staged in shared memory when they fit, else read from
 *                         global memory (then up to 512 threads per CTA)
 *   grid_cache            1: the body positions at the nodes of a round's new
 *                         segments are evaluated once per distinct node-time grid
 *                         (segments with the same start and length share one) and
 *                         copied; 0: evaluated for every segment
 * Defaults: 4, 1, 4, 8, 8, 1, 1, 4, 16, 1.  Profiling (pc_plan_set_profiling)
 * launches directly whatever `graphs` says. */
typedef struct {
  int setup_ctas_per_sm;
  int fp32_ctas_per_sm;
  int contract_ctas_per_sm;
  int rounds_per_batch;
  int repack_div;
  int graphs;
  int side_priority;
  int fp32_rows;
  int fp32_slots;
  int grid_cache;
} pc_tuning;

/* Reads / replaces the plan's tuning (PC_EINVAL on a value out of range). */
pc_status pc_plan_get_tuning(const pc_plan *plan, pc_tuning *out);
pc_status pc_plan_set_tuning(pc_plan *plan, const pc_tuning *t);

/* Autotuner: coordinate descent over the tuning fields (contraction CTAs,
 * set-up CTAs, FP32 tile shape and CTAs, side-branch priority, rounds per
 * batch, compaction threshold, graphs), each
 * candidate timed with CUDA events on a propagation of the caller's
 * trajectories x0 (device, planar [6][n_ic]) over [t0, tf] capped at
 * max_rounds sweep rounds (>= 16).  The fastest setting per round is kept in
 * the plan and copied to *best (may be NULL).  Allocates its own scratch
 * outputs; synchronizes `stream`.  Returns PC_OK, PC_EINVAL, PC_ENOMEM or
 * PC_ECUDA. */
pc_status pc_plan_autotune(pc_plan *plan, long long n_ic, const double *x0, double t0, double tf, int max_rounds,
                           pc_tuning *best, void *stream);

/* Uneven batching: n_groups groups of trajectories, group g propagated with
 * plans[g] (its own degree N, segment count and options) -- the paper's
 * two-level augmentation (Section "Two-level augmentation") with the outer
 * level keyed by degree.  The trajectories are one batch in planar layout,
 * group g at columns [counts[0] + .. + counts[g-1], + counts[g]) of
 *   x0, xf      device, planar [6][n_total]
 *   t0, tf      device [n_total]: each trajectory's own arc (tf < t0 backward)
 *   segments    device [n_total] base segment count per trajectory, or NULL
 *               (the plan's); per arc or per osculating period as the plan's
 *               seg_mode says
 *   status, iters, nseg   device [n_total] or NULL
 * Each group runs its own rounds (with its own compaction of finished
 * trajectories) on a stream of its plan, forked from and joined back to
 * `stream`; the host steps the groups in turn, so all groups keep the GPU busy
 * together.  A plan may appear once (its workspace serves one group).  An arc
 * outside a plan's ephemeris table sets PC_IC_OUT_OF_RANGE for that trajectory.
 * rounds: host, total sweep rounds over the groups, or NULL.
 * Returns PC_OK, PC_ENOTCONV, PC_EINVAL, PC_ENOMEM or PC_ECUDA. */
pc_status pc_propagate_groups(pc_plan *const *plans, int n_groups, const long long *counts, const double *x0,
                              const double *t0, const double *tf, const int *segments, double tol, double *xf,
                              int *status, int *iters, int *nseg, long long *rounds, void *stream);

/* ---- Reverse mode ----------------------------------------------------------
 * Gradients of the final state with respect to the initial state, through the
 * converged PC fixed point of every segment (the paper stops at the forward
 * propagation; its Conclusions name optimisation over the propagated states as
 * the use).  For a segment with converged nodes Y = 1 x0^T + omega2 K G(Y), a
 * cotangent ybar on its end state y_N gives
 *   x0bar = sum_j lambda_j,   lambda = Ybar + J^T (omega2 K^T lambda),
 * Ybar = ybar at node N, J = blockdiag(df/dy at the nodes); the linear adjoint
 * equation is swept like the forward one, from the last segment back.  The
 * segment schedule (including halvings) is held fixed: the result is the
 * derivative of the discrete map x0 -> xf that the forward pass computed. */

/* Forward pass that also records the tape the reverse sweep needs: for each
 * trajectory i and accepted segment k < max_seg, a record of 2 + 6(N+1)
 * doubles at tape[(i * max_seg + k) * (2 + 6(N+1))]:
 *   (t_a, t_b, y_0[6], y_1[6], ..., y_N[6])   -- the segment's converged nodes.
 *   x0, xf      device, planar [6][n_ic]
 *   t0, tf      device [n_ic], each trajectory's arc (tf < t0 backward)
 *   segments    device [n_ic] base segment counts, or NULL (the plan's)
 *   status      device [n_ic] PC_IC_* bits, or NULL
 *   nseg        device [n_ic], required: accepted segments (may exceed max_seg,
 *               in which case the tape misses the later ones and
 *               pc_adjoint_tape refuses it)
 *   tape        device, n_ic * max_seg * (2 + 6(N+1)) doubles, max_seg >= 1
 * Same rules and results as pc_propagate otherwise.  Returns PC_OK,
 * PC_ENOTCONV, PC_EINVAL, PC_ENOMEM or PC_ECUDA. */
pc_status pc_propagate_tape(pc_plan *plan, long long n_ic, const double *x0, const double *t0, const double *tf,
                            const int *segments, double tol, double *xf, int *status, int *nseg, int max_seg,
                            double *tape, void *stream);

/* Reverse sweep over a tape: x0_bar = (d xf / d x0)^T xf_bar per trajectory.
 *   nseg, tape   as written by pc_propagate_tape with the same plan and max_seg
 *   xf_bar       device, planar [6][n_ic], read only
 *   tol          stopping tolerance of the adjoint sweeps (<= 0: the plan's);
 *                the plan's stall rule applies, with twice its sweep cap
 *   x0_bar       device, planar [6][n_ic], written (may alias xf_bar)
 *   status       device [n_ic] or NULL: PC_IC_STALLED / NOT_CONVERGED / NONFINITE
 *                bits of the adjoint sweeps
 *   iters        device [n_ic] or NULL: adjoint sweeps spent
 * The call copies nseg to the host (it synchronizes `stream`) to order the
 * trajectories by segment count.  Returns PC_OK, PC_ENOTCONV (an adjoint
 * sweep hit its cap or blew up), PC_EINVAL (a count above max_seg, or a degree
 * whose tile does not fit in shared memory), PC_ENOMEM or PC_ECUDA. */
pc_status pc_adjoint_tape(pc_plan *plan, long long n_ic, const int *nseg, int max_seg, const double *tape,
                          const double *xf_bar, double tol, double *x0_bar, int *status, int *iters, void *stream);

/* Forward pass with a tape held by the plan, then the reverse sweep:
 * x0_bar = (d xf / d x0)^T xf_bar for the arc [t0, tf].  Device buffers,
 * planar [6][n_ic].  The tape (n_ic x segments x (2 + 6(N+1)) doubles) is
 * grown and the forward pass rerun if a trajectory needed more segments than
 * it had room for.  Synchronizes `stream`.  Returns PC_OK, PC_ENOTCONV,
 * PC_EINVAL, PC_ENOMEM or PC_ECUDA. */
pc_status pc_propagate_adjoint(pc_plan *plan, long long n_ic, const double *x0, double t0, double tf, double tol,
                               const double *xf_bar, double *x0_bar, void *stream);

/* b-plane coordinates (B.T, B.R) of n flybys of body `body` (index into the
 * plan's ephemeris, GM mu_body) at times t [n] from heliocentric states x
 * (planar [6][n]); the paper cites the b-plane without a formula.  With
 * rel = x - (r_b(t), v_b(t)) (body velocity = time derivative of its table
 * series), h = r x v, e_vec = ((v^2 - mu/|r|) r - (r.v) v)/mu, P = e_vec/e,
 * Q = (h/|h|) x P, incoming asymptote S = P/e + sqrt(e^2-1)/e Q,
 * T = S x z/|S x z| (z = (0,0,1)), R = S x T, B = S x h/v_inf.
 *   out      device planar [2][n] (B.T, B.R), or NULL
 *   jac      device planar [12][n]: d out_k / d x_q at row 6k + q, or NULL
 *   out_bar, x_bar   device planar [2][n] and [6][n]: x_bar = J^T out_bar
 *            (both or neither)
 * Forward-mode derivatives (exact to rounding).  A state that is not
 * hyperbolic with respect to the body gives NaN and PC_ENONFINITE. */
pc_status pc_bplane(pc_plan *plan, int body, double mu_body, long long n, const double *t, const double *x,
                    double *out, double *jac, const double *out_bar, double *x_bar, void *stream);

/* Copies the plan's operator K ((N+1) x (N+1), row-major) and nodes tau (N+1)
 * to host buffers (either may be NULL).  For tests and diagnostics. */
pc_status pc_plan_operator(const pc_plan *plan, double *K, double *tau);

/* Frees the plan (NULL is allowed).  Must not race with a call using it. */
void pc_plan_destroy(pc_plan *plan);

/* Static English description of a status code. */
const char *pc_status_string(pc_status s);

#ifdef __cplusplus
}
#endif
#endif /* PC_H_ */
