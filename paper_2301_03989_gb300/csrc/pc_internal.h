// Internal declarations of the GB300 batched Picard-Chebyshev library.
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "pc.h"

namespace pcx {

constexpr int kMaxBodies = 32;
constexpr int kMaxN = 512;
constexpr int kMaxNpl = 9;   // mixed precision: N + 1 <= 32 * kMaxNpl (N <= 287)

// Floats per node of an FP32 record (mixed precision), in float4 groups.
// New segment (k_fp32): (r_K, mu_c/|r_K|^3), (v_K, -), (indirect term, -),
// then one (r_K - r_b, -) per body from float 12.  Correction solve
// (k_corr32): (r, mu_c/|r|^3), (v, -), (residual 0..3), (residual 4..5, -, -),
// then one (r - r_b, mu_b/|r - r_b|^3) per body from float 16.  Shared by the
// allocation and the kernels.
__host__ __device__ constexpr int x32_stride(int B) { return 16 + 4 * B; }

// Split-digit FP64 contraction (PC_CONTRACT_SPLIT).  A value v of a column
// (or operator row) whose largest biased exponent is Bc is written as
// v = 2^(Bc - 1021) sum_{a=1..7} d_a 2^(-8a) with integer digits |d_a| <= 128
// (balanced base 256, the last one rounded to nearest): the 53-bit mantissa
// shifted to 55 bits of fixed point, then cut into bytes from the bottom.  A
// digit is exact in bf16, a product of two in FP32, and the sum over up to 129
// nodes of the products on one anti-diagonal a + b = d (at most 7 of them)
// stays below 2^24, so the bf16 tensor cores add them without rounding.
constexpr int kSplitDigits = 7;
__host__ __device__ inline void split_digits7(double v, int Bc, int d[kSplitDigits]) {
  unsigned long long b;
  memcpy(&b, &v, sizeof(b));
  const int be = (int)((b >> 52) & 0x7ff);
  long long M = 0;
  if (be != 0 && be != 0x7ff) {
    const unsigned long long m = (b & ((1ULL << 52) - 1)) | (1ULL << 52);
    const int sh = Bc - be - 2;  // >= -2 since be <= Bc: M < 2^55
    if (sh <= 0) M = (long long)(m << (-sh));
    else if (sh < 63) M = (long long)((m + (1ULL << (sh - 1))) >> sh);
    if (b >> 63) M = -M;
  }
  for (int a = kSplitDigits - 1; a >= 1; a--) {
    int r = (int)(M & 255);
    if (r >= 128) r -= 256;
    d[a] = r;
    M = (M - r) >> 8;
  }
  d[0] = (int)M;
}

// Trajectory phases: FP64 sweeps, finished, FP32 sweeps (mixed precision).
// PH_READY64: the FP32 phase ended in this round's k_fp32; the control kernel
// moves the trajectory to PH_ITER and onto the next round's FP64 list.
// PH_CORR32: after an FP64 sweep, the next round's k_corr32 solves in FP32 for
// the correction to the iterate, then the trajectory goes PH_READY64.
enum : int { PH_ITER = 0, PH_DONE = 1, PH_ITER32 = 2, PH_READY64 = 3, PH_CORR32 = 4 };

// Segment-attempt outcomes.
enum : int { SEG_CONTINUE = -1, SEG_OK = 0, SEG_STALLED = 1, SEG_FAIL_CAP = 2, SEG_FAIL_DIV = 3, SEG_FAIL_TRUNC = 4 };

// Read-only model data shared by every kernel (device pointers + scalars).
struct Model {
  int B;              // perturbing bodies
  double mu_c;        // central GM
  const double *mu;   // [B]
  int indirect;
  double t_begin, granule;
  int deg, n_gr;
  const double *coef; // [B][n_gr][3][deg+1]
  double c_light;     // > 0: Einstein-Infeld-Hoffmann terms in the FP64 force
};
// Per node, with the EIH terms: for the central body (0) and each table body
// (1..B) its barycentric velocity (3), Newtonian acceleration (3) and
// potential (1) from the other bodies.
__host__ __device__ constexpr int eih_stride(int B) { return 7 * (B + 1); }

// Per-trajectory control state, structure of arrays of length ld, indexed by
// slot.  Active trajectories are packed into slots [0, A); ic[slot] is the
// trajectory's index in the caller's arrays.
struct Ctl {
  double *x;          // [6][ld] state at the start of the current segment
  double *t0, *tf;    // the trajectory's arc
  double *total, *sgn;  // |tf - t0| and sign(tf - t0)
  double *hbase;      // base segment length
  double *ta, *tb, *w1, *w2;
  double *e_best;
  unsigned long long *err;  // this round's max change (FP64 phase), non-negative double bits
  long long *p;       // segment start, in units of hbase / 2^max_depth
  int *depth, *phase, *status, *sweeps, *seg_sweeps, *nstall, *nseg, *need_setup, *last, *ic;
  unsigned *err32;    // final FP32-phase change of a trajectory whose FP32 phase blew up
  int *ncorr;         // FP32 correction solves in the current segment attempt
  double *kc;         // [kKeplerConsts][ld] warm-start constants of the segment's start state
};
constexpr int kKeplerConsts = 11;
constexpr int kCtlDoubles = 16 + kKeplerConsts;  // x[6] + t0, tf, total, sgn, hbase, ta, tb, w1, w2, e_best, kc
constexpr int kCtlInts = 12;     // 10 ints + err32 + ncorr

// Sweep parameters of one call.
constexpr int kKepNodes = 17;  // interpolation nodes of the warm start

struct Sweep {
  int N, n, kpad, rows_pad;  // degree, nodes, padded k extent, padded output rows (nodes 1..N)
  int order;                 // 1: the paper's sweep; 2: its second-order form
  int kep_stride;            // warm start solved at nodes 0, kep_stride, ..., N (0: at every node)
  const float *Lint;         // [2][n][17] interpolation weights (kep_stride > 0) as FP32 pairs hi + lo
  float *YK17;               // [17][6][ld] float2 (hi, lo): Kepler solutions at those nodes minus the
                             // start state as FP32 pairs
  // Ephemeris of the round's new segments, evaluated once per distinct node-
  // time grid (w1, w2): an open-addressing table per round parity maps a grid
  // to its owning list entry and its index u in the cache EC.
  int eh_size;               // table slots, a power of two >= 2 ld (0: no cache)
  int eh_cap;                // grids the cache holds; grids beyond it are evaluated per entry
  int *eh_tab[2];            // [eh_size] owning list entry, -1 when free
  int *eh_uid[2];            // [eh_size] the owner's grid index u, -1 beyond eh_cap
  int *eh_ent;               // [ld] table slot of each list entry (-1: none)
  int *eh_own;               // [eh_cap] owning list entry of grid u
  int *eh_cnt;               // [2] grids of the round, by parity (cleared by the set-up kernel)
  double *EC;                // [n][3B + 3][eh_cap] body positions and summed indirect term by grid
  long long n_ic;
  int ld;                    // leading dimension over slots (multiple of 8)
  int A;                     // slots [0, A) may hold active trajectories
  // arcs: per trajectory from t0a / tfa / sega when given, else t0s / tfs / segments
  double t0s, tfs;
  const double *t0a, *tfa;
  const int *sega;
  // caller arrays hold this call's trajectories at columns io_off .. io_off + n_ic - 1
  // of planar arrays with leading dimension io_ld
  long long io_ld, io_off;
  int segments, seg_mode, max_depth, max_iters, stall_sweeps, relative, warm;
  double tol, stall_factor, div_limit, trunc_tol;
  double mu_c;               // central GM (warm-start constants)
  int mixed;                 // 1: segments start with FP32 sweeps
  double switch_tol;         // FP32 -> FP64 when the FP32 change is below this
  int refine;                // 1: FP32 correction solves between FP64 sweeps
  int max_corr;              // correction solves per segment attempt
  double corr_hi;            // an FP64 change below this may be followed by a correction solve
  int max_ckpt;
  double *ckpt;              // [n_ic][max_ckpt][7] or nullptr
  // adjoint checkpoints: per trajectory and accepted segment k < tape_seg a record
  // (t_a, t_b, y_j[6] for j = 0..N) of tape_rec() doubles, or nullptr
  int tape_seg;
  double *tape;              // [n_ic][tape_seg][2 + 6n]
  // outputs, indexed by trajectory, written when a trajectory finishes
  double *xf;                // [6][n_ic]
  int *status, *iters, *nseg;
  // Per-round lists, double-buffered by round parity: round r reads list
  // [r & 1] and its control kernel fills list [(r + 1) & 1].
  int *list[2];              // trajectories starting a new segment (setup)
  int *list_cnt;             // [2]
  int *l64[2];               // trajectories doing an FP64 sweep
  int *l64_cnt;              // [2]
  int *lc[2];                // trajectories doing an FP32 correction solve
  int *lc_cnt;               // [2]
  int list_cur;
  int *tile_ctr;             // dynamic tile counter of the FP64 contraction
  int *tile_ctr2;            // the same for the position pass of a second-order sweep
  int *fp32_ctr;             // [2] list-entry counters of the tiled FP32 kernels (new segment, correction),
                             // cleared by the round's set-up kernel
  unsigned long long *cnt64; // [0] FP64, [1] FP32 trajectory-sweeps of this call
};

struct Workspace {
  long long cap = 0;         // slots the buffers hold
  int ld = 0;
  double *Y[2] = {nullptr, nullptr};  // [n][6][ld] FP64 iterate (current / next; also repack target)
  double *G = nullptr;       // [kpad][6][ld]; rows n..kpad-1 stay zero
  double *tails = nullptr;   // [ceil(n/8)][14][ld] resolution-test partial sums of the round's FP64 sweeps
  double *E[2] = {nullptr, nullptr};    // [n][B][3][ld] body positions at the nodes (+ repack target)
  double *Aind[2] = {nullptr, nullptr}; // [n][3][ld] summed indirect acceleration (+ repack target)
  double *EX[2] = {nullptr, nullptr};   // [n][eih_stride(B)][ld] bodies' EIH data (c_light > 0; + repack target)
  // mixed precision (allocated when the plan asks for it), by new-segment list entry
  double *YK = nullptr;      // [entry][n][6] FP64 warm start
  float *YK17 = nullptr;     // [17][6][ld] float2 Kepler deviations at the interpolation nodes (FP32 pairs),
                             // by new-segment entry
  // per-round ephemeris cache (model with bodies): tables by parity, per-entry
  // slots, grid owners and the cache itself
  int eh_size = 0, eh_cap = 0;
  int *eh_tab = nullptr;     // [2][eh_size] owners, then [2][eh_size] grid indices
  int *eh_ent = nullptr;     // [ld]
  int *eh_own = nullptr;     // [eh_cap]
  double *EC = nullptr;      // [n][3B + 3][eh_cap]
  float *X32 = nullptr;      // [entry][n][x32_stride(B)] FP32 node records
  float *R32[2] = {nullptr, nullptr};   // [n][6][ld] FP64 sweep residual Y' - Y, rounded (+ repack target)
  Ctl ctl[2]{};              // live control state and repack target
  void *ctl_block[2] = {nullptr, nullptr};
  int *lists = nullptr;      // 6 x ld: setup lists [2], FP64 lists [2], correction lists [2]
  int *ints = nullptr;       // [0..1] done counters [finished, stopped], [2..3] setup list counts,
                             // [4] repack count, [5..6] FP64 list counts, [7] tile counter,
                             // [8..9] correction list counts, [10..11] FP32 list-entry counters,
                             // [12] tile counter of the second-order position pass,
                             // [13..14] ephemeris-cache grid counts
  int *pos = nullptr;        // [ld] repack destinations
  unsigned long long *cnt64 = nullptr;  // [0] FP64 trajectory-sweeps, [1] FP32 trajectory-sweeps
  unsigned long long *h_cnt64 = nullptr;
  int *h_ints = nullptr;     // pinned host mirror: 2 slots of 8 ints, [16] repack count
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // CUDA graph of one batch of rounds, valid for one (call, working-set shape)
  cudaGraphExec_t graph = nullptr;
  long long graph_key[5] = {-1, -1, -1, -1, -1};
  long long graph_launches = 0;  // kernels per replay
  int live = 0;              // which of E/Aind/ctl/YK/... is live
  int mixed = 0;             // mixed-precision buffers present
};

}  // namespace pcx

// Reverse-sweep workspace (pc_adjoint.cu).
struct AdjWorkspace {
  long long cap = 0;
  int *perm = nullptr;       // [cap] trajectories by segment count, descending
  double *xb = nullptr;      // [6][cap] running cotangent
  double *xf = nullptr;      // [6][cap] forward result of pc_propagate_adjoint
  int *nseg = nullptr;       // [cap]
  int *fail = nullptr;       // [1]
  int *h_fail = nullptr;     // pinned
  double *tape = nullptr;    // pc_propagate_adjoint's own tape
  size_t tape_bytes = 0;
  int tape_hint = 0;         // segment capacity that sufficed last time
};

struct pc_plan {
  int N = 0, n = 0, kpad = 0, rows_pad = 0;
  int segments = 0;
  pc_options opt{};
  pc_tuning tune{4, 1, 4, 8, 8, 1, 1, 4, 16, 1};
  long long session_id = 0;  // distinguishes calls for the graph cache
  int device = 0;
  // model (device copies)
  pcx::Model model{};
  double *d_mu = nullptr, *d_coef = nullptr;
  float *d_mu32 = nullptr;   // GMs rounded to FP32 (mixed precision)
  // operator: rows are nodes 1..N (row r <-> node r+1), padded to rows_pad x kpad, zeros outside
  double *d_K = nullptr;
  float *d_K32T = nullptr;   // the operator rounded to FP32 and transposed, [N+1][32 npl]
  int npl = 0;               // ceil((N+1)/32): K32T rows are 32 npl floats long (0: no mixed path)
  float *d_K32R = nullptr;   // tiled FP32 kernels: [N+1][rows32], K32R[k][r] = K[r+1][k], zero-padded
  // split-digit contraction: the operator rows' digits (rows = nodes 1..N) as
  // bf16 mma B fragments [n_nt][n_ks][7 digits][32 lanes] x 2 words, and each
  // row's largest biased exponent
  // warm start: Kepler's equation solved at every kep_stride-th node (the 17
  // nodes of the embedded degree-16 Chebyshev-Lobatto grid), the other nodes
  // interpolated with d_Lint [N+1][17]; kep_stride 0: solved at every node
  int kep_stride = 0;
  float *d_Lint = nullptr;
  unsigned *d_Kdig = nullptr;
  int *d_Kexp = nullptr;
  int split_nt = 0, split_ks = 0;   // ceil(N/8) node tiles, ceil((N+1)/16) k-steps
  int rows32 = 0;            // 32 ceil(N/32)
  double *d_tau = nullptr;   // [n]
  double *h_K = nullptr;     // host copy, (N+1) x (N+1)
  double *h_tau = nullptr;   // [n]
  pcx::Workspace ws;
  // adjoint: the operator transposed without its zero row, KTp[j][k'] = K[k'+1][j]
  // (j < N+1, k' < N), zero-padded to adj_mpad = 16 ceil((N+1)/16) rows and
  // adj_kpad = 4 ceil(N/4) columns
  double *d_KTp = nullptr;
  int adj_mpad = 0, adj_kpad = 0;
  int num_sms = 0;
  AdjWorkspace adj;
  // per-kernel timing: 6 events per recorded round (before setup, force,
  // contract, the FP32 kernels, control, after control)
  cudaStream_t own_stream = nullptr;  // created for multi-group calls and default-stream callers
  cudaEvent_t fork_ev = nullptr;      // orders own_stream after a default-stream caller
  // mixed precision: the new-segment branch of a round (set-up, FP32 phase) runs
  // on side_stream beside the FP64 branch (force, contraction)
  cudaStream_t side_stream = nullptr;
  int side_stream_prio = -1;          // side_priority the side stream was created with
  cudaEvent_t branch_ev[2] = {nullptr, nullptr};  // fork, join
  int prof_on = 0;
  std::vector<cudaEvent_t> prof_ev;
  long long prof_rounds = 0;
  long long acc_sweeps64 = 0, acc_sweeps32 = 0;  // since the last pc_plan_kernel_times
  mutable long long acc_launches = 0;
};

namespace pcx {
// pc_plan.cu
pc_status ensure_workspace(pc_plan *plan, long long n_ic, int mixed);
void free_workspace(pc_plan *plan);
// pc_adjoint.cu
void free_adjoint_workspace(pc_plan *plan);
// pc_api.cu
pc_status propagate_with_tape(pc_plan *p, long long n_ic, const double *x0, double t0s, double tfs,
                              const double *t0a, const double *tfa, const int *sega, double tol, double *xf,
                              int *status, int *iters, int *nseg, int tape_seg, double *tape, cudaStream_t st);
__host__ __device__ inline int tape_rec(int n) { return 2 + 6 * n; }
// pc_sweep.cu
cudaError_t launch_init(const pc_plan *plan, const Sweep &s, const double *x0, cudaStream_t st);
// Function attributes the round's kernels need (set outside any stream capture).
cudaError_t prepare_launches(const pc_plan *plan);
cudaError_t launch_round(const pc_plan *plan, const Sweep &s, int cur, cudaStream_t st,
                         cudaEvent_t *ev /* 5 events or nullptr */);
// Moves the active slots of [0, s.A) to the front of the spare buffers (Y[cur]
// -> Y[cur^1], E, Aind, control) and rebuilds list s.list_cur; the new count
// lands in ints[4].  The caller then flips cur and ws.live.
cudaError_t launch_repack(const pc_plan *plan, const Sweep &s, int cur, cudaStream_t st);
// Trajectories still active after the round cap: flagged NOT_CONVERGED, outputs written.
cudaError_t launch_abort(const pc_plan *plan, const Sweep &s, cudaStream_t st);
cudaError_t launch_eval_ephemeris(const pc_plan *plan, long long n_pts, const double *t, double *rb, cudaStream_t st);
cudaError_t launch_eval_dynamics(const pc_plan *plan, long long n_pts, const double *t, const double *y, double *f,
                                 cudaStream_t st);
cudaError_t launch_eval_warm(const pc_plan *plan, long long n_pts, const double *x0, const double *dt, double *x,
                             cudaStream_t st);
cudaError_t launch_apply_operator(const pc_plan *plan, long long n_ic, int ld, const double *x0, const double *G,
                                  double *Y, cudaStream_t st);
// pc_split.cu: the FP64 contraction by exact digit products on the bf16 tensor
// cores: over the round's FP64 list, Y' = x0 + K G with the change and the
// residual (SPLIT_FIRST_ORDER), or its second-order form in two passes, the
// second pass reading omega2 V' from G's velocity rows (SPLIT_SECOND_ORDER);
// or over columns 0..n_ic-1, Y' only (SPLIT_DIAG).
enum : int { SPLIT_FIRST_ORDER = 0, SPLIT_DIAG = 1, SPLIT_SECOND_ORDER = 2 };
cudaError_t launch_contract_split(const pc_plan *plan, const Sweep &s, const Ctl &c, double *G,
                                  const double *Yold, double *Ynew, float *R32, int mode, cudaStream_t st);
cudaError_t prepare_split(const pc_plan *plan);
bool split_supported(const pc_plan *plan);
}  // namespace pcx
