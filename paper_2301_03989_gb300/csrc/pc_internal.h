// Internal declarations of the GB300 batched Picard-Chebyshev library.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "pc.h"

namespace pcx {

constexpr int kMaxBodies = 32;
constexpr int kMaxN = 512;

// Trajectory phases.
enum : int { PH_ITER = 0, PH_DONE = 1 };

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
};

// Per-trajectory control state, structure of arrays of length ld, indexed by
// slot.  Active trajectories are packed into slots [0, A); ic[slot] is the
// trajectory's index in the caller's arrays.
struct Ctl {
  double *x;          // [6][ld] state at the start of the current segment
  double *hbase;      // base segment length
  double *ta, *tb, *w1, *w2;
  double *e_best;
  unsigned long long *err;  // this round's max change, as non-negative double bits
  long long *p;       // segment start, in units of hbase / 2^max_depth
  int *depth, *phase, *status, *sweeps, *seg_sweeps, *nstall, *nseg, *need_setup, *last, *ic;
};
constexpr int kCtlDoubles = 13;  // x[6] + hbase, ta, tb, w1, w2, e_best, spare
constexpr int kCtlInts = 10;

// Sweep parameters of one call.
struct Sweep {
  int N, n, kpad, rows_pad;  // degree, nodes, padded k extent, padded output rows (nodes 1..N)
  long long n_ic;
  int ld;                    // leading dimension over slots (multiple of 8)
  int A;                     // slots [0, A) may hold active trajectories
  double t0, tf, total, sgn;
  int segments, seg_mode, max_depth, max_iters, stall_sweeps, relative, warm;
  double tol, stall_factor, div_limit, trunc_tol;
  int max_ckpt;
  double *ckpt;              // [n_ic][max_ckpt][7] or nullptr
  // outputs, indexed by trajectory, written when a trajectory finishes
  double *xf;                // [6][n_ic]
  int *status, *iters, *nseg;
  // new-segment lists: setup of round r reads list (r & 1) and the control of
  // round r appends to list ((r + 1) & 1)
  int *list[2];
  int *list_cnt;             // [2]
  int list_cur;
};

struct Workspace {
  long long cap = 0;         // slots the buffers hold
  int ld = 0;
  double *Y[2] = {nullptr, nullptr};  // [n][6][ld]; the other buffer receives a repack
  double *G = nullptr;       // [kpad][6][ld]; rows n..kpad-1 stay zero
  double *E[2] = {nullptr, nullptr};    // [n][B][3][ld] body positions at the nodes (+ repack target)
  double *Aind[2] = {nullptr, nullptr}; // [n][3][ld] summed indirect acceleration (+ repack target)
  Ctl ctl[2]{};              // live control state and repack target
  void *ctl_block[2] = {nullptr, nullptr};
  int *lists = nullptr;      // 2 x ld slot lists
  int *ints = nullptr;       // [0..1] done counters [finished, stopped], [2..3] list counts, [4] repack count
  int *pos = nullptr;        // [ld] repack destinations
  int *h_ints = nullptr;     // pinned host mirror: 2 slots of 8 ints, [16] repack count
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int live = 0;              // which of E/Aind/ctl is live
};

}  // namespace pcx

struct pc_plan {
  int N = 0, n = 0, kpad = 0, rows_pad = 0;
  int segments = 0;
  pc_options opt{};
  int device = 0;
  // model (device copies)
  pcx::Model model{};
  double *d_mu = nullptr, *d_coef = nullptr;
  // operator: rows are nodes 1..N (row r <-> node r+1), padded to rows_pad x kpad, zeros outside
  double *d_K = nullptr;
  double *d_tau = nullptr;   // [n]
  double *h_K = nullptr;     // host copy, (N+1) x (N+1)
  double *h_tau = nullptr;   // [n]
  pcx::Workspace ws;
  // per-kernel timing: 5 events per recorded round (before setup, force,
  // contract, control, after control)
  int prof_on = 0;
  std::vector<cudaEvent_t> prof_ev;
  long long prof_rounds = 0;
};

namespace pcx {
// pc_plan.cu
pc_status ensure_workspace(pc_plan *plan, long long n_ic);
void free_workspace(pc_plan *plan);
// pc_sweep.cu
cudaError_t launch_init(const pc_plan *plan, const Sweep &s, const double *x0, cudaStream_t st);
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
}  // namespace pcx
