// Host driver of the batched sweep and the kernel-level entry points.
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "pc_internal.h"

using namespace pcx;

namespace {

pc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PC_OK;
  return e == cudaErrorMemoryAllocation ? PC_ENOMEM : PC_ECUDA;
}

}  // namespace

namespace {

// One propagation in flight on one plan: the host side of the round loop.
// begin() sets the call up and launches the initialisation, step() queues a
// batch of rounds and looks at the previous batch's counters (repacking the
// working set when 1/8 of it has finished), finish() closes the call.  The
// multi-group entry point steps several sessions in turn on their own streams.
struct Session {
  pc_plan *p = nullptr;
  Sweep s{};
  cudaStream_t st = nullptr;      // where the rounds run
  cudaStream_t caller = nullptr;  // the caller's stream, when st is the plan's own
  bool forked = false;
  cudaError_t e = cudaSuccess;
  long long n_ic = 0, rounds = 0, max_rounds = 0;
  int cur = 0, pending = -1, done_known = 0;
  bool finished = false, capped = false;
};

struct Arcs {
  double t0s, tfs;          // scalar arc (when the arrays are NULL)
  const double *t0a, *tfa;  // device, per trajectory, or NULL
  const int *sega;          // device, per trajectory, or NULL
};

pc_status session_begin(Session &S, pc_plan *p, long long n_ic, long long io_ld, long long io_off, const double *x0,
                        const Arcs &arcs, double tol, double *xf, int *status, int *iters, int *nseg, int max_ckpt,
                        double *ckpt, int tape_seg, double *tape, cudaStream_t st) {
  const pc_options &o = p->opt;
  const int mixed = o.precision == PC_PREC_MIXED ? 1 : 0;
  pc_status ps = ensure_workspace(p, n_ic, mixed);
  if (ps != PC_OK) return ps;
  Workspace &w = p->ws;
  Sweep &s = S.s;
  s = Sweep{};
  s.N = p->N;
  s.n = p->n;
  s.kpad = p->kpad;
  s.rows_pad = p->rows_pad;
  s.n_ic = n_ic;
  s.ld = w.ld;
  s.t0s = arcs.t0s;
  s.tfs = arcs.tfs;
  s.t0a = arcs.t0a;
  s.tfa = arcs.tfa;
  s.sega = arcs.sega;
  s.io_ld = io_ld;
  s.io_off = io_off;
  s.segments = p->segments;
  s.seg_mode = o.seg_mode;
  s.max_depth = o.max_depth;
  s.max_iters = o.max_iters;
  s.stall_sweeps = o.stall_sweeps;
  s.relative = o.relative;
  s.warm = o.warm_start;
  s.tol = tol > 0.0 ? tol : o.tol;
  s.stall_factor = o.stall_factor;
  s.div_limit = o.div_limit;
  s.trunc_tol = o.trunc_tol;
  s.max_ckpt = max_ckpt;
  s.ckpt = max_ckpt > 0 ? ckpt : nullptr;
  s.tape_seg = tape_seg;
  s.tape = tape_seg > 0 ? tape : nullptr;
  s.xf = xf;
  s.status = status;
  s.iters = iters;
  s.nseg = nseg;
  s.mixed = mixed;
  s.switch_tol = o.switch_tol;
  s.refine = mixed && o.refine32;
  s.mu_c = p->model.mu_c;
  s.max_corr = 2;
  s.corr_hi = 1e-3;
  s.list[0] = w.lists;
  s.list[1] = w.lists + w.ld;
  s.list_cnt = w.ints + 2;
  s.l64[0] = w.lists + 2 * (size_t)w.ld;
  s.l64[1] = w.lists + 3 * (size_t)w.ld;
  s.l64_cnt = w.ints + 5;
  s.lc[0] = w.lists + 4 * (size_t)w.ld;
  s.lc[1] = w.lists + 5 * (size_t)w.ld;
  s.lc_cnt = w.ints + 8;
  s.tile_ctr = w.ints + 7;
  s.tile_ctr2 = w.ints + 12;
  s.fp32_ctr = w.ints + 10;
  s.order = o.order;
  s.kep_stride = p->kep_stride;
  s.Lint = p->d_Lint;
  s.YK17 = w.YK17;
  s.eh_size = (w.EC && p->tune.grid_cache) ? w.eh_size : 0;
  s.eh_cap = w.eh_cap;
  s.eh_tab[0] = w.eh_tab;
  s.eh_tab[1] = w.eh_tab + w.eh_size;
  s.eh_uid[0] = w.eh_tab + 2 * (size_t)w.eh_size;
  s.eh_uid[1] = w.eh_tab + 3 * (size_t)w.eh_size;
  s.eh_ent = w.eh_ent;
  s.eh_own = w.eh_own;
  s.eh_cnt = w.ints + 13;
  s.EC = w.EC;
  s.cnt64 = w.cnt64;
  s.list_cur = 0;
  s.A = (int)n_ic;
  w.live = 0;
  S.p = p;
  S.st = st;
  S.caller = st;
  S.forked = false;
  // A default stream cannot be captured into a graph: run on the plan's own
  // stream, ordered after the caller's work by an event (joined back at finish).
  if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) {
    cudaError_t e = cudaSuccess;
    if (!p->own_stream) e = cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !p->fork_ev) e = cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(p->fork_ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->own_stream, p->fork_ev, 0);
    if (e != cudaSuccess) return cuda_status(e);
    S.st = p->own_stream;
    S.forked = true;
  }
  st = S.st;
  S.n_ic = n_ic;
  S.rounds = 0;
  S.max_rounds = o.max_rounds > 0 ? o.max_rounds : 10000000LL;
  S.cur = 0;
  S.pending = -1;
  S.done_known = 0;
  S.finished = S.capped = false;
  p->session_id += 1;  // a new call: kernel arguments differ, no cached graph applies
  S.e = prepare_launches(p);
  if (S.e == cudaSuccess && mixed && p->side_stream && p->side_stream_prio != p->tune.side_priority) {
    S.e = cudaStreamSynchronize(p->side_stream);
    cudaStreamDestroy(p->side_stream);
    p->side_stream = nullptr;
  }
  if (S.e == cudaSuccess && mixed && !p->side_stream) {
    int least = 0, greatest = 0;
    S.e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (S.e == cudaSuccess)
      S.e = cudaStreamCreateWithPriority(&p->side_stream, cudaStreamNonBlocking,
                                         p->tune.side_priority ? greatest : 0);
    p->side_stream_prio = p->tune.side_priority;
  }
  for (int k = 0; k < 2 && S.e == cudaSuccess && mixed; k++)
    if (!p->branch_ev[k]) S.e = cudaEventCreateWithFlags(&p->branch_ev[k], cudaEventDisableTiming);
  if (S.e == cudaSuccess) S.e = launch_init(p, s, x0, st);
  return S.e == cudaSuccess ? PC_OK : cuda_status(S.e);
}

// One batch of R rounds as a CUDA graph.  The rounds' kernel arguments depend
// only on the call, the working-set size and the buffer parities, so the graph
// is captured once per (call, A, parities) and replayed until a compaction
// changes them.
cudaError_t run_batch_graph(Session &S, int R) {
  pc_plan *p = S.p;
  Workspace &w = p->ws;
  Sweep &s = S.s;
  const long long key[5] = {p->session_id, s.A, S.cur, s.list_cur, (long long)w.live * 1024 + R};
  cudaError_t e = cudaSuccess;
  if (!w.graph || !std::equal(key, key + 5, w.graph_key)) {
    if (w.graph) {
      cudaGraphExecDestroy(w.graph);
      w.graph = nullptr;
    }
    e = cudaStreamBeginCapture(S.st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const long long l0 = p->acc_launches;
    Sweep sc = s;
    int cc = S.cur;
    cudaError_t le = cudaSuccess;
    for (int r = 0; r < R && le == cudaSuccess; r++) {
      le = launch_round(p, sc, cc, S.st, nullptr);
      cc ^= 1;
      sc.list_cur ^= 1;
    }
    w.graph_launches = p->acc_launches - l0;
    p->acc_launches = l0;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(S.st, &g);
    if (e == cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&w.graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      w.graph = nullptr;
      return e;
    }
    std::copy(key, key + 5, w.graph_key);
  }
  e = cudaGraphLaunch(w.graph, S.st);
  p->acc_launches += w.graph_launches;
  return e;
}

void session_step(Session &S) {
  if (S.finished || S.e != cudaSuccess) return;
  pc_plan *p = S.p;
  Sweep &s = S.s;
  Workspace &w = p->ws;
  cudaError_t &e = S.e;
  const int R = p->tune.rounds_per_batch;
  if (p->tune.graphs && !p->prof_on && (R % 2) == 0 && s.A > 0) {
    // replay: an even number of rounds returns both parities to where they were
    e = run_batch_graph(S, R);
    S.rounds += R;
  }
  for (int r = 0; r < R && e == cudaSuccess && s.A > 0 && !(p->tune.graphs && !p->prof_on && (R % 2) == 0);
       r++) {
    cudaEvent_t *ev = nullptr;
    if (p->prof_on) {
      const size_t need = (size_t)(p->prof_rounds + 1) * 6;
      while (e == cudaSuccess && p->prof_ev.size() < need) {
        cudaEvent_t x;
        e = cudaEventCreate(&x);
        if (e == cudaSuccess) p->prof_ev.push_back(x);
      }
      if (e != cudaSuccess) return;
      ev = p->prof_ev.data() + (size_t)p->prof_rounds * 6;
      p->prof_rounds++;
    }
    e = launch_round(p, s, S.cur, S.st, ev);
    S.cur ^= 1;
    s.list_cur ^= 1;
    S.rounds++;
  }
  if (e != cudaSuccess) return;
  const int slot = (S.pending < 0) ? 0 : (S.pending ^ 1);
  e = cudaMemcpyAsync(w.h_ints + 8 * slot, w.ints, 8 * sizeof(int), cudaMemcpyDeviceToHost, S.st);
  if (e == cudaSuccess) e = cudaEventRecord(w.ev[slot], S.st);
  if (e != cudaSuccess) return;
  if (S.pending >= 0) {
    e = cudaEventSynchronize(w.ev[S.pending]);
    if (e != cudaSuccess) return;
    S.done_known = w.h_ints[8 * S.pending];
    if (S.done_known >= S.n_ic) S.finished = true;
  }
  S.pending = slot;
  if (S.finished) return;
  if (S.rounds >= S.max_rounds) {
    S.capped = true;
    S.finished = true;
    return;
  }
  // Compaction: when at least 1/repack_div of the slots hold finished trajectories,
  // move the active ones to the front so later rounds launch over fewer slots
// (with the default repack_div of 8).
  const long long active = S.n_ic - S.done_known;
  const long long dead = (long long)s.A - active;
  if (dead > 0 && dead * p->tune.repack_div >= (long long)s.A) {
    e = launch_repack(p, s, S.cur, S.st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.h_ints + 16, w.ints + 4, sizeof(int), cudaMemcpyDeviceToHost, S.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S.st);
    if (e != cudaSuccess) return;
    s.A = w.h_ints[16];
    S.cur ^= 1;
    w.live ^= 1;
    S.pending = -1;
    if (s.A == 0) S.finished = true;
  }
}

pc_status session_finish(Session &S, long long *rounds_out) {
  pc_plan *p = S.p;
  Workspace &w = p->ws;
  cudaError_t e = S.e;
  if (e == cudaSuccess && S.capped) e = launch_abort(p, S.s, S.st);
  // aggregate: did any trajectory stop early?
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.h_ints, w.ints, 8 * sizeof(int), cudaMemcpyDeviceToHost, S.st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.h_cnt64, w.cnt64, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, S.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S.st);
  if (e == cudaSuccess && S.forked) {
    e = cudaEventRecord(p->fork_ev, S.st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S.caller, p->fork_ev, 0);
  }
  if (rounds_out) *rounds_out += S.rounds;
  if (e != cudaSuccess) return cuda_status(e);
  p->acc_sweeps64 += (long long)w.h_cnt64[0];
  p->acc_sweeps32 += (long long)w.h_cnt64[1];
  if (S.capped || w.h_ints[1] > 0) return PC_ENOTCONV;
  return PC_OK;
}

}  // namespace

extern "C" pc_status pc_propagate_ex(pc_plan *p, long long n_ic, const double *x0, double t0, double tf,
                                     double tol, double *xf, int *status, int *iters, int *nseg, int max_ckpt,
                                     double *ckpt, long long *rounds_out, void *stream) {
  if (rounds_out) *rounds_out = 0;
  if (!p || n_ic < 0) return PC_EINVAL;
  if (n_ic == 0) return PC_OK;
  if (!x0 || !xf || !std::isfinite(t0) || !std::isfinite(tf) || max_ckpt < 0 || (max_ckpt > 0 && !ckpt))
    return PC_EINVAL;
  if (n_ic > (1LL << 30)) return PC_EINVAL;
  const Model &md = p->model;
  if (md.B > 0) {
    const double lo = md.t_begin, hi = md.t_begin + md.granule * md.n_gr;
    if (std::fmin(t0, tf) < lo || std::fmax(t0, tf) > hi) return PC_EINVAL;
  }
  Session S;
  const Arcs arcs{t0, tf, nullptr, nullptr, nullptr};
  pc_status ps = session_begin(S, p, n_ic, n_ic, 0, x0, arcs, tol, xf, status, iters, nseg, max_ckpt, ckpt, 0,
                               nullptr, (cudaStream_t)stream);
  if (ps != PC_OK) return ps;
  while (!S.finished && S.e == cudaSuccess) session_step(S);
  return session_finish(S, rounds_out);
}

namespace pcx {
// One-group propagation with per-trajectory or scalar arcs that records the
// adjoint tape (pc_adjoint.cu).
pc_status propagate_with_tape(pc_plan *p, long long n_ic, const double *x0, double t0s, double tfs,
                              const double *t0a, const double *tfa, const int *sega, double tol, double *xf,
                              int *status, int *iters, int *nseg, int tape_seg, double *tape, cudaStream_t st) {
  Session S;
  const Arcs arcs{t0s, tfs, t0a, tfa, sega};
  pc_status ps = session_begin(S, p, n_ic, n_ic, 0, x0, arcs, tol, xf, status, iters, nseg, 0, nullptr, tape_seg,
                               tape, st);
  if (ps != PC_OK) return ps;
  while (!S.finished && S.e == cudaSuccess) session_step(S);
  return session_finish(S, nullptr);
}
}  // namespace pcx

extern "C" pc_status pc_propagate(pc_plan *p, long long n_ic, const double *x0, double t0, double tf, double tol,
                                  double *xf, int *status, int *iters, void *stream) {
  return pc_propagate_ex(p, n_ic, x0, t0, tf, tol, xf, status, iters, nullptr, 0, nullptr, nullptr, stream);
}

extern "C" pc_status pc_propagate_groups(pc_plan *const *plans, int n_groups, const long long *counts,
                                         const double *x0, const double *t0, const double *tf, const int *segments,
                                         double tol, double *xf, int *status, int *iters, int *nseg,
                                         long long *rounds_out, void *stream) {
  if (rounds_out) *rounds_out = 0;
  if (!plans || n_groups < 1 || n_groups > 64 || !counts || !t0 || !tf) return PC_EINVAL;
  long long total = 0;
  for (int g = 0; g < n_groups; g++) {
    if (!plans[g] || counts[g] < 0) return PC_EINVAL;
    for (int h = 0; h < g; h++)
      if (plans[h] == plans[g] && counts[g] > 0 && counts[h] > 0) return PC_EINVAL;  // one workspace per group
    total += counts[g];
  }
  if (total == 0) return PC_OK;
  if (!x0 || !xf || total > (1LL << 30)) return PC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // fork: every group waits for the caller's stream, runs on its plan's own
  // stream, and the caller's stream waits for all groups at the end
  cudaEvent_t fork = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(fork, st);
  std::vector<Session> S(n_groups);
  pc_status result = PC_OK;
  long long off = 0;
  for (int g = 0; g < n_groups && e == cudaSuccess; g++) {
    pc_plan *p = plans[g];
    if (counts[g] > 0) {
      if (!p->own_stream) e = cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(p->own_stream, fork, 0);
      if (e != cudaSuccess) break;
      const Arcs arcs{0.0, 0.0, t0, tf, segments};
      pc_status ps = session_begin(S[g], p, counts[g], total, off, x0, arcs, tol, xf, status, iters, nseg, 0,
                                   nullptr, 0, nullptr, p->own_stream);
      if (ps != PC_OK) {
        result = ps;
        S[g].finished = true;
      }
    } else {
      S[g].finished = true;
    }
    off += counts[g];
  }
  bool busy = true;
  while (busy && e == cudaSuccess) {
    busy = false;
    for (int g = 0; g < n_groups; g++) {
      if (S[g].finished || S[g].e != cudaSuccess) continue;
      session_step(S[g]);
      busy = busy || (!S[g].finished && S[g].e == cudaSuccess);
    }
  }
  for (int g = 0; g < n_groups; g++) {
    if (counts[g] == 0 || !S[g].p) continue;
    pc_status ps = session_finish(S[g], rounds_out);
    if (ps != PC_OK && result == PC_OK) result = ps;
    if (e == cudaSuccess) e = cudaEventRecord(fork, plans[g]->own_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, fork, 0);
  }
  if (fork) cudaEventDestroy(fork);
  if (e != cudaSuccess) return cuda_status(e);
  return result;
}

extern "C" pc_status pc_eval_ephemeris(pc_plan *p, long long n, const double *t, double *rb, void *stream) {
  if (!p || n < 0 || (n > 0 && (!t || !rb))) return PC_EINVAL;
  if (n == 0 || p->model.B == 0) return PC_OK;
  return cuda_status(launch_eval_ephemeris(p, n, t, rb, (cudaStream_t)stream));
}

extern "C" pc_status pc_eval_dynamics(pc_plan *p, long long n, const double *t, const double *y, double *f,
                                      void *stream) {
  if (!p || n < 0 || (n > 0 && (!t || !y || !f))) return PC_EINVAL;
  if (n == 0) return PC_OK;
  return cuda_status(launch_eval_dynamics(p, n, t, y, f, (cudaStream_t)stream));
}

extern "C" pc_status pc_eval_warm_start(pc_plan *p, long long n, const double *x0, const double *dt, double *x,
                                        void *stream) {
  if (!p || n < 0 || (n > 0 && (!x0 || !dt || !x))) return PC_EINVAL;
  if (n == 0) return PC_OK;
  return cuda_status(launch_eval_warm(p, n, x0, dt, x, (cudaStream_t)stream));
}

// The contraction kernel wants G with kpad rows and a leading dimension that
// is a multiple of 8; the caller's arrays are [N+1][6][n_ic].  They are staged
// through the workspace (G, Y[1]) with 2-D copies.
extern "C" pc_status pc_apply_operator(pc_plan *p, long long n_ic, const double *x0, const double *g, double *y,
                                       void *stream) {
  if (!p || n_ic < 0 || (n_ic > 0 && (!x0 || !g || !y))) return PC_EINVAL;
  if (n_ic == 0) return PC_OK;
  pc_status ps = ensure_workspace(p, n_ic, 0);
  if (ps != PC_OK) return ps;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace &w = p->ws;
  const size_t ld = (size_t)w.ld, rows = (size_t)p->n * 6;
  double *xs = w.ctl[w.live].x;
  cudaError_t e = cudaMemcpy2DAsync(xs, ld * 8, x0, (size_t)n_ic * 8, (size_t)n_ic * 8, 6, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(w.G, ld * 8, g, (size_t)n_ic * 8, (size_t)n_ic * 8, rows, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = launch_apply_operator(p, n_ic, w.ld, xs, w.G, w.Y[1], st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(y, (size_t)n_ic * 8, w.Y[1], ld * 8, (size_t)n_ic * 8, rows, cudaMemcpyDeviceToDevice, st);
  return cuda_status(e);
}

extern "C" pc_status pc_plan_set_profiling(pc_plan *p, int on) {
  if (!p) return PC_EINVAL;
  p->prof_on = on ? 1 : 0;
  return PC_OK;
}

extern "C" pc_status pc_plan_kernel_times(pc_plan *p, pc_kernel_times *out) {
  if (!p || !out) return PC_EINVAL;
  for (int k = 0; k < PC_KERNEL_KINDS; k++) {
    out->launches[k] = 0;
    out->ms[k] = 0.0;
  }
  cudaError_t e = cudaSuccess;
  for (long long r = 0; r < p->prof_rounds && e == cudaSuccess; r++) {
    cudaEvent_t *ev = p->prof_ev.data() + (size_t)r * 6;
    e = cudaEventSynchronize(ev[5]);
    for (int k = 0; k < PC_KERNEL_KINDS && e == cudaSuccess; k++) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      out->ms[k] += ms;
      out->launches[k] += 1;
    }
  }
  p->prof_rounds = 0;
  out->sweeps64 = p->acc_sweeps64;
  out->sweeps32 = p->acc_sweeps32;
  out->kernel_launches = p->acc_launches;
  p->acc_sweeps64 = p->acc_sweeps32 = 0;
  p->acc_launches = 0;
  return cuda_status(e);
}

extern "C" pc_status pc_plan_get_tuning(const pc_plan *p, pc_tuning *out) {
  if (!p || !out) return PC_EINVAL;
  *out = p->tune;
  return PC_OK;
}

extern "C" pc_status pc_plan_set_tuning(pc_plan *p, const pc_tuning *t) {
  if (!p || !t) return PC_EINVAL;
  if (t->setup_ctas_per_sm < 1 || t->setup_ctas_per_sm > 16 || t->fp32_ctas_per_sm < 1 || t->fp32_ctas_per_sm > 16 ||
      t->contract_ctas_per_sm < 1 || t->contract_ctas_per_sm > 16 || t->rounds_per_batch < 1 ||
      t->rounds_per_batch > 64 || t->repack_div < 2 || t->repack_div > 64 || (t->graphs != 0 && t->graphs != 1) ||
      (t->side_priority != 0 && t->side_priority != 1) ||
      (t->fp32_rows != 0 && t->fp32_rows != 4 && t->fp32_rows != 8) || t->fp32_slots < 8 || t->fp32_slots > 64 ||
      t->fp32_slots % 8 != 0 || (t->grid_cache != 0 && t->grid_cache != 1))
    return PC_EINVAL;
  p->tune = *t;
  return PC_OK;
}

extern "C" pc_status pc_plan_autotune(pc_plan *p, long long n_ic, const double *x0, double t0, double tf,
                                      int max_rounds, pc_tuning *best, void *stream) {
  if (!p || n_ic < 1 || !x0 || max_rounds < 16 || n_ic > (1LL << 30)) return PC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double *xf = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaMalloc((void **)&xf, sizeof(double) * 6 * (size_t)n_ic);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  const long long saved_rounds = p->opt.max_rounds;
  const int saved_prof = p->prof_on;
  p->opt.max_rounds = max_rounds;
  p->prof_on = 0;
  pc_status ps = PC_OK;
  // time per round of a propagation capped at max_rounds with tuning t
  auto trial = [&](const pc_tuning &t, double *ms_per_round) -> pc_status {
    p->tune = t;
    if ((e = cudaEventRecord(ev[0], st)) != cudaSuccess) return cuda_status(e);
    long long rounds = 0;
    pc_status r = pc_propagate_ex(p, n_ic, x0, t0, tf, 0.0, xf, nullptr, nullptr, nullptr, 0, nullptr, &rounds, st);
    if (r != PC_OK && r != PC_ENOTCONV) return r;
    if ((e = cudaEventRecord(ev[1], st)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaEventSynchronize(ev[1])) != cudaSuccess) return cuda_status(e);
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, ev[0], ev[1])) != cudaSuccess) return cuda_status(e);
    *ms_per_round = rounds > 0 ? ms / (double)rounds : 1e30;
    return PC_OK;
  };
  pc_tuning cur = p->tune;
  double cur_ms = 0.0;
  if (e != cudaSuccess) ps = cuda_status(e);
  if (ps == PC_OK) ps = trial(cur, &cur_ms);  // warm-up: workspace allocation, first captures
  if (ps == PC_OK) ps = trial(cur, &cur_ms);
  const bool mixed = p->opt.precision == PC_PREC_MIXED;
  // Coordinate descent over single fields, plus joint moves where one field's
  // best value depends on another's (the one-trajectory FP32 kernel wants
  // several CTAs per SM, the tiled one about one).
  struct Move {
    std::vector<std::pair<int pc_tuning::*, int>> set;
  };
  std::vector<Move> moves;
  auto axis = [&](int pc_tuning::*f, std::initializer_list<int> vals) {
    for (int v : vals) moves.push_back(Move{{{f, v}}});
  };
  axis(&pc_tuning::contract_ctas_per_sm, {2, 3, 4, 6, 8, 12, 16});
  axis(&pc_tuning::setup_ctas_per_sm, {2, 4, 8, 16});
  if (mixed) {
    for (int r : {0, 4, 8})
      for (int c : (r == 0 ? std::vector<int>{4, 6, 8, 12} : std::vector<int>{1, 2}))
        moves.push_back(Move{{{&pc_tuning::fp32_rows, r}, {&pc_tuning::fp32_ctas_per_sm, c}}});
    axis(&pc_tuning::fp32_slots, {8, 16, 32});
    axis(&pc_tuning::side_priority, {0, 1});
  }
  axis(&pc_tuning::rounds_per_batch, {4, 8, 16, 32});
  axis(&pc_tuning::repack_div, {4, 8, 16});
  axis(&pc_tuning::graphs, {0, 1});
  if (p->model.B > 0) axis(&pc_tuning::grid_cache, {0, 1});
  for (const Move &mv : moves) {
    if (ps != PC_OK) break;
    pc_tuning cand = cur;
    bool same = true;
    for (const auto &fv : mv.set) {
      same = same && cur.*(fv.first) == fv.second;
      cand.*(fv.first) = fv.second;
    }
    if (same) continue;
    double ms = 0.0;
    ps = trial(cand, &ms);
    if (ps == PC_OK && ms < 0.99 * cur_ms) {  // keep a change only for a clear gain
      cur = cand;
      cur_ms = ms;
    }
  }
  p->tune = cur;
  p->opt.max_rounds = saved_rounds;
  p->prof_on = saved_prof;
  if (best) *best = cur;
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  cudaFree(xf);
  return ps;
}
