// Host driver of the batched sweep and the kernel-level entry points.
#include <cmath>

#include "pc_internal.h"

using namespace pcx;

namespace {

pc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PC_OK;
  return e == cudaErrorMemoryAllocation ? PC_ENOMEM : PC_ECUDA;
}

// Rounds issued between two looks at the done counter.  The host keeps one
// batch in flight while it waits for the previous batch's counter, so the GPU
// does not idle during the check.
constexpr int kRoundsPerBatch = 8;

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
  const pc_options &o = p->opt;
  const int mixed = o.precision == PC_PREC_MIXED ? 1 : 0;
  pc_status ps = ensure_workspace(p, n_ic, mixed);
  if (ps != PC_OK) return ps;
  cudaStream_t st = (cudaStream_t)stream;
  Sweep s{};
  s.N = p->N;
  s.n = p->n;
  s.kpad = p->kpad;
  s.rows_pad = p->rows_pad;
  s.n_ic = n_ic;
  s.ld = p->ws.ld;
  s.t0 = t0;
  s.tf = tf;
  s.total = std::fabs(tf - t0);
  s.sgn = (tf >= t0) ? 1.0 : -1.0;
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
  Workspace &w = p->ws;
  s.xf = xf;
  s.status = status;
  s.iters = iters;
  s.nseg = nseg;
  s.mixed = mixed;
  s.switch_tol = o.switch_tol;
  s.list[0] = w.lists;
  s.list[1] = w.lists + w.ld;
  s.list_cnt = w.ints + 2;
  s.l64[0] = w.lists + 2 * (size_t)w.ld;
  s.l64[1] = w.lists + 3 * (size_t)w.ld;
  s.l64_cnt = w.ints + 5;
  s.tile_ctr = w.ints + 7;
  s.cnt64 = w.cnt64;
  s.list_cur = 0;
  s.A = (int)n_ic;
  w.live = 0;

  cudaError_t e = launch_init(p, s, x0, st);
  const long long max_rounds = o.max_rounds > 0 ? o.max_rounds : 10000000LL;
  long long rounds = 0;
  int cur = 0;
  int pending = -1;         // slot of the batch whose counter copy is in flight
  int done_known = 0;       // finished trajectories at the last completed check
  bool finished = false, capped = false;
  while (e == cudaSuccess && !finished) {
    for (int r = 0; r < kRoundsPerBatch && e == cudaSuccess && s.A > 0; r++) {
      cudaEvent_t *ev = nullptr;
      if (p->prof_on) {
        const size_t need = (size_t)(p->prof_rounds + 1) * 6;
        while (e == cudaSuccess && p->prof_ev.size() < need) {
          cudaEvent_t x;
          e = cudaEventCreate(&x);
          if (e == cudaSuccess) p->prof_ev.push_back(x);
        }
        if (e != cudaSuccess) break;
        ev = p->prof_ev.data() + (size_t)p->prof_rounds * 6;
        p->prof_rounds++;
      }
      e = launch_round(p, s, cur, st, ev);
      cur ^= 1;
      s.list_cur ^= 1;
      rounds++;
    }
    if (e != cudaSuccess) break;
    const int slot = (pending < 0) ? 0 : (pending ^ 1);
    e = cudaMemcpyAsync(w.h_ints + 8 * slot, w.ints, 8 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(w.ev[slot], st);
    if (e != cudaSuccess) break;
    if (pending >= 0) {
      e = cudaEventSynchronize(w.ev[pending]);
      if (e != cudaSuccess) break;
      done_known = w.h_ints[8 * pending];
      if (done_known >= n_ic) finished = true;
    }
    pending = slot;
    if (finished) break;
    if (rounds >= max_rounds) {
      capped = true;
      break;
    }
    // Compaction: when at least 1/8 of the slots hold finished trajectories,
    // move the active ones to the front so later rounds launch over fewer slots.
    const long long active = n_ic - done_known;
    const long long dead = (long long)s.A - active;
    if (dead > 0 && dead * 8 >= (long long)s.A) {
      e = launch_repack(p, s, cur, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(w.h_ints + 16, w.ints + 4, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) break;
      s.A = w.h_ints[16];
      cur ^= 1;
      w.live ^= 1;
      pending = -1;
      if (s.A == 0) finished = true;
    }
  }
  if (e == cudaSuccess && capped) e = launch_abort(p, s, st);
  // aggregate: did any trajectory stop early?
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.h_ints, w.ints, 8 * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.h_cnt64, w.cnt64, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (rounds_out) *rounds_out = rounds;
  if (e != cudaSuccess) return cuda_status(e);
  p->acc_sweeps64 += (long long)w.h_cnt64[0];
  p->acc_sweeps32 += (long long)w.h_cnt64[1];
  if (capped || w.h_ints[1] > 0) return PC_ENOTCONV;
  return PC_OK;
}

extern "C" pc_status pc_propagate(pc_plan *p, long long n_ic, const double *x0, double t0, double tf, double tol,
                                  double *xf, int *status, int *iters, void *stream) {
  return pc_propagate_ex(p, n_ic, x0, t0, tf, tol, xf, status, iters, nullptr, 0, nullptr, nullptr, stream);
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
