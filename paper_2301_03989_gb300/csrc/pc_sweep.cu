// Device kernels of the batched Picard-Chebyshev sweep and their launchers.
//
// One "round" advances every unfinished trajectory by one step of its own
// current segment (Section "Matrix form for vectorized and parallel
// computation"; Eq. 2):
//   k_setup      new segments only: node times, ephemeris at the nodes,
//                Keplerian warm start (Sections "Integration concept",
//                "Dynamics model"), and for mixed precision the FP32 inputs
//   k_fp32       mixed precision, one CTA per trajectory: the FP32 phase of a
//                new segment (Encke-form deviation from the warm start) or an
//                FP32 correction solve after an FP64 sweep; the result goes to
//                the next round's buffer
//   k_force      FP64 sweep: F = omega2 f(Y, t) (the paper's dynamics kernel)
//   k_contract   FP64 sweep: Y' = 1 x0^T + K F on the FP64 tensor cores
//                (DMMA), fused with the per-trajectory change
//                max_j max(|dr|/|r|, |dv|/|v|) (the paper's errCompute +
//                maxReduce, Section "CPU-GPU cooperated iteration error
//                computation", without the host round trip) and the residual
//   k_control    per trajectory: stop / stall / resolution tests, segment
//                accept / halve / advance (piecewise integration), hand-over
//                of FP32 results, choice of correction solves
// In mixed precision k_setup and k_fp32 (new segments, corrections) and
// k_force and k_contract (this round's FP64 list) touch disjoint trajectories
// and run on two streams, joined before k_control.
// State layout: node-major, component-planar Y[j][c][slot] (Section "Dynamics
// model, array sorting, and CUDA kernel"), leading dimension ld over slots.
// Active trajectories occupy slots [0, A); finished ones are packed out.
#include <algorithm>
#include <cstdint>

#include "pc_device.cuh"
#include "pc_internal.h"

namespace pcx {
namespace {

// Warp-aggregated append of `flag` lanes to list[] with counter *cnt.  Every
// lane of the warp must call it.
__device__ __forceinline__ void warp_append(bool flag, int value, int *list, int *cnt) {
  const unsigned mask = __ballot_sync(0xffffffffu, flag);
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(cnt, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (flag) list[base + __popc(mask & ((1u << lane) - 1u))] = value;
}

// ---------------------------------------------------------------------------
// Keplerian two-body propagation by dt (warm start).  Kepler's equation in the
// eccentric-anomaly increment X over dt,
//   F(X) = X - (e cos E0) sin X + (e sin E0)(1 - cos X) - n dt = 0,
// with e cos E0 = 1 - r0/a and e sin E0 = r0.v0/sqrt(mu a), is solved by
// Halley's method (third order: X <- X - 2 F F' / (2 F'^2 - F F'')), kept
// inside the bracket [n dt - 2, n dt + 2] by bisection, from the first-order
// root X = n dt a/r0 (clamped into the bracket).  Once a step is below 1e-6
// the cubic convergence puts the next error below 1e-17 and the iteration
// stops after applying it.  The Lagrange coefficients then map (r0, v0) to
// (r, v).  The quantities that depend only on the start state are formed once
// per segment (kepler_consts, when the segment is scheduled) and shared by all
// its nodes.  A start state that is not a bound ellipse, or an iteration that
// does not settle, gives no warm start.
// ---------------------------------------------------------------------------
constexpr int kKepConsts = kKeplerConsts;
// c[0] = 1/a (<= 0: not elliptic), c[1] = a, c[2] = e cos E0, c[3] = e sin E0,
// c[4] = n, c[5] = (r0.v0/sqrt(mu)) sqrt(a), c[6] = a/r0,
// c[7] = a (r0.v0)/mu, c[8] = r0 sqrt(a)/sqrt(mu), c[9] = -sqrt(mu) sqrt(a) / r0, c[10] = r0
__device__ void kepler_consts(double mu, const double x0[6], double c[kKepConsts]) {
  const double r0 = sqrt(x0[0] * x0[0] + x0[1] * x0[1] + x0[2] * x0[2]);
  const double vv = x0[3] * x0[3] + x0[4] * x0[4] + x0[5] * x0[5];
  const double rv = x0[0] * x0[3] + x0[1] * x0[4] + x0[2] * x0[5];
  const double inv_a = 2.0 / r0 - vv / mu;
  c[0] = inv_a;
  for (int k = 1; k < kKepConsts; k++) c[k] = 0.0;
  if (!(inv_a > 0.0)) return;
  const double a = 1.0 / inv_a;
  const double sqrt_a = sqrt(a);
  const double sqrt_mu = sqrt(mu);
  c[1] = a;
  c[2] = 1.0 - r0 * inv_a;
  c[3] = rv / (sqrt_mu * sqrt_a);
  c[4] = sqrt_mu * inv_a / sqrt_a;  // sqrt(mu / a^3)
  c[5] = rv / sqrt_mu * sqrt_a;
  c[6] = a / r0;
  c[7] = a * rv / mu;
  c[8] = r0 * sqrt_a / sqrt_mu;
  c[9] = -sqrt_mu * sqrt_a / r0;
  c[10] = r0;
}

// The iteration runs first in FP32 (same steps and bracket, to a step below
// 2e-6), which leaves the FP64 iteration one Halley step from that start in
// the usual case; the sine and cosine at the root then follow from those at
// the last iterate by the angle-addition formulas with the step's Taylor
// series (|step| <= 1e-5: the dropped terms are below 1e-32).  Only when the
// FP32 start is poor does the FP64 iteration take more steps.  An iterate
// with F = 0 is the root, and a Halley step onto the bracket's end is kept:
// at the root rounding can put the step exactly there, and bisecting from
// it would cost some thirty steps.
__device__ bool kepler_solve(const double c[kKepConsts], const double x0[6], double dt, double out[6]) {
  if (!(c[0] > 0.0)) return false;
  const double a = c[1], ecE = c[2], esE = c[3];
  const double M = c[4] * dt;
  double lo = M - 2.0, hi = M + 2.0;
  double X = fmin(fmax(M * c[6], lo + 0.5), hi - 0.5);
  {
    const float Mf = (float)M, ef = (float)ecE, sf = (float)esE;
    float lof = (float)lo, hif = (float)hi, Xf = (float)X;
    for (int it = 0; it < 32; it++) {
      float sXf, cXf;
      sincosf(Xf, &sXf, &cXf);
      const float F = Xf - ef * sXf + sf * (1.0f - cXf) - Mf;
      if (F == 0.0f) break;
      if (F > 0.0f) hif = Xf; else lof = Xf;
      const float d1 = 1.0f - ef * cXf + sf * sXf;
      const float d2 = ef * sXf + sf * cXf;
      float Xn = Xf - 2.0f * F * d1 / (2.0f * d1 * d1 - F * d2);
      if (!(Xn >= lof && Xn <= hif)) Xn = 0.5f * (lof + hif);
      const float step = fabsf(Xn - Xf);
      Xf = Xn;
      if (!(step > 2e-6f * (1.0f + fabsf(Xf)))) break;
    }
    if (isfinite(Xf)) X = fmin(fmax((double)Xf, lo), hi);
  }
  bool ok = false;
  double sX = 0.0, cX = 1.0, dl = 0.0;  // sine, cosine at the last evaluated iterate, step from it
  bool rotate = false;
  for (int it = 0; it < 64; it++) {
    sincos(X, &sX, &cX);
    const double F = X - ecE * sX + esE * (1.0 - cX) - M;
    if (F == 0.0) {
      ok = rotate = true;  // dl = 0: sX, cX are the root's
      dl = 0.0;
      break;
    }
    if (F > 0.0) hi = X; else lo = X;
    const double d1 = 1.0 - ecE * cX + esE * sX;
    const double d2 = ecE * sX + esE * cX;
    double Xn = X - 2.0 * F * d1 / (2.0 * d1 * d1 - F * d2);
    const bool halley = Xn >= lo && Xn <= hi;
    if (!halley) Xn = 0.5 * (lo + hi);
    dl = Xn - X;
    const double step = fabs(dl);
    X = Xn;
    if ((halley && step <= 1e-6 * (1.0 + fabs(X))) || step <= 1e-15 * (1.0 + fabs(X))) {
      ok = true;
      rotate = step <= 1e-5;
      break;
    }
  }
  if (!ok) return false;
  if (rotate) {
    // sin, cos at X = (previous iterate) + dl by angle addition
    const double d2 = dl * dl;
    const double sd = dl * (1.0 - d2 * (1.0 / 6.0) * (1.0 - d2 * 0.05));
    const double cd = 1.0 - d2 * 0.5 * (1.0 - d2 * (1.0 / 12.0));
    const double s1 = sX * cd + cX * sd, c1 = cX * cd - sX * sd;
    sX = s1;
    cX = c1;
  } else {
    sincos(X, &sX, &cX);
  }
  const double omc = 1.0 - cX;
  const double r = a + (c[10] - a) * cX + c[5] * sX;
  const double f = 1.0 - c[6] * omc;
  const double g = c[7] * omc + c[8] * sX;
  const double fd = c[9] / r * sX;
  const double gd = 1.0 - a / r * omc;
  for (int q = 0; q < 3; q++) {
    out[q] = f * x0[q] + g * x0[3 + q];
    out[3 + q] = fd * x0[q] + gd * x0[3 + q];
  }
  return true;
}

__device__ bool kepler_dt(double mu, const double x0[6], double dt, double out[6]) {
  double c[kKepConsts];
  kepler_consts(mu, x0, c);
  return kepler_solve(c, x0, dt, out);
}

// ---------------------------------------------------------------------------
// Segment schedule.  The arc [t0, tf] is measured in units u = hbase / 2^D; a
// segment at depth d starting at unit p spans 2^(D-d) units and is clipped to
// end exactly at tf.  Products and sums are rounded one at a time (no fused
// multiply-add) so every trajectory's segment bounds and node times are the
// exactly rounded values of these formulas.
// ---------------------------------------------------------------------------
__device__ void schedule(const Sweep &s, Ctl &c, int m, int list_next) {
  const int D = s.max_depth;
  const double u = scalbn(c.hbase[m], -D);
  const long long L = 1LL << (D - c.depth[m]);
  const long long p = c.p[m];
  const double t0 = c.t0[m], sgn = c.sgn[m];
  const double ta = dadd(t0, dmul(sgn, dmul((double)p, u)));
  double tb;
  int last = 0;
  if (dmul((double)(p + L), u) >= c.total[m]) {
    tb = c.tf[m];
    last = 1;
  } else {
    tb = dadd(t0, dmul(sgn, dmul((double)(p + L), u)));
  }
  c.ta[m] = ta;
  c.tb[m] = tb;
  if (s.warm) {
    double x0[6], kc[kKepConsts];
    for (int q = 0; q < 6; q++) x0[q] = c.x[q * s.ld + m];
    kepler_consts(s.mu_c, x0, kc);
    for (int q = 0; q < kKepConsts; q++) c.kc[q * s.ld + m] = kc[q];
  }
  c.w1[m] = dmul(0.5, dadd(tb, ta));
  c.w2[m] = dmul(0.5, dsub(tb, ta));
  c.last[m] = last;
  c.need_setup[m] = 1;
  c.seg_sweeps[m] = 0;
  c.nstall[m] = 0;
  c.ncorr[m] = 0;
  c.e_best[m] = __longlong_as_double(0x7FF0000000000000LL);  // +inf
  c.phase[m] = s.mixed ? PH_ITER32 : PH_ITER;
  const int k = atomicAdd(s.list_cnt + list_next, 1);
  s.list[list_next][k] = m;
}

// Final outputs of a trajectory, written when it finishes.
__device__ __forceinline__ void write_outputs(const Sweep &s, const Ctl &c, int m) {
  const long long i = s.io_off + c.ic[m];
  for (int q = 0; q < 6; q++) s.xf[q * s.io_ld + i] = c.x[q * s.ld + m];
  if (s.status) s.status[i] = c.status[m];
  if (s.iters) s.iters[i] = c.sweeps[m];
  if (s.nseg) s.nseg[i] = c.nseg[m];
}

__global__ void k_init(Sweep s, Ctl c, Model md, const double *__restrict__ x0, int *done) {
  const long long mm = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = (int)mm;
  bool to64 = false;
  if (mm < s.n_ic) {
    const int ld = s.ld;
    double x[6];
    bool finite = true;
    for (int q = 0; q < 6; q++) {
      x[q] = x0[q * s.io_ld + s.io_off + m];
      c.x[q * ld + m] = x[q];
      finite = finite && isfinite(x[q]);
    }
    const double t0 = s.t0a ? s.t0a[s.io_off + m] : s.t0s;
    const double tf = s.tfa ? s.tfa[s.io_off + m] : s.tfs;
    const int segs = s.sega ? s.sega[s.io_off + m] : s.segments;
    const double total = fabs(dsub(tf, t0));
    c.t0[m] = t0;
    c.tf[m] = tf;
    c.total[m] = total;
    c.sgn[m] = (tf >= t0) ? 1.0 : -1.0;
    // an arc outside the ephemeris table, or a bad segment count, is refused
    bool arc_ok = isfinite(t0) && isfinite(tf) && segs >= 1;
    if (md.B > 0) {
      const double lo = md.t_begin, hi = dadd(md.t_begin, dmul(md.granule, (double)md.n_gr));
      arc_ok = arc_ok && fmin(t0, tf) >= lo && fmax(t0, tf) <= hi;
    }
    double h = total / (double)(segs >= 1 ? segs : 1);
    if (s.seg_mode == 1 && finite) {
      const double r0 = sqrt(dadd(dadd(dmul(x[0], x[0]), dmul(x[1], x[1])), dmul(x[2], x[2])));
      const double v2 = dadd(dadd(dmul(x[3], x[3]), dmul(x[4], x[4])), dmul(x[5], x[5]));
      const double alpha = dsub(2.0 / r0, v2 / md.mu_c);
      if (alpha > 0.0) {
        const double a = 1.0 / alpha;
        const double twopi = 6.283185307179586;  // 2 * M_PI rounded
        h = dmul(twopi, sqrt(dmul(dmul(a, a), a) / md.mu_c)) / (double)(segs >= 1 ? segs : 1);
      }
    }
    c.ic[m] = m;
    c.hbase[m] = h;
    c.p[m] = 0;
    c.depth[m] = 0;
    c.status[m] = (finite ? 0 : PC_IC_NONFINITE) | (arc_ok ? 0 : PC_IC_OUT_OF_RANGE);
    c.sweeps[m] = 0;
    c.nseg[m] = 0;
    c.err[m] = 0ULL;
    c.err32[m] = 0u;
    c.need_setup[m] = 0;
    if (!finite || !arc_ok || !(total > 0.0)) {
      c.phase[m] = PH_DONE;
      write_outputs(s, c, m);
      atomicAdd(done, 1);
      if (!finite || !arc_ok) atomicAdd(done + 1, 1);
    } else {
      schedule(s, c, m, s.list_cur);
      to64 = c.phase[m] == PH_ITER;
    }
  }
  warp_append(to64, m, s.l64[s.list_cur], s.l64_cnt + s.list_cur);
}

// Indirect (frame) term of body b: the central body's own acceleration
// mu_b r_b/|r_b|^3, summed over bodies; it depends on the node time only.
__device__ __forceinline__ void add_indirect(const Model &md, int b, const double r[3], double ind[3]) {
  const double d2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  const double rs = rsqrt(d2);
  const double k = md.mu[b] * rs * rs * rs;
  for (int ax = 0; ax < 3; ax++) ind[ax] = fma(k, r[ax], ind[ax]);
}

// The warm start of a segment is interpolated from 17 nodes when the segment
// spans at most 1.5 rad of mean anomaly (a degree-16 Chebyshev interpolant of
// the Kepler arc is then exact to rounding); longer segments, and arcs with
// no mean motion, are solved at every node.
constexpr double kInterpMaxAnomaly = 1.5;
__device__ __forceinline__ bool kepler_interpolated(const Sweep &s, const Ctl &c, int m) {
  return s.kep_stride > 0 && fabs(c.kc[4 * s.ld + m] * (c.tb[m] - c.ta[m])) <= kInterpMaxAnomaly &&
         c.kc[(size_t)0 * s.ld + m] > 0.0;
}

// Warm start of the new segments at the 17 interpolation nodes j = i *
// kep_stride (grid-stride over list entries x those nodes, entries fastest):
// Kepler's equation solved as at every node before, stored as the deviation
// from the start state in an FP32 pair hi + lo (about 48 bits), NaN where the
// iteration does not settle (k_setup then starts the whole segment cold).
// Node 0 is the start state.
__global__ void k_kepler17(Sweep s, Ctl c, const double *__restrict__ tau) {
  const int cur = s.list_cur;
  const long long count = s.list_cnt[cur];
  const int *__restrict__ list = s.list[cur];
  const long long total = count * kKepNodes;
  const int ld = s.ld;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / count);
    const long long e = i - (long long)k * count;
    const int m = list[e];
    if (!kepler_interpolated(s, c, m)) continue;
    const int j = k * s.kep_stride;
    double x0[6], y[6];
    for (int q = 0; q < 6; q++) x0[q] = c.x[q * ld + m];
    bool ok = true;
    if (j > 0) {
      double kc[kKepConsts];
      for (int q = 0; q < kKepConsts; q++) kc[q] = c.kc[q * ld + m];
      const double t = dadd(c.w1[m], dmul(c.w2[m], tau[j]));
      ok = kepler_solve(kc, x0, dsub(t, c.ta[m]), y);
    } else {
      for (int q = 0; q < 6; q++) y[q] = x0[q];
    }
    for (int q = 0; q < 6; q++) {
      const double d = y[q] - x0[q];
      const float hi = ok ? (float)d : __int_as_float(0x7FC00000);
      reinterpret_cast<float2 *>(s.YK17)[((size_t)k * 6 + q) * ld + e] =
          make_float2(hi, ok ? (float)(d - (double)hi) : hi);
    }
  }
}

// ---------------------------------------------------------------------------
// Ephemeris of the new segments by node-time grid.  Segments with the same
// (w1, w2) have the same node times t_j = w1 + w2 tau_j bit for bit (uniform
// schedules over a common arc start many segments together), so the body
// positions and the summed indirect term are evaluated once per grid:
// k_grid_keys gives every list entry its grid's table slot (the first entry of
// a grid owns it and takes the next cache index u), k_grid_ephem evaluates the
// cache EC at every (grid, node), and k_setup copies from it.  The arithmetic
// per node is the same as k_setup's own, so the copies are bitwise equal.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long grid_hash(unsigned long long a, unsigned long long b) {
  // the splitmix64 finaliser (Steele, Lea and Flood; constants by Vigna) of a mix of both keys
  unsigned long long x = a ^ (b * 0x9E3779B97F4A7C15ULL);
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ULL;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBULL;
  x ^= x >> 31;
  return x;
}

// Inserts list entry e's grid (k1, k2) = bits of (w1, w2) by linear probing
// from slot hk; returns the slot holding the grid.  At most eh_size probes:
// the table holds at least twice the list capacity, so a free slot exists.
__device__ int grid_insert(const Sweep &s, const Ctl &c, int cur, int e, long long k1, long long k2,
                           unsigned long long hk) {
  int *tab = s.eh_tab[cur];
  const unsigned msk = (unsigned)s.eh_size - 1u;
  unsigned h = (unsigned)hk & msk;
  for (int it = 0; it < s.eh_size; it++) {
    const int o = atomicCAS(tab + h, -1, e);
    if (o == -1) {
      const int u = atomicAdd(s.eh_cnt + cur, 1);
      if (u < s.eh_cap) s.eh_own[u] = e;
      s.eh_uid[cur][h] = u < s.eh_cap ? u : -1;
      return (int)h;
    }
    const int mo = s.list[cur][o];
    if (__double_as_longlong(c.w1[mo]) == k1 && __double_as_longlong(c.w2[mo]) == k2) return (int)h;
    h = (h + 1u) & msk;
  }
  return -1;
}

// One thread per list entry, whole warps per loop trip; the lanes of a warp
// with the same grid insert it once (their leader's slot is shared).
__global__ void k_grid_keys(Sweep s, Ctl c) {
  const int cur = s.list_cur;
  const long long count = s.list_cnt[cur];
  const int *__restrict__ list = s.list[cur];
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long wb = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); wb < count; wb += stride) {
    const long long e = wb + lane;
    const bool act = e < count;
    const unsigned am = __ballot_sync(0xFFFFFFFFu, act);
    if (!act) continue;
    const int m = list[e];
    const long long k1 = __double_as_longlong(c.w1[m]), k2 = __double_as_longlong(c.w2[m]);
    const unsigned long long hk = grid_hash((unsigned long long)k1, (unsigned long long)k2);
    const unsigned grp = __match_any_sync(am, hk);
    const int leader = __ffs(grp) - 1;
    const long long l1 = __shfl_sync(am, k1, leader), l2 = __shfl_sync(am, k2, leader);
    const bool same = l1 == k1 && l2 == k2;
    int h = -1;
    if (lane == leader || !same) h = grid_insert(s, c, cur, (int)e, k1, k2, hk);
    const int hl = __shfl_sync(am, h, leader);
    s.eh_ent[e] = (same && lane != leader) ? hl : h;
  }
}

// Body positions and summed indirect term of every cached grid at every node
// (grid-stride over grids x nodes, grids fastest).
__global__ void k_grid_ephem(Sweep s, Ctl c, Model md, const double *__restrict__ tau) {
  const int cur = s.list_cur;
  const long long U = min(s.eh_cnt[cur], s.eh_cap);
  const long long total = U * s.n;
  const int B = md.B;
  const size_t cap = (size_t)s.eh_cap;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / U);
    const long long u = i - (long long)j * U;
    const int m = s.list[cur][s.eh_own[u]];
    const double t = dadd(c.w1[m], dmul(c.w2[m], tau[j]));
    double *ec = s.EC + (size_t)j * (3 * B + 3) * cap + u;
    double ind[3] = {0.0, 0.0, 0.0};
    ephem_all(md, ephem_locate(md, t), [&](int b, const double r[3]) {
      for (int ax = 0; ax < 3; ax++) ec[(size_t)(3 * b + ax) * cap] = r[ax];
      if (md.indirect) add_indirect(md, b, r, ind);
    });
    for (int ax = 0; ax < 3; ax++) ec[(size_t)(3 * B + ax) * cap] = ind[ax];
  }
}

// Mixed-precision inputs of the new segments, by list entry e (not slot):
//   YK[e][j][6]        FP64 warm start y_K at node j
//   X32[e][j][xs]      FP32 record of node j, in float4 groups:
//                      (r_K, mu_c/|r_K|^3), (v_K, -), (summed indirect term, -),
//                      then per body (r_K - r_b formed in FP64 then rounded, -)
struct Mix {
  double *YK;
  float *X32;
  int xs;          // floats per node record: 12 + 4B
};
// New segments: node times, body positions and summed indirect term at the
// nodes, warm start -- only for the slots on this round's new-segment list
// (grid-stride over list entries x nodes, entries fastest).  With mixed
// precision the warm start goes to YK and the FP32 node records to X32 (both
// by list entry) for k_fp32; otherwise the warm start is the first iterate.
// Block 0 clears the lists this round's control kernel fills.
__global__ void k_setup(Sweep s, Ctl c, Model md, const double *__restrict__ tau, double *__restrict__ Y,
                        double *__restrict__ E, double *__restrict__ Aind, Mix mx) {
  const int cur = s.list_cur;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s.list_cnt[cur ^ 1] = 0;
    s.l64_cnt[cur ^ 1] = 0;
    s.lc_cnt[cur ^ 1] = 0;
    s.fp32_ctr[0] = 0;  // this round's FP32 kernels run after this kernel
    s.fp32_ctr[1] = 0;
    if (s.eh_size > 0) s.eh_cnt[cur ^ 1] = 0;
  }
  // the next round's grid table (this round's grids are read below)
  if (s.eh_size > 0)
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < s.eh_size;
         i += (long long)gridDim.x * blockDim.x)
      s.eh_tab[cur ^ 1][i] = -1;
  const long long count = s.list_cnt[cur];
  const int *__restrict__ list = s.list[cur];
  const long long total = count * s.n;
  const int ld = s.ld, B = md.B;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / count);
    const long long e = i - (long long)j * count;
    const int m = list[e];
    const double t = dadd(c.w1[m], dmul(c.w2[m], tau[j]));
    double x0[6], y[6];
    for (int q = 0; q < 6; q++) x0[q] = c.x[q * ld + m];
    bool ok = false;
    if (j > 0 && s.warm) {
      if (kepler_interpolated(s, c, m)) {
        // The deviation from the start state interpolated from the 17 solved
        // nodes in compensated FP32 arithmetic (each product split exactly
        // by an FMA, each sum by Knuth's TwoSum, the remainders and the lo
        // parts summed beside): about 1e-13 of the deviation, as the FP64
        // sum was, at the cost of FP32 operations.  The FP32 phase relies on
        // this accuracy: it treats the warm start as an exact Kepler arc.
        float sh[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, sl[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        bool fin = true;
        const float *Lh = s.Lint + (size_t)j * kKepNodes;
        const float *Ll = s.Lint + ((size_t)s.n + j) * kKepNodes;
        for (int k = 1; k < kKepNodes; k++) {
          const float lh = Lh[k], ll = Ll[k];
#pragma unroll
          for (int q = 0; q < 6; q++) {
            const float2 dd = reinterpret_cast<const float2 *>(s.YK17)[((size_t)k * 6 + q) * ld + e];
            const float dh = dd.x, dl = dd.y;
            fin = fin && isfinite(dh);
            const float pr = __fmul_rn(lh, dh);
            const float pe = __fmaf_rn(lh, dh, -pr);  // lh dh - pr, exactly
            const float sm = __fadd_rn(sh[q], pr);
            const float bv = __fsub_rn(sm, sh[q]);
            const float se = __fadd_rn(__fsub_rn(sh[q], __fsub_rn(sm, bv)), __fsub_rn(pr, bv));  // sh + pr - sm
            sh[q] = sm;
            sl[q] = __fadd_rn(sl[q], __fadd_rn(__fadd_rn(se, pe), __fmaf_rn(lh, dl, __fmul_rn(ll, dh))));
          }
        }
        ok = fin;
        if (ok)
          for (int q = 0; q < 6; q++) y[q] = x0[q] + ((double)sh[q] + (double)sl[q]);
      } else {
        double kc[kKepConsts];
        for (int q = 0; q < kKepConsts; q++) kc[q] = c.kc[q * ld + m];
        ok = kepler_solve(kc, x0, dsub(t, c.ta[m]), y);
      }
    }
    if (!ok)
      for (int q = 0; q < 6; q++) y[q] = x0[q];
    float *rec = s.mixed ? mx.X32 + ((size_t)e * s.n + j) * mx.xs : nullptr;
    auto body = [&](int b, const double r[3]) {
      for (int ax = 0; ax < 3; ax++) E[((size_t)(j * B + b) * 3 + ax) * ld + m] = r[ax];
      if (rec)
        reinterpret_cast<float4 *>(rec)[3 + b] =
            make_float4((float)(y[0] - r[0]), (float)(y[1] - r[1]), (float)(y[2] - r[2]), 0.0f);
    };
    double ind[3] = {0.0, 0.0, 0.0};
    const int slot = s.eh_size > 0 ? s.eh_ent[e] : -1;
    const int u = slot >= 0 ? s.eh_uid[cur][slot] : -1;
    if (u >= 0) {
      // the segment's grid is cached
      const size_t cap = (size_t)s.eh_cap;
      const double *ec = s.EC + (size_t)j * (3 * B + 3) * cap + u;
      for (int b = 0; b < B; b++) {
        const double r[3] = {ec[(size_t)(3 * b) * cap], ec[(size_t)(3 * b + 1) * cap], ec[(size_t)(3 * b + 2) * cap]};
        body(b, r);
      }
      for (int ax = 0; ax < 3; ax++) ind[ax] = ec[(size_t)(3 * B + ax) * cap];
    } else {
      ephem_all(md, ephem_locate(md, t), [&](int b, const double r[3]) {
        if (md.indirect) add_indirect(md, b, r, ind);
        body(b, r);
      });
    }
    for (int ax = 0; ax < 3; ax++) Aind[(size_t)(j * 3 + ax) * ld + m] = ind[ax];
    if (rec) {
      // 16-byte stores: a record is 12 + 4B floats, a warm start 6 doubles
      double2 *yk = reinterpret_cast<double2 *>(mx.YK + ((size_t)e * s.n + j) * 6);
      yk[0] = make_double2(y[0], y[1]);
      yk[1] = make_double2(y[2], y[3]);
      yk[2] = make_double2(y[4], y[5]);
      const double rr = rsqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
      float4 *r4 = reinterpret_cast<float4 *>(rec);
      r4[0] = make_float4((float)y[0], (float)y[1], (float)y[2], (float)(md.mu_c * rr * rr * rr));
      r4[1] = make_float4((float)y[3], (float)y[4], (float)y[5], 0.0f);
      r4[2] = make_float4((float)ind[0], (float)ind[1], (float)ind[2], 0.0f);
    } else {
      for (int q = 0; q < 6; q++) Y[(size_t)(j * 6 + q) * ld + m] = y[q];
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 force: F[j][.][m] = omega2 * (v, a(r, t_j)).  One thread per (node,
// FP64-list entry).
// ---------------------------------------------------------------------------
// Body b's position component ax is Eb[(b*3 + ax) * es]; the summed indirect
// term component ax is Ai[ax * es].
__device__ __forceinline__ void accel(const Model &md, const double *__restrict__ Eb, const double *__restrict__ Ai,
                                      size_t es, const double r[3], double a[3]) {
  const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  const double rs = rsqrt(r2);
  const double kc = md.mu_c * rs * rs * rs;
  a[0] = -kc * r[0];
  a[1] = -kc * r[1];
  a[2] = -kc * r[2];
  for (int b = 0; b < md.B; b++) {
    const double d0 = r[0] - Eb[(size_t)(b * 3 + 0) * es];
    const double d1 = r[1] - Eb[(size_t)(b * 3 + 1) * es];
    const double d2 = r[2] - Eb[(size_t)(b * 3 + 2) * es];
    const double dd = d0 * d0 + d1 * d1 + d2 * d2;
    const double ds = rsqrt(dd);
    const double kb = md.mu[b] * ds * ds * ds;
    a[0] -= kb * d0;
    a[1] -= kb * d1;
    a[2] -= kb * d2;
  }
  if (md.indirect) {
    a[0] -= Ai[0];
    a[1] -= Ai[es];
    a[2] -= Ai[2 * es];
  }
}

// Resolution-test sums, accumulated while the force table is built (see the
// resolution test below): per trajectory, for each component q,
//   sN[q]  = sum''_j (-1)^(N+j) F_j[q],   sN1[q] = sum''_j (-1)^(N+j) tau_j F_j[q]
// and the largest |r_j|^2, |v_j|^2 of the iterate.  Each block sums its
// kForceNodes nodes in node order into partials[nb][v][slot] (node block nb;
// v = 0..5 sN, 6..11 sN1, 12 max|r|^2, 13 max|v|^2); the control kernel adds
// the node blocks in order.  The sums never depend on scheduling.
constexpr int kTailVals = 14;
constexpr int kForceNodes = 8;

// Block = 32 FP64-list entries (x) by kForceNodes nodes (y); one thread per
// (entry, node).  Three blocks per SM (at most 80 registers): the kernel is
// bound by GB300's FP64 pipe, and 16 warps per SM left it 68 % busy.
__global__ void __launch_bounds__(32 * kForceNodes, 3) k_force(Sweep s, Ctl c, Model md, const double *__restrict__ Y,
                                                          const double *__restrict__ E,
                                                          const double *__restrict__ Aind, double *__restrict__ G,
                                                          const double *__restrict__ tau,
                                                          double *__restrict__ partials,
                                                          const double *__restrict__ EX) {
  __shared__ double red[kForceNodes][kTailVals][32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * 32 + tx;
  const int j = blockIdx.y * kForceNodes + ty;
  const int count = s.l64_cnt[s.list_cur];
  const bool valid = i < count;
  const int m = valid ? s.l64[s.list_cur][i] : 0;
  const int ld = s.ld, N = s.N;
  // this node's resolution-sum terms go straight to shared memory (zero for
  // an idle thread); thread ty = 0 adds the block's nodes in node order below
  if (valid && j <= N) {
    const double w2 = c.w2[m];
    const size_t yb = (size_t)j * 6 * ld + m;
    double y[6];
#pragma unroll
    for (int q = 0; q < 6; q++) y[q] = Y[yb + (size_t)q * ld];
    double a[3];
    accel(md, E + (size_t)j * md.B * 3 * ld + m, Aind + (size_t)j * 3 * ld + m, (size_t)ld, y, a);
    if (md.c_light > 0.0) {  // Einstein-Infeld-Hoffmann terms
      double e3[3];
      eih_terms(md, E + (size_t)j * md.B * 3 * ld + m, EX + (size_t)j * eih_stride(md.B) * ld + m, (size_t)ld, y,
                y + 3, e3);
      for (int q = 0; q < 3; q++) a[q] += e3[q];
    }
    const double g[6] = {w2 * y[3], w2 * y[4], w2 * y[5], w2 * a[0], w2 * a[1], w2 * a[2]};
#pragma unroll
    for (int q = 0; q < 6; q++) G[yb + (size_t)q * ld] = g[q];
    const double wj = (j == 0 || j == N) ? 0.5 : 1.0;
    const double sg = ((N + j) & 1) ? -wj : wj;
    const double st = sg * tau[j];
#pragma unroll
    for (int q = 0; q < 6; q++) {
      red[ty][q][tx] = sg * g[q];
      red[ty][6 + q][tx] = st * g[q];
    }
    red[ty][12][tx] = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    red[ty][13][tx] = y[3] * y[3] + y[4] * y[4] + y[5] * y[5];
  } else {
#pragma unroll
    for (int v = 0; v < kTailVals; v++) red[ty][v][tx] = 0.0;
  }
  __syncthreads();
  if (ty == 0 && valid) {
    double acc[kTailVals];
#pragma unroll
    for (int v = 0; v < kTailVals; v++) acc[v] = red[0][v][tx];
    for (int u = 1; u < kForceNodes; u++) {
#pragma unroll
      for (int v = 0; v < 12; v++) acc[v] += red[u][v][tx];
      acc[12] = fmax(acc[12], red[u][12][tx]);
      acc[13] = fmax(acc[13], red[u][13][tx]);
    }
    double *pp = partials + (size_t)blockIdx.y * kTailVals * ld + m;
#pragma unroll
    for (int v = 0; v < kTailVals; v++) pp[(size_t)v * ld] = acc[v];
  }
}

// ---------------------------------------------------------------------------
// Contraction on the FP64 tensor cores: mma.sync m16n8k4 f64.
// A warp tile is output nodes j = 1 + 16*rt + (0..15) for 8 trajectories and
// all six components (six 16x8 accumulators), streaming K[rows][k] and
// F[k][c][m] fragments straight from L2/L1 -- FP64 throughput, not bandwidth,
// bounds this kernel.  In the sweep the 8 trajectories are 8 consecutive
// entries of the round's FP64 list, and warps take tiles from a counter until
// none are left (no partial last wave).  Fragment layouts (PTX ISA,
// mma.m16n8k4 .f64): with g = lane/4, t = lane%4:  A: a0 = A[g][t],
// a1 = A[g+8][t];  B: b0 = B[t][g];  C: c0,c1 = C[g][2t..2t+1],
// c2,c3 = C[g+8][2t..2t+1].  Epilogue: Y' = x0 + acc and (unless DIAG) the
// per-trajectory maximum change, reduced over the warp, merged with atomicMax.
// ---------------------------------------------------------------------------
// One CTA of kSplit warps computes one tile; warp w accumulates the k-steps
// [w*ks/kSplit, (w+1)*ks/kSplit) of it (ks = kpad/4 steps of 4), the partial
// accumulators meet in shared memory and warp 0 adds them in warp order (a
// fixed order, so results do not depend on scheduling) and runs the epilogue.
// Splitting k cuts the latency of a tile by kSplit and spreads few tiles over
// more SM sub-partitions.
constexpr int kSplit = 4;

template <bool DIAG>
__device__ __forceinline__ void contract_tile_split(const Sweep &s, const Ctl &c, const double *__restrict__ K,
                                                    const double *__restrict__ G, const double *__restrict__ Yold,
                                                    double *__restrict__ Ynew, int rt, int e0, int ncols,
                                                    const int *__restrict__ map, double *part,
                                                    float *__restrict__ R32) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int ld = s.ld;
  // entry e0 + g feeds the B fragment (a past-the-end entry reuses entry e0's
  // column; its results are never stored); entries e0 + 2t + {0,1} own C
  const int eb = (e0 + g < ncols) ? e0 + g : e0;
  const int mb = DIAG ? eb : map[eb];
  double acc[6][4];
#pragma unroll
  for (int q = 0; q < 6; q++)
#pragma unroll
    for (int i = 0; i < 4; i++) acc[q][i] = 0.0;
  const int ks = s.kpad / 4;
  const int kb = (w * ks) / kSplit, ke = ((w + 1) * ks) / kSplit;
  const double *Ka = K + (size_t)(rt * 16 + g) * s.kpad + t;
  const double *Kb = Ka + (size_t)8 * s.kpad;
  const double *Gp = G + ((size_t)kb * 4 + t) * 6 * ld + mb;
  const size_t gstep = (size_t)4 * 6 * ld;
  for (int kk = kb; kk < ke; kk++) {
    const int k0 = kk * 4;
    const double a0 = __ldg(Ka + k0), a1 = __ldg(Kb + k0);
#pragma unroll
    for (int q = 0; q < 6; q++) dmma16x8x4(acc[q], a0, a1, __ldg(Gp + (size_t)q * ld));
    Gp += gstep;
  }
  if (w > 0) {
    double *pw = part + ((size_t)(w - 1) * 32 + lane) * 24;
#pragma unroll
    for (int q = 0; q < 6; q++)
#pragma unroll
      for (int i = 0; i < 4; i++) pw[q * 4 + i] = acc[q][i];
  }
  __syncthreads();
  if (w == 0) {
    for (int v = 1; v < kSplit; v++) {
      const double *pv = part + ((size_t)(v - 1) * 32 + lane) * 24;
#pragma unroll
      for (int q = 0; q < 6; q++)
#pragma unroll
        for (int i = 0; i < 4; i++) acc[q][i] += pv[q * 4 + i];
    }
    double emax[2] = {0.0, 0.0};
    int mc[2];
#pragma unroll
    for (int e = 0; e < 2; e++) {
      const int ec = e0 + 2 * t + e;
      mc[e] = (ec < ncols) ? (DIAG ? ec : map[ec]) : -1;
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int j = 1 + rt * 16 + g + 8 * h;
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int m = mc[e];
        if (j > s.N || m < 0) continue;
        double yn[6];
        const size_t base = (size_t)j * 6 * ld + m;
#pragma unroll
        for (int q = 0; q < 6; q++) {
          yn[q] = c.x[q * ld + m] + acc[q][2 * h + e];
          Ynew[base + (size_t)q * ld] = yn[q];
        }
        if (!DIAG) {
          double d[6];
#pragma unroll
          for (int q = 0; q < 6; q++) d[q] = yn[q] - Yold[base + (size_t)q * ld];
          if (R32)  // the sweep's residual, for an FP32 correction solve next round
#pragma unroll
            for (int q = 0; q < 6; q++) R32[base + (size_t)q * ld] = (float)d[q];
          double dr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
          double dv = sqrt(d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
          if (s.relative) {
            const double nr = sqrt(yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2]);
            const double nv = sqrt(yn[3] * yn[3] + yn[4] * yn[4] + yn[5] * yn[5]);
            if (nr > 0.0) dr = dr / nr;
            if (nv > 0.0) dv = dv / nv;
          }
          emax[e] = nanmax(emax[e], nanmax(dr, dv));
        }
      }
    }
    // node 0 is the segment's initial state
    if (rt == 0 && g == 0) {
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int m = mc[e];
        if (m >= 0)
#pragma unroll
          for (int q = 0; q < 6; q++) Ynew[(size_t)q * ld + m] = c.x[q * ld + m];
      }
    }
    if (!DIAG) {
#pragma unroll
      for (int e = 0; e < 2; e++) {
        double v = emax[e];
        v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, 4));
        v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, 8));
        v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, 16));
        if (g == 0 && mc[e] >= 0) atomicMax(c.err + mc[e], err_bits(v));
      }
    }
  }
  __syncthreads();  // the partials are reused by the next tile
}

// Sweep contraction over the round's FP64 list: persistent CTAs take tiles
// (row tile fastest, so the CTAs of one column group run together and share F
// in L1/L2) from a counter that the round's setup kernel cleared.
__global__ void __launch_bounds__(32 * kSplit) k_contract(Sweep s, Ctl c, const double *__restrict__ K,
                                                          const double *__restrict__ G,
                                                          const double *__restrict__ Yold, double *__restrict__ Ynew,
                                                          float *__restrict__ R32) {
  __shared__ double part[(kSplit - 1) * 32 * 24];
  __shared__ int tile_sh;
  const int ncols = s.l64_cnt[s.list_cur];
  const int *map = s.l64[s.list_cur];
  const int n_rt = s.rows_pad / 16;
  const int n_tiles = n_rt * ((ncols + 7) / 8);
  for (;;) {
    if (threadIdx.x == 0) tile_sh = atomicAdd(s.tile_ctr, 1);
    __syncthreads();
    const int tile = tile_sh;
    __syncthreads();
    if (tile >= n_tiles) break;
    contract_tile_split<false>(s, c, K, G, Yold, Ynew, tile % n_rt, (tile / n_rt) * 8, ncols, map, part, R32);
  }
}

// Kernel-level entry point: the same tile code over columns 0..n_ic-1.
__global__ void __launch_bounds__(32 * kSplit) k_contract_diag(Sweep s, Ctl c, const double *__restrict__ K,
                                                               const double *__restrict__ G,
                                                               double *__restrict__ Ynew) {
  __shared__ double part[(kSplit - 1) * 32 * 24];
  const int n_rt = s.rows_pad / 16;
  const int ncols = (int)s.n_ic;
  const int n_tiles = n_rt * ((ncols + 7) / 8);
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x)
    contract_tile_split<true>(s, c, K, G, nullptr, Ynew, tile % n_rt, (tile / n_rt) * 8, ncols, nullptr, part,
                              nullptr);
}

// ---------------------------------------------------------------------------
// FP32 sweeps (mixed precision, an extension of the paper), two modes.
//
// KEPLER (new segments): the iterate is y = y_K + delta with y_K the FP64
// warm start.  The Picard map gives delta' = rho + omega2 K (f(y_K + delta) -
// f_K), with f_K the two-body derivative of y_K and rho = x0 + omega2 K f_K -
// y_K the operator's residual on the Kepler arc (below the resolution
// tolerance on accepted segments; dropped here and restored by the FP64
// sweeps that follow).  The central force deviation is formed without
// cancellation (Encke):
//   (mu_c/|r_K|^3) [F(q) (r_K + dr) - dr],  q = dr.(2 r_K + dr)/|r_K|^2,
//   F = 1 - (1+q)^(-3/2) = q s^2 (1 + s + s^2)/(1 + s),  s = (1+q)^(-1/2),
// plus the bodies' terms with r - r_b = (r_K - r_b) + dr, where r_K - r_b was
// formed in FP64 before rounding.  Its rounding error is relative to |delta|,
// not to |y|.
//
// CORRECTION (iterative refinement): an FP64 sweep took the iterate Y to
// Y' = x0 + omega2 K G(Y) with residual R = Y' - Y (kept rounded to FP32).  The
// fixed point Y* satisfies Y* = Y + c with c = R + omega2 K [G(Y + c) - G(Y)],
// solved about the base Y = Y' - R (formed in FP64): the central and every
// body term as Encke differences (base-to-body vectors formed in FP64 then
// rounded), the velocity rows as omega2 c_v.  Then Y* = Y' + omega2 K [G(Y + c)
// - G(Y)] (the last sweep's contraction) is written in FP64.
//
// One CTA per trajectory, one thread per node (the CTA has 32 ceil((N+1)/32)
// threads): a thread keeps its node's deviation in registers across sweeps,
// writes its force row into the CTA's table in shared memory, and forms its
// row of the contraction from K (read coalesced) and the table (broadcast
// reads); the trajectory's node records sit in shared memory for all sweeps.  The sweeps stop when the change is below the FP32 floor
// (or switch_tol, KEPLER), fails to halve the best change for two sweeps, or
// reaches max_iters.  Then the result goes to the next round's buffer and the
// control kernel puts the trajectory on the next round's FP64 list.  A
// non-finite or huge change: KEPLER leaves the trajectory in the FP32 phase
// with that change and the control kernel halves the segment; CORRECTION
// keeps Y' and allows no further corrections in this segment attempt.
// ---------------------------------------------------------------------------
constexpr float kFp32Floor = 2e-6f;
// A correction solve stops at a change below 2e-5 of the correction: the FP64
// sweep after it measures the change and decides convergence, so the floor
// only trades FP32 sweeps against FP64 ones.  On config 3, 2e-5 cuts 8 % of the
// FP32 sweeps with the same FP64 sweeps as 2e-6; 1e-4 adds 2 % FP64 sweeps.
constexpr float kFp32CorrFloor = 2e-5f;
constexpr int kFp32MaxThreads = 288;  // N + 1 <= 288

// Shared-memory stride of a node record: an odd number of float4 so that the
// 16-byte reads of consecutive threads fall in different bank groups.
__host__ __device__ constexpr int fp32_rec_stride(int xs) { return ((xs / 4) % 2 == 0) ? xs + 4 : xs; }
enum : int { FP32_KEPLER = 0, FP32_CORR = 1 };

__device__ __forceinline__ float encke_F(float q) {
  const float sq = rsqrtf(1.0f + q);
  return q * sq * sq * (1.0f + sq + sq * sq) / (1.0f + sq);
}

template <int MODE>
__global__ void __launch_bounds__(kFp32MaxThreads) k_fp32(Sweep s, Ctl c, Model md, const float *__restrict__ K32T,
                                                        const float *__restrict__ mu32, const double *__restrict__ Yc,
                                                        double *__restrict__ Yn, const double *__restrict__ E,
                                                        const float *__restrict__ R32, Mix mx) {
  extern __shared__ float4 fp32_sm4[];
  const int xss = fp32_rec_stride(mx.xs);
  float *Rs = reinterpret_cast<float *>(fp32_sm4);  // [n][xss] node records of the CTA's trajectory
  float *Gs = Rs + (size_t)s.n * xss;               // [n][6] force table
  float *red = Gs + (size_t)s.n * 6;                // [2][warps] change / size partial maxima
  const int j = threadIdx.x, lane = j & 31, warp = j >> 5, nw = blockDim.x >> 5;
  const int N = s.N, n = s.n, ld = s.ld, B = md.B, np = 32 * ((N + 32) / 32);
  const bool node = j <= N;
  const int cur = s.list_cur;
  const int count = MODE == FP32_KEPLER ? s.list_cnt[cur] : s.lc_cnt[cur];
  const int *list = MODE == FP32_KEPLER ? s.list[cur] : s.lc[cur];
  const int boff = MODE == FP32_KEPLER ? 3 : 4;  // float4 index of the first body record
  for (int e = blockIdx.x; e < count; e += gridDim.x) {
    const int m = list[e];
    const float w2f = (float)c.w2[m];
    const float4 *rc = reinterpret_cast<const float4 *>(Rs + (size_t)(node ? j : 0) * xss);
    const size_t yb = (size_t)j * 6 * ld + m;
    if (node) {
      // the node record written by the set-up kernel (k_setup for new segments,
      // k_corr_setup for correction solves), to shared memory
      const float4 *src = reinterpret_cast<const float4 *>(mx.X32 + ((size_t)e * n + j) * mx.xs);
      float4 *dst = reinterpret_cast<float4 *>(Rs + (size_t)j * xss);
      for (int v = 0; v < mx.xs / 4; v++) dst[v] = src[v];
    }
    float dl[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, acc[6];
    float res[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (MODE == FP32_CORR && node) {
      const float4 r0 = rc[2], r1 = rc[3];
      res[0] = r0.x; res[1] = r0.y; res[2] = r0.z; res[3] = r0.w; res[4] = r1.x; res[5] = r1.y;
    }
    float ebest = __int_as_float(0x7f800000), efin = 0.0f;
    int nst = 0, it = 0;
    bool fail = false;
    for (;;) {
      // force deviation at this thread's node
      if (node) {
        const float4 rk = rc[0];
        const float d0 = dl[0], d1 = dl[1], d2 = dl[2];
        const float rr = rk.x * rk.x + rk.y * rk.y + rk.z * rk.z;
        const float F = encke_F((d0 * (2.0f * rk.x + d0) + d1 * (2.0f * rk.y + d1) + d2 * (2.0f * rk.z + d2)) / rr);
        float a0 = rk.w * (F * (rk.x + d0) - d0);
        float a1 = rk.w * (F * (rk.y + d1) - d1);
        float a2 = rk.w * (F * (rk.z + d2) - d2);
        for (int b = 0; b < B; b++) {
          const float4 D = rc[boff + b];
          if (MODE == FP32_KEPLER) {
            const float x0 = D.x + d0, x1 = D.y + d1, x2 = D.z + d2;
            const float ds = rsqrtf(x0 * x0 + x1 * x1 + x2 * x2);
            const float kb = mu32[b] * ds * ds * ds;
            a0 -= kb * x0;
            a1 -= kb * x1;
            a2 -= kb * x2;
          } else {
            const float dd = D.x * D.x + D.y * D.y + D.z * D.z;
            const float Fb = encke_F((d0 * (2.0f * D.x + d0) + d1 * (2.0f * D.y + d1) + d2 * (2.0f * D.z + d2)) / dd);
            a0 += D.w * (Fb * (D.x + d0) - d0);
            a1 += D.w * (Fb * (D.y + d1) - d1);
            a2 += D.w * (Fb * (D.z + d2) - d2);
          }
        }
        if (MODE == FP32_KEPLER && md.indirect) {
          const float4 ai = rc[2];
          a0 -= ai.x;
          a1 -= ai.y;
          a2 -= ai.z;
        }
        float2 *g = reinterpret_cast<float2 *>(Gs + (size_t)j * 6);
        g[0] = make_float2(w2f * dl[3], w2f * dl[4]);
        g[1] = make_float2(w2f * dl[5], w2f * a0);
        g[2] = make_float2(w2f * a1, w2f * a2);
      }
      __syncthreads();
      // this node's row of the contraction
#pragma unroll
      for (int q = 0; q < 6; q++) acc[q] = 0.0f;
      if (s.order == 2) {
        // second-order form: velocity rows from the accelerations, then the
        // position rows from omega2 times the new velocity deviations
        if (node) {
          const float *kr = K32T + j;
#pragma unroll 8
          for (int k = 0; k < n; k++) {
            const float kv = __ldg(kr + (size_t)k * np);
            const float *g = Gs + k * 6;
            acc[3] = fmaf(kv, g[3], acc[3]);
            acc[4] = fmaf(kv, g[4], acc[4]);
            acc[5] = fmaf(kv, g[5], acc[5]);
          }
        }
        __syncthreads();  // every thread has read the acceleration rows
        // the position rows integrate the change of the sweep's velocities:
        // delta_v (new segment) or c_v - R_v (correction after a second-order
        // FP64 sweep, whose residual already holds R_v)
        if (node)
#pragma unroll
          for (int q = 0; q < 3; q++) Gs[j * 6 + q] = w2f * acc[3 + q];
        __syncthreads();
        if (node) {
          const float *kr = K32T + j;
#pragma unroll 8
          for (int k = 0; k < n; k++) {
            const float kv = __ldg(kr + (size_t)k * np);
            const float *g = Gs + k * 6;
            acc[0] = fmaf(kv, g[0], acc[0]);
            acc[1] = fmaf(kv, g[1], acc[1]);
            acc[2] = fmaf(kv, g[2], acc[2]);
          }
        }
      } else if (node) {
        const float *kr = K32T + j;
#pragma unroll 8
        for (int k = 0; k < n; k++) {
          const float kv = __ldg(kr + (size_t)k * np);
          const float2 *g2 = reinterpret_cast<const float2 *>(Gs + k * 6);
          const float2 ga = g2[0], gb = g2[1], gc = g2[2];
          acc[0] = fmaf(kv, ga.x, acc[0]);
          acc[1] = fmaf(kv, ga.y, acc[1]);
          acc[2] = fmaf(kv, gb.x, acc[2]);
          acc[3] = fmaf(kv, gb.y, acc[3]);
          acc[4] = fmaf(kv, gc.x, acc[4]);
          acc[5] = fmaf(kv, gc.y, acc[5]);
        }
      }
      // change and size of the deviation, relative to the iterate
      float emax = 0.0f, dmax = 0.0f;
      if (node) {
        const float4 rk = rc[0], vk = rc[1];
        const float yk[6] = {rk.x, rk.y, rk.z, vk.x, vk.y, vk.z};
        float d[6], y[6], cn[6];
#pragma unroll
        for (int q = 0; q < 6; q++) {
          cn[q] = res[q] + acc[q];
          d[q] = cn[q] - dl[q];
          y[q] = yk[q] + cn[q];
          dl[q] = cn[q];
        }
        float dr = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        float dv = sqrtf(d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
        float mr = sqrtf(cn[0] * cn[0] + cn[1] * cn[1] + cn[2] * cn[2]);
        float mv = sqrtf(cn[3] * cn[3] + cn[4] * cn[4] + cn[5] * cn[5]);
        if (s.relative) {
          const float nr = sqrtf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
          const float nv = sqrtf(y[3] * y[3] + y[4] * y[4] + y[5] * y[5]);
          if (nr > 0.0f) { dr /= nr; mr /= nr; }
          if (nv > 0.0f) { dv /= nv; mv /= nv; }
        }
        emax = nanmaxf(dr, dv);
        dmax = fmaxf(mr, mv);
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        emax = nanmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      }
      if (lane == 0) {
        red[warp] = emax;
        red[nw + warp] = dmax;
      }
      __syncthreads();
      emax = 0.0f;
      dmax = 0.0f;
      for (int w = 0; w < nw; w++) {
        emax = nanmaxf(emax, red[w]);
        dmax = fmaxf(dmax, red[nw + w]);
      }
      it++;
      efin = emax;
      if (!((double)emax <= s.div_limit)) {
        fail = true;
        break;
      }
      // The FP32 floor: the change cannot fall much below the rounding of the
      // contraction, ~sqrt(N) FP32 ulps of the deviation itself, so a change
      // under kFp32Floor * max|deviation|/|y| ends the phase (a correction
      // solve: kFp32CorrFloor times its correction).  Failing to halve
      // the best change for two sweeps (fluctuation at the floor) also ends it.
      if (emax < 0.5f * ebest) {
        nst = 0;
      } else {
        nst++;
      }
      ebest = fminf(ebest, emax);
      if ((MODE == FP32_KEPLER && (double)emax < s.switch_tol) ||
          emax < (MODE == FP32_CORR ? kFp32CorrFloor : kFp32Floor) * dmax || nst >= 2 ||
          it >= s.max_iters)
        break;
      __syncthreads();  // the table is rewritten by the next sweep
    }
    if (node) {
      if (MODE == FP32_KEPLER) {
        if (!fail) {
          const double *yk = mx.YK + ((size_t)e * n + j) * 6;
#pragma unroll
          for (int q = 0; q < 6; q++) Yn[yb + (size_t)q * ld] = yk[q] + (double)dl[q];
        }
      } else {
#pragma unroll
        for (int q = 0; q < 6; q++) Yn[yb + (size_t)q * ld] = Yc[yb + (size_t)q * ld] + (fail ? 0.0 : (double)acc[q]);
      }
    }
    if (j == 0) {
      c.sweeps[m] += it;
      atomicAdd(s.cnt64 + 1, (unsigned long long)it);
      if (MODE == FP32_KEPLER) {
        if (fail) {
          c.err32[m] = err_bits32(efin);
        } else {
          c.phase[m] = PH_READY64;
          c.seg_sweeps[m] = 0;
          c.nstall[m] = 0;
          c.e_best[m] = __longlong_as_double(0x7FF0000000000000LL);
        }
      } else {
        if (fail) c.ncorr[m] = s.max_corr;
        c.phase[m] = PH_READY64;
      }
    }
    __syncthreads();  // the table and the partial maxima are reused by the next trajectory
  }
}

// ---------------------------------------------------------------------------
// FP32 sweeps, tiled: the same two modes and the same arithmetic per
// trajectory as k_fp32, with T trajectories ("slots") per CTA so that one
// copy of the FP32 operator in shared memory serves all of them.
//
// Thread (rg, t) owns output rows rg*R .. rg*R + R - 1 (nodes rg*R + 1 ..
// rg*R + R; row 0 of K is zero, so node 0 never changes) of slot t: it keeps
// those nodes' deviations in registers across sweeps, evaluates their force
// rows (thread rg = 0 also node 0) into the CTA's table G[k][t][6] in shared
// memory, and accumulates its R x 6 block of K G over k = 0..N in ascending
// order with one fused multiply-add per term -- the order k_fp32 uses, so
// every trajectory's result is bitwise that of k_fp32.  A warp is 4 row
// groups x 8 slots: the operator reads of a warp touch 4 rows (broadcast to 8
// lanes each), the table reads 8 slots (broadcast to 4 lanes each).
//
// Slots are filled from the round's list: slot t of CTA b starts with entry
// t * gridDim + b (so a short list spreads over all CTAs), and a slot whose
// trajectory stops takes the next entry from a counter -- converged
// trajectories leave the working set after every sweep.  The per-slot stop
// decision is made by thread t after the change and size maxima of the
// slot's rows are reduced.
// ---------------------------------------------------------------------------
constexpr int kFp32tMaxThreads = 256;   // node records staged in shared memory
constexpr int kFp32tMaxThreadsG = 512;  // node records read from global memory (4 rows per thread)
__host__ __device__ constexpr int fp32t_max_threads(int R, bool rsm) {
  return rsm ? kFp32tMaxThreads : (R == 4 ? kFp32tMaxThreadsG : kFp32tMaxThreads);
}
constexpr int kFp32tMaxSlots = 64;

struct Fp32Slots {
  int e[kFp32tMaxSlots];       // list entry of the slot's trajectory (-1: idle)
  int m[kFp32tMaxSlots];       // its control slot
  float w2[kFp32tMaxSlots];    // its omega2
  int it[kFp32tMaxSlots], nst[kFp32tMaxSlots], stop[kFp32tMaxSlots];
  float ebest[kFp32tMaxSlots];
};

// Force row of one node in FP32 (deviation d, node record rc), the arithmetic
// of k_fp32.
template <int MODE>
__device__ __forceinline__ void fp32_force_row(const float4 *__restrict__ rc, int B, const float *__restrict__ mus,
                                               int indirect, const float d[6], float w2f, float g[6]) {
  const int boff = MODE == FP32_KEPLER ? 3 : 4;
  const float4 rk = rc[0];
  const float d0 = d[0], d1 = d[1], d2 = d[2];
  const float rr = rk.x * rk.x + rk.y * rk.y + rk.z * rk.z;
  const float F = encke_F((d0 * (2.0f * rk.x + d0) + d1 * (2.0f * rk.y + d1) + d2 * (2.0f * rk.z + d2)) / rr);
  float a0 = rk.w * (F * (rk.x + d0) - d0);
  float a1 = rk.w * (F * (rk.y + d1) - d1);
  float a2 = rk.w * (F * (rk.z + d2) - d2);
  for (int b = 0; b < B; b++) {
    const float4 D = rc[boff + b];
    if (MODE == FP32_KEPLER) {
      const float x0 = D.x + d0, x1 = D.y + d1, x2 = D.z + d2;
      const float ds = rsqrtf(x0 * x0 + x1 * x1 + x2 * x2);
      const float kb = mus[b] * ds * ds * ds;
      a0 -= kb * x0;
      a1 -= kb * x1;
      a2 -= kb * x2;
    } else {
      const float dd = D.x * D.x + D.y * D.y + D.z * D.z;
      const float Fb = encke_F((d0 * (2.0f * D.x + d0) + d1 * (2.0f * D.y + d1) + d2 * (2.0f * D.z + d2)) / dd);
      a0 += D.w * (Fb * (D.x + d0) - d0);
      a1 += D.w * (Fb * (D.y + d1) - d1);
      a2 += D.w * (Fb * (D.z + d2) - d2);
    }
  }
  if (MODE == FP32_KEPLER && indirect) {
    const float4 ai = rc[2];
    a0 -= ai.x;
    a1 -= ai.y;
    a2 -= ai.z;
  }
  g[0] = w2f * d[3];
  g[1] = w2f * d[4];
  g[2] = w2f * d[5];
  g[3] = w2f * a0;
  g[4] = w2f * a1;
  g[5] = w2f * a2;
}

// Correction-solve node record (k_fp32's CORR layout, with the node's
// residual) of node j of trajectory m, written to rec.
__device__ __forceinline__ void fp32_corr_record(const Sweep &s, const Model &md, const float *__restrict__ mus,
                                                 const double *__restrict__ Yc, const double *__restrict__ E,
                                                 const float *__restrict__ R32, int j, int m, float4 *rec) {
  const int ld = s.ld, B = md.B;
  const size_t yb = (size_t)j * 6 * ld + m;
  double base[6];
  float res[6];
#pragma unroll
  for (int q = 0; q < 6; q++) {
    res[q] = (j == 0) ? 0.0f : R32[yb + (size_t)q * ld];
    base[q] = Yc[yb + (size_t)q * ld] - (double)res[q];
  }
  const float bx = (float)base[0], by = (float)base[1], bz = (float)base[2];
  const float ir = rsqrtf(bx * bx + by * by + bz * bz);
  rec[0] = make_float4(bx, by, bz, (float)md.mu_c * ir * ir * ir);
  rec[1] = make_float4((float)base[3], (float)base[4], (float)base[5], 0.0f);
  rec[2] = make_float4(res[0], res[1], res[2], res[3]);
  rec[3] = make_float4(res[4], res[5], 0.0f, 0.0f);
  for (int b = 0; b < B; b++) {
    const double *eb = E + (size_t)(j * B + b) * 3 * ld + m;
    const float dx = (float)(base[0] - eb[0]), dy = (float)(base[1] - eb[(size_t)ld]),
                dz = (float)(base[2] - eb[(size_t)2 * ld]);
    const float id = rsqrtf(dx * dx + dy * dy + dz * dz);
    rec[4 + b] = make_float4(dx, dy, dz, mus[b] * id * id * id);
  }
}

// Correction-solve records: for every entry e of the round's correction list
// and every node j, the record of fp32_corr_record in X32[e][j] (grid-stride
// over entries x nodes, entries fastest, so neighbouring threads read
// neighbouring slots of the FP64 arrays).  Runs after the new-segment FP32
// kernel, which is done with X32, and before the correction solves.
__global__ void k_corr_setup(Sweep s, Model md, const float *__restrict__ mu32, const double *__restrict__ Yc,
                             const double *__restrict__ E, const float *__restrict__ R32, Mix mx) {
  const int cur = s.list_cur;
  const long long count = s.lc_cnt[cur];
  const int *__restrict__ list = s.lc[cur];
  const long long total = count * s.n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / count);
    const long long e = i - (long long)j * count;
    fp32_corr_record(s, md, mu32, Yc, E, R32, j, list[e],
                     reinterpret_cast<float4 *>(mx.X32 + ((size_t)e * s.n + j) * mx.xs));
  }
}

// Shared-memory layout of the tiled FP32 kernel (floats): operator (when
// staged), force table, MMA output table (tensor-core contraction), node
// records of the slots (when staged), reduction partials, GMs.  With the
// tensor-core contraction the operator rows are 16 MT + 8 floats long and the
// table rows 6T + 8 (k-rows padded to a multiple of 8 with zeros), so that
// the fragment loads of a warp fall in 32 distinct banks.
struct Fp32tLayout {
  size_t ks, gs, os, rs;  // sizes of the four arrays
  int kst, gst;           // row strides of the operator and the force table
};
__host__ __device__ inline Fp32tLayout fp32t_layout(int N, int n, int rows32, int T, bool ksm, bool rsm, bool mma,
                                                    int B) {
  Fp32tLayout L;
  const int MT = (N + 15) / 16, kp8 = (n + 7) / 8 * 8;
  L.kst = mma ? 16 * MT + 8 : rows32;
  L.gst = 6 * T + (mma ? 8 : 0);
  L.ks = ksm ? (size_t)(mma ? kp8 : n) * L.kst : 0;
  L.gs = (size_t)(mma ? kp8 : n) * L.gst;
  L.os = mma ? (size_t)16 * MT * L.gst : 0;
  L.rs = rsm ? (size_t)T * n * fp32_rec_stride(x32_stride(B)) : 0;
  return L;
}
__host__ __device__ inline size_t fp32t_smem_bytes(int N, int n, int rows32, int T, int RG, bool ksm, bool rsm,
                                                   bool mma, int B) {
  const Fp32tLayout L = fp32t_layout(N, n, rows32, T, ksm, rsm, mma, B);
  return sizeof(float) * (L.ks + L.gs + L.os + L.rs + 2 * (size_t)T * (RG / 4) + B + 4);
}

// TF32 high part of x: x rounded to 10 mantissa bits (to nearest, ties away
// from zero: half a TF32 ulp added to the bit pattern, the low 13 bits
// cleared), as mma operand bits.  x - hi is exact in FP32, at most 2^-11 |x|
// and of either sign; passed as an operand, the tensor core keeps its leading
// 11 bits, so hi and lo together carry x to about 2^-22.  Integer operations
// instead of conversions, which run at a fraction of the FP32 rate.
__device__ __forceinline__ unsigned tf32_hi(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }
__device__ __forceinline__ void mma_tf32_1688(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The operator contraction of one FP32 sweep (or pass) on the tensor cores:
// O[r][c] = sum_k K[r+1][k] G[k][c] over the CTA's T slots, column c = (slot
// c / NC, component Q0 + c % NC).  Each operand is split into TF32 high and
// low parts and the product taken as K_lo G_hi + K_hi G_lo + K_hi G_hi (the
// dropped K_lo G_lo is below 2^-22 of the term), accumulated in FP32: close
// to the accuracy of FP32 multiply-adds.  The CTA's MT x (T/8) warps each take
// one 16-row tile and NC column tiles of 8; A fragments come from the operator
// (Ks[k][r]), B fragments from the force table, and the results go to Os.
template <int NC, int Q0>
__device__ __forceinline__ void fp32_mma_contract(const float *__restrict__ Ks, int kst, const float *__restrict__ Gs,
                                                  int gst, float *__restrict__ Os, int MT, int kp8) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const int mt = w % MT, part = w / MT;
  float acc[NC][4];
  int boff[NC];
#pragma unroll
  for (int jn = 0; jn < NC; jn++) {
#pragma unroll
    for (int i = 0; i < 4; i++) acc[jn][i] = 0.0f;
    const int col = (part * NC + jn) * 8 + g;
    boff[jn] = (col / NC) * 6 + Q0 + col % NC;
  }
  const float *A0 = Ks + mt * 16 + g;
  for (int k0 = 0; k0 < kp8; k0 += 8) {
    const float *Ak = A0 + (size_t)(k0 + t4) * kst;
    const float av[4] = {Ak[0], Ak[8], Ak[(size_t)4 * kst], Ak[(size_t)4 * kst + 8]};
    unsigned ah[4], al[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      ah[i] = tf32_hi(av[i]);
      al[i] = __float_as_uint(av[i] - __uint_as_float(ah[i]));
    }
    const float *Bk = Gs + (size_t)(k0 + t4) * gst;
#pragma unroll
    for (int jn = 0; jn < NC; jn++) {
      const float b0 = Bk[boff[jn]], b1 = Bk[(size_t)4 * gst + boff[jn]];
      const unsigned bh0 = tf32_hi(b0), bh1 = tf32_hi(b1);
      const unsigned bl0 = __float_as_uint(b0 - __uint_as_float(bh0)), bl1 = __float_as_uint(b1 - __uint_as_float(bh1));
      mma_tf32_1688(acc[jn], al, bh0, bh1);
      mma_tf32_1688(acc[jn], ah, bl0, bl1);
      mma_tf32_1688(acc[jn], ah, bh0, bh1);
    }
  }
#pragma unroll
  for (int jn = 0; jn < NC; jn++) {
    const int col = (part * NC + jn) * 8 + 2 * t4;
    *reinterpret_cast<float2 *>(Os + (size_t)(mt * 16 + g) * gst + col) = make_float2(acc[jn][0], acc[jn][1]);
    *reinterpret_cast<float2 *>(Os + (size_t)(mt * 16 + g + 8) * gst + col) = make_float2(acc[jn][2], acc[jn][3]);
  }
}

// 16-byte asynchronous copy global -> shared (no register staging).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

template <int MODE, int R, bool KSM, bool RSM, bool MMA>
__global__ void __launch_bounds__(fp32t_max_threads(R, RSM), 1)
    k_fp32t(Sweep s, Ctl c, Model md, const float *__restrict__ K32R, int rows32, const float *__restrict__ mu32,
            const double *__restrict__ Yc, double *__restrict__ Yn, const double *__restrict__ E,
            const float *__restrict__ R32, Mix mx, int T) {
  extern __shared__ float4 fp32t_sm4[];
  __shared__ Fp32Slots sl;
  const int N = s.N, n = s.n, ld = s.ld, B = md.B;
  const int RG = blockDim.x / T, RG4 = RG / 4;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int rg_hi = wid % RG4, rg = rg_hi * 4 + (lane & 3), t = (wid / RG4) * 8 + (lane >> 2);
  const Fp32tLayout lay = fp32t_layout(N, n, rows32, T, KSM, RSM, MMA, B);
  const int gst = lay.gst, MT = (N + 15) / 16, kp8 = (n + 7) / 8 * 8;
  float *Ks = reinterpret_cast<float *>(fp32t_sm4);          // [n or kp8][kst] when KSM
  float *Gs = Ks + lay.ks;                                     // [n or kp8][gst]: slot t at t * 6
  float *Os = Gs + lay.gs;                                     // [16 MT][gst] tensor-core results (MMA)
  const int xs4 = mx.xs / 4, xss = fp32_rec_stride(mx.xs), xss4 = xss / 4;
  float *Rs = Os + lay.os;                                     // [T][n][xss] node records of the slots (RSM)
  float *red = Rs + lay.rs;                                    // [2][T][RG4]
  const int rstr = RSM ? xss4 : xs4;                           // float4s between the node records
  float *mus = red + 2 * T * RG4;                              // [B]
  const int cur = s.list_cur;
  const int count = MODE == FP32_KEPLER ? s.list_cnt[cur] : s.lc_cnt[cur];
  const int *list = MODE == FP32_KEPLER ? s.list[cur] : s.lc[cur];
  if ((int)blockIdx.x >= count) return;  // no entry for this CTA, now or later
  int *ctr = s.fp32_ctr + (MODE == FP32_KEPLER ? 0 : 1);
  const int first_refill = gridDim.x * T;

  if (MMA) {
    // operator rows padded to kst, k-rows n..kp8-1 of both tables zero
    for (int i = tid; i < kp8 * lay.kst; i += blockDim.x) {
      const int k = i / lay.kst, r = i - k * lay.kst;
      Ks[i] = (k < n && r < rows32) ? __ldg(K32R + (size_t)k * rows32 + r) : 0.0f;
    }
    for (int i = n * gst + tid; i < kp8 * gst; i += blockDim.x) Gs[i] = 0.0f;
  } else if (KSM) {
    for (int i = tid; i < n * rows32 / 4; i += blockDim.x)
      reinterpret_cast<float4 *>(Ks)[i] = __ldg(reinterpret_cast<const float4 *>(K32R) + i);
  }
  for (int b = tid; b < B; b += blockDim.x) mus[b] = mu32[b];
  if (tid < T) {
    const int e = tid * gridDim.x + blockIdx.x;
    const bool ok = e < count;
    sl.e[tid] = ok ? e : -1;
    sl.m[tid] = ok ? list[e] : 0;
    sl.w2[tid] = ok ? (float)c.w2[list[e]] : 0.0f;
    sl.it[tid] = 0;
    sl.nst[tid] = 0;
    sl.stop[tid] = 0;
    sl.ebest[tid] = __int_as_float(0x7f800000);
  }
  __syncthreads();

  // the thread's rows: R consecutive nodes from j0 (the multiply-add
  // contraction loads them as float4s), or with the tensor-core contraction
  // nodes 1 + rg + i RG, so that neighbouring lanes own neighbouring rows of
  // the force and result tables (distinct banks) and node records
  const int j0 = rg * R + 1;
  auto row = [&](int i) { return MMA ? 1 + rg + i * RG : j0 + i; };
  const float *Kk = KSM ? Ks + rg * R : K32R + rg * R;
  const float *Gk = Gs + t * 6;
  int e = sl.e[t];
  int m = sl.m[t];
  float w2f = sl.w2[t];
  bool fresh = true;
  // the slot's node records (written by the set-up kernels) to shared memory,
  // once per trajectory, by the slot's threads
  auto load_records = [&](int entry) {
    const float4 *src = reinterpret_cast<const float4 *>(mx.X32) + (size_t)entry * n * xs4;
    float4 *dst = reinterpret_cast<float4 *>(Rs) + (size_t)t * n * xss4;
    for (int idx = rg; idx < n * xs4; idx += RG) {
      const int j = idx / xs4, v = idx - j * xs4;
      cp_async16(dst + (size_t)j * xss4 + v, src + idx);
    }
  };
  if (RSM && e >= 0) load_records(e);
  cp_async_wait_all();
  __syncthreads();
  float dl[R][6], acc[R][6];
  for (;;) {
    const bool live = e >= 0;
    if (live && fresh) {
#pragma unroll
      for (int i = 0; i < R; i++)
#pragma unroll
        for (int q = 0; q < 6; q++) dl[i][q] = 0.0f;
    }
    fresh = false;
    // force rows of the thread's nodes
    const float4 *rb = RSM ? reinterpret_cast<const float4 *>(Rs) + (size_t)t * n * xss4
                           : reinterpret_cast<const float4 *>(mx.X32) + (size_t)(e >= 0 ? e : 0) * n * xs4;
    if (live) {
      float g[6];
      if (rg == 0) {
        const float z[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        fp32_force_row<MODE>(rb, B, mus, md.indirect, z, w2f, g);
        float2 *gp = reinterpret_cast<float2 *>(Gs + t * 6);
        gp[0] = make_float2(g[0], g[1]);
        gp[1] = make_float2(g[2], g[3]);
        gp[2] = make_float2(g[4], g[5]);
      }
#pragma unroll
      for (int i = 0; i < R; i++) {
        const int j = row(i);
        if (j <= N) {
          fp32_force_row<MODE>(rb + (size_t)j * rstr, B, mus, md.indirect, dl[i], w2f, g);
          float2 *gp = reinterpret_cast<float2 *>(Gs + (size_t)j * gst + t * 6);
          gp[0] = make_float2(g[0], g[1]);
          gp[1] = make_float2(g[2], g[3]);
          gp[2] = make_float2(g[4], g[5]);
        }
      }
    }
    __syncthreads();
    // the thread's R x 6 block of K G, k ascending (second-order form: the
    // velocity rows from the accelerations, then the position rows from
    // omega2 times the new velocity deviations written into the table)
    float emax = 0.0f, dmax = 0.0f;
    auto contract = [&](int q0, int nq) {
#pragma unroll 2
      for (int k = 0; k < n; k++) {
        float kv[R];
#pragma unroll
        for (int i = 0; i < R; i += 4) {
          const float4 k4 = KSM ? *reinterpret_cast<const float4 *>(Kk + (size_t)k * rows32 + i)
                                : __ldg(reinterpret_cast<const float4 *>(Kk + (size_t)k * rows32 + i));
          kv[i] = k4.x;
          kv[i + 1] = k4.y;
          kv[i + 2] = k4.z;
          kv[i + 3] = k4.w;
        }
        const float *gk = Gk + (size_t)k * gst;
        if (nq == 6) {
          const float2 *g2 = reinterpret_cast<const float2 *>(gk);
          const float2 ga = g2[0], gb = g2[1], gc = g2[2];
#pragma unroll
          for (int i = 0; i < R; i++) {
            acc[i][0] = fmaf(kv[i], ga.x, acc[i][0]);
            acc[i][1] = fmaf(kv[i], ga.y, acc[i][1]);
            acc[i][2] = fmaf(kv[i], gb.x, acc[i][2]);
            acc[i][3] = fmaf(kv[i], gb.y, acc[i][3]);
            acc[i][4] = fmaf(kv[i], gc.x, acc[i][4]);
            acc[i][5] = fmaf(kv[i], gc.y, acc[i][5]);
          }
        } else {
          const float g0 = gk[q0], g1 = gk[q0 + 1], g2v = gk[q0 + 2];
#pragma unroll
          for (int i = 0; i < R; i++) {
            acc[i][q0] = fmaf(kv[i], g0, acc[i][q0]);
            acc[i][q0 + 1] = fmaf(kv[i], g1, acc[i][q0 + 1]);
            acc[i][q0 + 2] = fmaf(kv[i], g2v, acc[i][q0 + 2]);
          }
        }
      }
    };
    if (live)
#pragma unroll
      for (int i = 0; i < R; i++)
#pragma unroll
        for (int q = 0; q < 6; q++) acc[i][q] = 0.0f;
    if (MMA) {
      // the whole CTA runs each pass on the tensor cores into Os (row j - 1 =
      // rg R + i, column t NC + component), then each thread takes its block
      if (s.order == 2) {
        fp32_mma_contract<3, 3>(Ks, lay.kst, Gs, gst, Os, MT, kp8);
        __syncthreads();
        if (live)
#pragma unroll
          for (int i = 0; i < R; i++) {
            const int j = row(i);
#pragma unroll
            for (int q = 0; q < 3; q++) acc[i][3 + q] = Os[(size_t)(j - 1) * gst + t * 3 + q];
            if (j <= N)
#pragma unroll
              for (int q = 0; q < 3; q++) Gs[(size_t)j * gst + t * 6 + q] = w2f * acc[i][3 + q];
          }
        __syncthreads();  // the table's velocity rows hold the new deviations
        fp32_mma_contract<3, 0>(Ks, lay.kst, Gs, gst, Os, MT, kp8);
        __syncthreads();
        if (live)
#pragma unroll
          for (int i = 0; i < R; i++)
#pragma unroll
            for (int q = 0; q < 3; q++) acc[i][q] = Os[(size_t)(row(i) - 1) * gst + t * 3 + q];
      } else {
        fp32_mma_contract<6, 0>(Ks, lay.kst, Gs, gst, Os, MT, kp8);
        __syncthreads();
        if (live)
#pragma unroll
          for (int i = 0; i < R; i++)
#pragma unroll
            for (int q = 0; q < 6; q++) acc[i][q] = Os[(size_t)(row(i) - 1) * gst + t * 6 + q];
      }
    } else if (s.order == 2) {
      if (live) {
        contract(3, 3);
#pragma unroll
        for (int i = 0; i < R; i++) {
          const int j = row(i);
          // the position rows integrate the change of the sweep's velocities:
          // delta_v (new segment) or c_v - R_v (correction after a
          // second-order FP64 sweep, whose residual already holds R_v)
          if (j <= N)
#pragma unroll
            for (int q = 0; q < 3; q++) Gs[(size_t)j * gst + t * 6 + q] = w2f * acc[i][3 + q];
        }
      }
      __syncthreads();  // the table's velocity rows hold the new deviations
      if (live) contract(0, 3);
    } else if (live) {
      contract(0, 6);
    }
    if (live) {
      // change and size of the deviation, relative to the iterate
#pragma unroll
      for (int i = 0; i < R; i++) {
        const int j = row(i);
        if (j <= N) {
          const float4 *rj = rb + (size_t)j * rstr;
          const float4 rk = rj[0], vk = rj[1];
          const float yk[6] = {rk.x, rk.y, rk.z, vk.x, vk.y, vk.z};
          float res[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
          if (MODE == FP32_CORR) {
            const float4 ra = rj[2], rv = rj[3];
            res[0] = ra.x; res[1] = ra.y; res[2] = ra.z; res[3] = ra.w; res[4] = rv.x; res[5] = rv.y;
          }
          float d[6], y[6], cn[6];
#pragma unroll
          for (int q = 0; q < 6; q++) {
            cn[q] = res[q] + acc[i][q];
            d[q] = cn[q] - dl[i][q];
            y[q] = yk[q] + cn[q];
            dl[i][q] = cn[q];
          }
          float dr = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
          float dv = sqrtf(d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
          float mr = sqrtf(cn[0] * cn[0] + cn[1] * cn[1] + cn[2] * cn[2]);
          float mv = sqrtf(cn[3] * cn[3] + cn[4] * cn[4] + cn[5] * cn[5]);
          if (s.relative) {
            const float nr = sqrtf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
            const float nv = sqrtf(y[3] * y[3] + y[4] * y[4] + y[5] * y[5]);
            if (nr > 0.0f) { dr /= nr; mr /= nr; }
            if (nv > 0.0f) { dv /= nv; mv /= nv; }
          }
          emax = nanmaxf(emax, nanmaxf(dr, dv));
          dmax = fmaxf(dmax, fmaxf(mr, mv));
        }
      }
    }
    // maxima over the slot's row groups: 4 lanes of the warp, then RG4 warps
    emax = nanmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
    dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, 1));
    emax = nanmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, 2));
    dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, 2));
    if ((lane & 3) == 0) {
      red[t * RG4 + rg_hi] = emax;
      red[(T + t) * RG4 + rg_hi] = dmax;
    }
    __syncthreads();
    // stop decision per slot (k_fp32's rules), bookkeeping, next entry
    bool more = false;
    if (tid < T && sl.e[tid] >= 0) {
      float em = 0.0f, dm = 0.0f;
      for (int h = 0; h < RG4; h++) {
        em = nanmaxf(em, red[tid * RG4 + h]);
        dm = fmaxf(dm, red[(T + tid) * RG4 + h]);
      }
      const int it = sl.it[tid] + 1;
      sl.it[tid] = it;
      int stop = 0;
      if (!((double)em <= s.div_limit)) {
        stop = 2;
      } else {
        int nst = sl.nst[tid];
        const float eb = sl.ebest[tid];
        nst = (em < 0.5f * eb) ? 0 : nst + 1;
        sl.nst[tid] = nst;
        sl.ebest[tid] = fminf(eb, em);
        if ((MODE == FP32_KEPLER && (double)em < s.switch_tol) ||
            em < (MODE == FP32_CORR ? kFp32CorrFloor : kFp32Floor) * dm || nst >= 2 ||
            it >= s.max_iters)
          stop = 1;
      }
      sl.stop[tid] = stop;
      if (stop) {
        const int mm = sl.m[tid];
        c.sweeps[mm] += it;
        atomicAdd(s.cnt64 + 1, (unsigned long long)it);
        if (MODE == FP32_KEPLER) {
          if (stop == 2) {
            c.err32[mm] = err_bits32(em);
          } else {
            c.phase[mm] = PH_READY64;
            c.seg_sweeps[mm] = 0;
            c.nstall[mm] = 0;
            c.e_best[mm] = __longlong_as_double(0x7FF0000000000000LL);
          }
        } else {
          if (stop == 2) c.ncorr[mm] = s.max_corr;
          c.phase[mm] = PH_READY64;
        }
        const int nx = first_refill + atomicAdd(ctr, 1);
        const bool ok = nx < count;
        sl.e[tid] = ok ? nx : -1;
        sl.m[tid] = ok ? list[nx] : 0;
        sl.w2[tid] = ok ? (float)c.w2[list[nx]] : 0.0f;
        sl.it[tid] = 0;
        sl.nst[tid] = 0;
        sl.ebest[tid] = __int_as_float(0x7f800000);
      }
      more = sl.e[tid] >= 0;
    }
    const bool any = __syncthreads_or(more);
    // a stopped slot writes its trajectory's result and takes the next one
    if (live && sl.stop[t]) {
      const bool fail = sl.stop[t] == 2;
      if (MODE == FP32_KEPLER) {
        if (!fail) {
          const double *yk = mx.YK + (size_t)e * n * 6;
          if (rg == 0)
#pragma unroll
            for (int q = 0; q < 6; q++) Yn[(size_t)q * ld + m] = yk[q] + (double)0.0f;
#pragma unroll
          for (int i = 0; i < R; i++) {
            const int j = row(i);
            if (j <= N)
#pragma unroll
              for (int q = 0; q < 6; q++) Yn[((size_t)j * 6 + q) * ld + m] = yk[(size_t)j * 6 + q] + (double)dl[i][q];
          }
        }
      } else {
        if (rg == 0)
#pragma unroll
          for (int q = 0; q < 6; q++) Yn[(size_t)q * ld + m] = Yc[(size_t)q * ld + m] + (double)0.0f;
#pragma unroll
        for (int i = 0; i < R; i++) {
          const int j = row(i);
          if (j <= N)
#pragma unroll
            for (int q = 0; q < 6; q++) {
              const size_t o = ((size_t)j * 6 + q) * ld + m;
              Yn[o] = Yc[o] + (fail ? 0.0 : (double)acc[i][q]);
            }
        }
      }
      e = sl.e[t];
      m = sl.m[t];
      w2f = sl.w2[t];
      fresh = true;
      if (RSM && e >= 0) load_records(e);
    }
    cp_async_wait_all();
    __syncthreads();  // the new trajectories' records are in place
    if (!any) break;
  }
}

// ---------------------------------------------------------------------------
// Resolution test (Chebyshev tail of the force fit).  On the CGL nodes
// T_N(tau_j) = (-1)^(N+j) and T_{N-1}(tau_j) = (-1)^(N+j) tau_j, so the two
// top coefficients of the interpolant of g are
//   a_N = (1/N) sum''_j (-1)^(N+j) g_j,   a_{N-1} = (2/N) sum''_j (-1)^(N+j) tau_j g_j
// (sum'' halves the end terms; the sums come from k_force).  The integrated
// error is about 2 |omega2| (|a_{N-1}| + |a_N|) per unit of g; F already
// carries omega2.  Position components are measured against max_j |r_j|,
// velocity ones against max_j |v_j| of the iterate the force was evaluated on
// (relative mode).
// ---------------------------------------------------------------------------
__device__ double tail_estimate(const Sweep &s, const double *__restrict__ partials, int m) {
  const int ld = s.ld;
  const int nb = (s.n + kForceNodes - 1) / kForceNodes;
  double sums[12], r2 = 0.0, v2 = 0.0;
#pragma unroll
  for (int v = 0; v < 12; v++) sums[v] = 0.0;
  for (int b = 0; b < nb; b++) {
    const double *pp = partials + (size_t)b * kTailVals * ld + m;
#pragma unroll
    for (int v = 0; v < 12; v++) sums[v] += pp[(size_t)v * ld];
    r2 = fmax(r2, pp[(size_t)12 * ld]);
    v2 = fmax(v2, pp[(size_t)13 * ld]);
  }
  const double invN = 1.0 / (double)s.N;
  double er = 0.0, ev = 0.0;
#pragma unroll
  for (int q = 0; q < 6; q++) {
    const double tl = 2.0 * (fabs(2.0 * sums[6 + q] * invN) + fabs(sums[q] * invN));
    if (q < 3) er = nanmax(er, tl); else ev = nanmax(ev, tl);
  }
  if (s.relative) {
    if (r2 > 0.0) er /= sqrt(r2);
    if (v2 > 0.0) ev /= sqrt(v2);
  }
  return nanmax(er, ev);
}

// Per-trajectory decisions after a sweep.  FP64 phase: same rules, same order
// as the oracle (blow-up, tolerance, stall, cap; then the resolution test on an
// accepted segment; accept or halve).  A trajectory still in the FP32 phase
// failed it (blow-up) and is halved.  Finished trajectories write their outputs.  Trajectories doing an FP64 sweep next
// round go on the next FP64 list.  The block size is a multiple of 32 and every
// lane reaches the warp-cooperative steps.
__global__ void k_control(Sweep s, Ctl c, const double *__restrict__ tails, const double *__restrict__ Ynew,
                          int *done) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int phase = (m < s.A) ? c.phase[m] : PH_DONE;
  const bool act = phase == PH_ITER || phase == PH_ITER32;
  const bool ready = phase == PH_READY64;  // FP32 phase done this round: FP64 sweeps from the next
  const int ld = s.ld;
  const int list_next = s.list_cur ^ 1;
  int out = SEG_CONTINUE;
  double e_sweep = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // this round's contraction is over
    *s.tile_ctr = 0;
    *s.tile_ctr2 = 0;
  }
  if (ready) {
    c.need_setup[m] = 0;
    c.phase[m] = PH_ITER;
  }
  {
    const unsigned n64 = __popc(__ballot_sync(0xffffffffu, phase == PH_ITER));
    if (lane == 0 && n64) atomicAdd(s.cnt64, (unsigned long long)n64);
  }
  if (act) {
    c.need_setup[m] = 0;
    if (phase == PH_ITER) {
      c.sweeps[m] += 1;
      const double e = __longlong_as_double((long long)c.err[m]);
      e_sweep = e;
      c.err[m] = 0ULL;
      const int ss = ++c.seg_sweeps[m];
      if (!(e <= s.div_limit)) {
        out = SEG_FAIL_DIV;
      } else if (e < s.tol) {
        out = SEG_OK;
      } else {
        if (e < c.e_best[m]) {
          c.e_best[m] = e;
          c.nstall[m] = 0;
        } else {
          c.nstall[m] += 1;
        }
        if (c.nstall[m] >= s.stall_sweeps && c.e_best[m] < s.stall_factor * s.tol) out = SEG_STALLED;
        else if (ss >= s.max_iters) out = SEG_FAIL_CAP;
      }
    } else {
      // still in the FP32 phase after k_fp32: its change blew up
      c.err32[m] = 0u;
      out = SEG_FAIL_DIV;
    }
  }
  if (act && out != SEG_CONTINUE) {
    if ((out == SEG_OK || out == SEG_STALLED) && s.trunc_tol > 0.0 && !(tail_estimate(s, tails, m) <= s.trunc_tol))
      out = SEG_FAIL_TRUNC;
    const int D = s.max_depth;
    bool accept = (out == SEG_OK || out == SEG_STALLED);
    if (out == SEG_FAIL_TRUNC && c.depth[m] >= D) {
      accept = true;
      c.status[m] |= PC_IC_UNRESOLVED;
    }
    if (accept) {
      if (out == SEG_STALLED) c.status[m] |= PC_IC_STALLED;
      const int k = c.nseg[m];
      if (s.ckpt && k < s.max_ckpt) {
        double *ck = s.ckpt + ((size_t)(s.io_off + c.ic[m]) * s.max_ckpt + k) * 7;
        ck[0] = c.ta[m];
        for (int q = 0; q < 6; q++) ck[1 + q] = c.x[q * ld + m];
      }
      if (s.tape && k < s.tape_seg) {
        double *rec = s.tape + ((size_t)(s.io_off + c.ic[m]) * s.tape_seg + k) * (size_t)tape_rec(s.n);
        rec[0] = c.ta[m];
        rec[1] = c.tb[m];
        for (int j = 0; j < s.n; j++)
          for (int q = 0; q < 6; q++) rec[2 + 6 * j + q] = Ynew[((size_t)j * 6 + q) * ld + m];
      }
      const size_t last_row = (size_t)s.N * 6 * ld + m;
      for (int q = 0; q < 6; q++) c.x[q * ld + m] = Ynew[last_row + (size_t)q * ld];
      c.nseg[m] = k + 1;
      c.p[m] += 1LL << (D - c.depth[m]);
      if (c.last[m]) {
        c.phase[m] = PH_DONE;
        write_outputs(s, c, m);
        atomicAdd(done, 1);
      } else {
        if (c.depth[m] > 0) c.depth[m] -= 1;
        schedule(s, c, m, list_next);
      }
    } else {
      c.depth[m] += 1;
      if (c.depth[m] > D) {
        c.status[m] |= (out == SEG_FAIL_DIV) ? PC_IC_NONFINITE : PC_IC_NOT_CONVERGED;
        c.phase[m] = PH_DONE;
        write_outputs(s, c, m);
        atomicAdd(done, 1);
        atomicAdd(done + 1, 1);
      } else {
        schedule(s, c, m, list_next);
      }
    }
  }
  // an FP64 sweep that left the segment unfinished with a small change: solve
  // for the correction to its iterate in FP32 next round instead of sweeping on
  bool to_corr = false;
  if (act && phase == PH_ITER && out == SEG_CONTINUE && s.refine && e_sweep < s.corr_hi &&
      c.ncorr[m] < s.max_corr) {
    c.phase[m] = PH_CORR32;
    c.ncorr[m] += 1;
    to_corr = true;
  }
  warp_append(to_corr, m, s.lc[list_next], s.lc_cnt + list_next);
  const bool next64 = (act && c.phase[m] == PH_ITER) || ready;
  warp_append(next64, m, s.l64[list_next], s.l64_cnt + list_next);
}

// ---- repack: move active slots to the front of the spare buffers ------------
__global__ void k_repack_pos(int A, const int *__restrict__ phase, int *__restrict__ pos, int *counter) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool alive = m < A && phase[m] != PH_DONE;
  const unsigned mask = __ballot_sync(0xffffffffu, alive);
  int base = 0;
  if (mask) {
    const int leader = __ffs(mask) - 1;
    if (lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
  }
  if (m < A) pos[m] = alive ? base + __popc(mask & ((1u << lane) - 1u)) : -1;
}

// Copies rows [0, rows) of a [rows][ld] array (T = double or float) for every
// slot that moves.
template <typename T>
__global__ void k_repack_rows(int A, int ld, long long rows, const int *__restrict__ pos, const T *__restrict__ src,
                              T *__restrict__ dst) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= A) return;
  const int d = pos[m];
  if (d < 0) return;
  for (long long r = blockIdx.y; r < rows; r += gridDim.y) dst[(size_t)r * ld + d] = src[(size_t)r * ld + m];
}

// Moves the control state and rebuilds the lists the next round reads.  The
// block size is a multiple of 32 and every lane reaches the list append.
__global__ void k_repack_ctl(Sweep s, Ctl a, Ctl b, const int *__restrict__ pos) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int d = (m < s.A) ? pos[m] : -1;
  const int list_next = s.list_cur;  // the list the next round reads
  bool to64 = false;
  if (d >= 0) {
    const int ld = s.ld;
    for (int q = 0; q < 6; q++) b.x[q * ld + d] = a.x[q * ld + m];
    b.t0[d] = a.t0[m];
    b.tf[d] = a.tf[m];
    b.total[d] = a.total[m];
    b.sgn[d] = a.sgn[m];
    b.hbase[d] = a.hbase[m];
    b.ta[d] = a.ta[m];
    b.tb[d] = a.tb[m];
    b.w1[d] = a.w1[m];
    b.w2[d] = a.w2[m];
    b.e_best[d] = a.e_best[m];
    for (int q = 0; q < kKepConsts; q++) b.kc[q * ld + d] = a.kc[q * ld + m];
    b.err[d] = a.err[m];
    b.p[d] = a.p[m];
    b.depth[d] = a.depth[m];
    b.phase[d] = a.phase[m];
    b.status[d] = a.status[m];
    b.sweeps[d] = a.sweeps[m];
    b.seg_sweeps[d] = a.seg_sweeps[m];
    b.nstall[d] = a.nstall[m];
    b.nseg[d] = a.nseg[m];
    b.need_setup[d] = a.need_setup[m];
    b.last[d] = a.last[m];
    b.ic[d] = a.ic[m];
    b.err32[d] = a.err32[m];
    b.ncorr[d] = a.ncorr[m];
    if (a.need_setup[m]) {
      const int k = atomicAdd(s.list_cnt + list_next, 1);
      s.list[list_next][k] = d;
    }
    to64 = a.phase[m] == PH_ITER;
  }
  warp_append(to64, d, s.l64[list_next], s.l64_cnt + list_next);
  warp_append(d >= 0 && a.phase[m] == PH_CORR32, d, s.lc[list_next], s.lc_cnt + list_next);
}

// Round cap reached: remaining trajectories stop with NOT_CONVERGED.
__global__ void k_abort(Sweep s, Ctl c) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= s.A || c.phase[m] == PH_DONE) return;
  c.status[m] |= PC_IC_NOT_CONVERGED;
  c.phase[m] = PH_DONE;
  write_outputs(s, c, m);
}

// ---- kernel-level diagnostics ------------------------------------------------
__global__ void k_eval_ephem(Model md, long long n, const double *__restrict__ t, double *__restrict__ rb) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const EphemLoc L = ephem_locate(md, t[i]);
  ephem_all(md, L, [&](int b, const double r[3]) {
    for (int ax = 0; ax < 3; ax++) rb[(size_t)(b * 3 + ax) * n + i] = r[ax];
  });
}

__global__ void k_eval_warm(Model md, long long n, const double *__restrict__ x0, const double *__restrict__ dt,
                            double *__restrict__ x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[6], y[6];
  for (int q = 0; q < 6; q++) a[q] = x0[q * n + i];
  const bool ok = kepler_dt(md.mu_c, a, dt[i], y);
  for (int q = 0; q < 6; q++) x[q * n + i] = ok ? y[q] : a[q];
}

__global__ void k_eval_dyn(Model md, long long n, const double *__restrict__ t, const double *__restrict__ y,
                           double *__restrict__ f) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double rb[kMaxBodies * 3];
  double ind[3] = {0.0, 0.0, 0.0};
  const EphemLoc L = ephem_locate(md, t[i]);
  for (int b = 0; b < md.B; b++) {
    ephem_body(md, L, b, rb + 3 * b);
    if (md.indirect) add_indirect(md, b, rb + 3 * b, ind);
  }
  const double r[3] = {y[i], y[n + i], y[2 * n + i]};
  double a[3];
  accel(md, rb, ind, 1, r, a);
  if (md.c_light > 0.0) {
    double vb[kMaxBodies * 3], X[7 * (kMaxBodies + 1)], e3[3];
    ephem_vel_all(md, L, [&](int b, const double v[3]) {
      for (int ax = 0; ax < 3; ax++) vb[3 * b + ax] = v[ax];
    });
    eih_bodies(md, rb, vb, X);
    const double v[3] = {y[3 * n + i], y[4 * n + i], y[5 * n + i]};
    eih_terms(md, rb, X, 1, r, v, e3);
    for (int q = 0; q < 3; q++) a[q] += e3[q];
  }
  for (int q = 0; q < 3; q++) {
    f[q * n + i] = y[(3 + q) * n + i];
    f[(3 + q) * n + i] = a[q];
  }
}

// EIH data of the bodies at the nodes of the new segments (grid-stride over
// list entries x nodes, entries fastest, as k_setup): EX[j][f][slot] with the
// layout of eih_bodies.
__global__ void k_setup_eih(Sweep s, Ctl c, Model md, const double *__restrict__ tau, double *__restrict__ EX) {
  const int cur = s.list_cur;
  const long long count = s.list_cnt[cur];
  const int *__restrict__ list = s.list[cur];
  const long long total = count * s.n;
  const int ld = s.ld, B = md.B, xs = eih_stride(B);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / count);
    const long long e = i - (long long)j * count;
    const int m = list[e];
    const double t = dadd(c.w1[m], dmul(c.w2[m], tau[j]));
    const EphemLoc L = ephem_locate(md, t);
    double rb[kMaxBodies * 3], vb[kMaxBodies * 3], X[7 * (kMaxBodies + 1)];
    ephem_all(md, L, [&](int b, const double r[3]) {
      for (int ax = 0; ax < 3; ax++) rb[3 * b + ax] = r[ax];
    });
    ephem_vel_all(md, L, [&](int b, const double v[3]) {
      for (int ax = 0; ax < 3; ax++) vb[3 * b + ax] = v[ax];
    });
    eih_bodies(md, rb, vb, X);
    for (int f = 0; f < xs; f++) EX[((size_t)j * xs + f) * ld + m] = X[f];
  }
}

constexpr int kThreads = 128;

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

Mix live_mix(const pc_plan *p) {
  const Workspace &w = p->ws;
  Mix mx{};
  mx.YK = w.YK;
  mx.X32 = w.X32;
  mx.xs = x32_stride(p->model.B);
  return mx;
}

// FP64 sweeps contract with the split-digit kernel when the plan asks for it
// and its operator digits exist (N <= 255).
bool use_split(const pc_plan *p) { return p->opt.contraction == PC_CONTRACT_SPLIT && split_supported(p); }

unsigned sm_ctas(const pc_plan *p, int per_sm) { return (unsigned)((p->num_sms > 0 ? p->num_sms : 152) * per_sm); }

size_t fp32_smem_bytes(const pc_plan *p) {
  const int threads = 32 * ((p->n + 31) / 32);
  const int xss = fp32_rec_stride(x32_stride(p->model.B));
  return sizeof(float) * ((size_t)p->n * (xss + 6) + 2 * (threads / 32));
}

// Launch shape of the tiled FP32 kernel: R rows per thread, RG row groups
// (threads per slot), T trajectory slots per CTA.  Node records either staged
// in shared memory (at most 256 threads) or read from global memory through
// L1 (4 rows per thread: up to 512 threads, 16 warps, in the shared memory
// the records would take); the operator in shared memory, or read through L1
// when it does not fit beside staged records.  The slot count asked for is
// met with staged records when they fit, else by reading them from global
// memory; failing both (N > 256) one trajectory per CTA.
struct Fp32tShape {
  int R, RG, T, threads;
  bool ksm, rsm, mma, ok;
  size_t smem;
};
constexpr size_t kMaxDynSmem = 220 * 1024;

Fp32tShape fp32t_shape(const pc_plan *p) {
  Fp32tShape sh{};
  const int N = p->N, n = p->n, B = p->model.B;
  sh.R = p->tune.fp32_rows == 4 ? 4 : 8;
  sh.RG = 4 * ((N + 4 * sh.R - 1) / (4 * sh.R));
  if (sh.R == 4 && sh.RG * 8 > kFp32tMaxThreadsG) {
    sh.R = 8;
    sh.RG = 4 * ((N + 31) / 32);
  }
  sh.ok = false;
  const int want = std::max(8, std::min(p->tune.fp32_slots / 8 * 8, kFp32tMaxSlots));
  if (p->opt.fp32_mma) {
    // the tensor-core contraction: 4 rows per thread, node records from
    // global memory, whatever fp32_rows says (the arithmetic is the option's,
    // the launch shape the tuning's); FP32 multiply-adds only when N is too
    // large for it
    const int RG4 = 4 * ((N + 15) / 16);
    int T = std::min(want, kFp32tMaxThreadsG / RG4 / 8 * 8);
    while (T >= 8 && fp32t_smem_bytes(N, n, p->rows32, T, RG4, true, false, true, B) > kMaxDynSmem) T -= 8;
    if (T >= 8) {
      sh.R = 4;
      sh.RG = RG4;
      sh.T = T;
      sh.ksm = sh.mma = true;
      sh.rsm = false;
      sh.ok = true;
      sh.threads = sh.RG * sh.T;
      sh.smem = fp32t_smem_bytes(N, n, p->rows32, T, RG4, true, false, true, B);
      return sh;
    }
  }
  if (p->tune.fp32_rows == 0 || sh.RG * 8 > kFp32tMaxThreads) return sh;
  // largest T <= want (multiple of 8) for a variant, 0 if none
  auto slots = [&](bool ksm, bool rsm) {
    int T = std::min(want, fp32t_max_threads(sh.R, rsm) / sh.RG / 8 * 8);
    while (T >= 8 && fp32t_smem_bytes(N, n, p->rows32, T, sh.RG, ksm, rsm, false, B) > kMaxDynSmem) T -= 8;
    return T >= 8 ? T : 0;
  };
  const int t_staged = slots(true, true);
  const int t_global = slots(true, false);
  if (t_staged > 0 && t_staged >= t_global) {
    sh.T = t_staged;
    sh.ksm = sh.rsm = true;
  } else if (t_global > 0) {
    sh.T = t_global;
    sh.ksm = true;
    sh.rsm = false;
  } else if (slots(false, true) > 0) {
    sh.T = slots(false, true);
    sh.ksm = false;
    sh.rsm = true;
  } else {
    return sh;
  }
  sh.ok = true;
  sh.threads = sh.RG * sh.T;
  sh.smem = fp32t_smem_bytes(N, n, p->rows32, sh.T, sh.RG, sh.ksm, sh.rsm, false, B);
  return sh;
}

template <int MODE, int R, bool KSM, bool RSM, bool MMA = false>
void launch_fp32t_one(const pc_plan *p, const Fp32tShape &sh, const Sweep &s, const double *Yc, double *Yn,
                      const double *E, const float *R32, const Mix &mx, cudaStream_t st) {
  const Ctl &c = p->ws.ctl[p->ws.live];
  k_fp32t<MODE, R, KSM, RSM, MMA><<<sm_ctas(p, p->tune.fp32_ctas_per_sm), sh.threads, sh.smem, st>>>(
      s, c, p->model, p->d_K32R, p->rows32, p->d_mu32, Yc, Yn, E, R32, mx, sh.T);
}

template <int MODE, int R, bool KSM, bool RSM, bool MMA = false>
cudaError_t fp32t_attr(size_t smem) {
  return cudaFuncSetAttribute(k_fp32t<MODE, R, KSM, RSM, MMA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

template <int MODE, int R>
void launch_fp32t_r(const pc_plan *p, const Fp32tShape &sh, const Sweep &s, const double *Yc, double *Yn,
                    const double *E, const float *R32, const Mix &mx, cudaStream_t st) {
  if (!sh.rsm) launch_fp32t_one<MODE, R, true, false>(p, sh, s, Yc, Yn, E, R32, mx, st);
  else if (sh.ksm) launch_fp32t_one<MODE, R, true, true>(p, sh, s, Yc, Yn, E, R32, mx, st);
  else launch_fp32t_one<MODE, R, false, true>(p, sh, s, Yc, Yn, E, R32, mx, st);
}

template <int R>
cudaError_t fp32t_attr_r(const Fp32tShape &sh) {
  cudaError_t e;
  if (sh.mma) {
    e = fp32t_attr<FP32_KEPLER, 4, true, false, true>(sh.smem);
    if (e == cudaSuccess) e = fp32t_attr<FP32_CORR, 4, true, false, true>(sh.smem);
  } else if (!sh.rsm) {
    e = fp32t_attr<FP32_KEPLER, R, true, false>(sh.smem);
    if (e == cudaSuccess) e = fp32t_attr<FP32_CORR, R, true, false>(sh.smem);
  } else if (sh.ksm) {
    e = fp32t_attr<FP32_KEPLER, R, true, true>(sh.smem);
    if (e == cudaSuccess) e = fp32t_attr<FP32_CORR, R, true, true>(sh.smem);
  } else {
    e = fp32t_attr<FP32_KEPLER, R, false, true>(sh.smem);
    if (e == cudaSuccess) e = fp32t_attr<FP32_CORR, R, false, true>(sh.smem);
  }
  return e;
}

// FP32 sweeps of one mode over this round's list: with fp32_mma the tiled
// kernel with its contraction on the tensor cores; otherwise the tiled kernel
// (T trajectories per CTA) or, with fp32_rows = 0, one trajectory per CTA of
// 32 ceil((N+1)/32) threads, which give bitwise the same results.
template <int MODE>
void launch_fp32(const pc_plan *p, const Sweep &s, const double *Yc, double *Yn, const double *E, const float *R32,
                 const Mix &mx, cudaStream_t st) {
  const Fp32tShape sh = fp32t_shape(p);
  if (!sh.ok) {
    const int threads = 32 * ((p->n + 31) / 32);
    const size_t smem = fp32_smem_bytes(p);
    const Ctl &c = p->ws.ctl[p->ws.live];
    k_fp32<MODE><<<sm_ctas(p, p->tune.fp32_ctas_per_sm), threads, smem, st>>>(s, c, p->model, p->d_K32T, p->d_mu32,
                                                                             Yc, Yn, E, R32, mx);
    return;
  }
  if (sh.mma) launch_fp32t_one<MODE, 4, true, false, true>(p, sh, s, Yc, Yn, E, R32, mx, st);
  else if (sh.R == 4) launch_fp32t_r<MODE, 4>(p, sh, s, Yc, Yn, E, R32, mx, st);
  else launch_fp32t_r<MODE, 8>(p, sh, s, Yc, Yn, E, R32, mx, st);
}

}  // namespace

// ---- launchers ----------------------------------------------------------------
cudaError_t prepare_launches(const pc_plan *p) {
  if (use_split(p)) {
    const cudaError_t e = prepare_split(p);
    if (e != cudaSuccess) return e;
  }
  if (!p->npl) return cudaSuccess;
  const int bytes = (int)fp32_smem_bytes(p);
  cudaError_t e = cudaFuncSetAttribute(k_fp32<FP32_KEPLER>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fp32<FP32_CORR>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  const Fp32tShape sh = fp32t_shape(p);
  if (e != cudaSuccess || !sh.ok) return e;
  return sh.R == 4 ? fp32t_attr_r<4>(sh) : fp32t_attr_r<8>(sh);
}

cudaError_t launch_init(const pc_plan *p, const Sweep &s, const double *x0, cudaStream_t st) {
  const Workspace &w = p->ws;
  cudaError_t e = cudaMemsetAsync(w.ints, 0, 16 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.cnt64, 0, 2 * sizeof(unsigned long long), st);
  if (e == cudaSuccess && s.eh_size > 0) e = cudaMemsetAsync(s.eh_tab[0], 0xFF, 2 * sizeof(int) * s.eh_size, st);
  if (e != cudaSuccess) return e;
  p->acc_launches += 1;
  k_init<<<blocks_for(s.n_ic, kThreads), kThreads, 0, st>>>(s, w.ctl[w.live], p->model, x0, w.ints);
  return cudaGetLastError();
}

cudaError_t launch_round(const pc_plan *p, const Sweep &s, int cur, cudaStream_t st, cudaEvent_t *ev) {
  const Workspace &w = p->ws;
  if (s.A <= 0) return cudaSuccess;
  const Ctl &c = w.ctl[w.live];
  double *Yc = w.Y[cur], *Yn = w.Y[cur ^ 1];
  double *E = w.E[w.live], *Ai = w.Aind[w.live];
  const Mix mx = live_mix(p);
  // Mixed precision without per-kernel events: the new-segment branch (set-up,
  // FP32 phase; its trajectories join the FP64 list next round) and the FP64
  // branch (force, contraction over this round's FP64 list) touch disjoint
  // trajectories, so they run side by side and join before the control kernel.
  const bool branches = s.mixed && !ev && p->side_stream;
  cudaStream_t sb = branches ? p->side_stream : st;
  cudaError_t e = cudaSuccess;
  if (branches) {
    e = cudaEventRecord(p->branch_ev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sb, p->branch_ev[0], 0);
    if (e != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[0], st);
  if (s.eh_size > 0) {
    k_grid_keys<<<sm_ctas(p, p->tune.setup_ctas_per_sm), kThreads, 0, sb>>>(s, c);
    k_grid_ephem<<<sm_ctas(p, p->tune.setup_ctas_per_sm), kThreads, 0, sb>>>(s, c, p->model, p->d_tau);
    p->acc_launches += 2;
  }
  if (s.warm && s.kep_stride > 0) {
    k_kepler17<<<sm_ctas(p, p->tune.setup_ctas_per_sm), kThreads, 0, sb>>>(s, c, p->d_tau);
    p->acc_launches += 1;
  }
  k_setup<<<sm_ctas(p, p->tune.setup_ctas_per_sm), kThreads, 0, sb>>>(s, c, p->model, p->d_tau, Yc, E, Ai, mx);
  if (p->model.c_light > 0.0) {
    k_setup_eih<<<sm_ctas(p, p->tune.setup_ctas_per_sm), kThreads, 0, sb>>>(s, c, p->model, p->d_tau, w.EX[w.live]);
    p->acc_launches += 1;
  }
  if (ev) cudaEventRecord(ev[1], st);
  float *R32 = s.refine ? w.R32[w.live] : nullptr;
  if (s.mixed) launch_fp32<FP32_KEPLER>(p, s, Yc, Yn, E, R32, mx, sb);
  if (s.refine) {
    k_corr_setup<<<sm_ctas(p, p->tune.setup_ctas_per_sm), kThreads, 0, sb>>>(s, p->model, p->d_mu32, Yc, E, R32, mx);
    p->acc_launches += 1;
    launch_fp32<FP32_CORR>(p, s, Yc, Yn, E, R32, mx, sb);
  }
  if (branches) {
    e = cudaEventRecord(p->branch_ev[1], sb);
    if (e != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[2], st);
  k_force<<<dim3(blocks_for(s.A, 32), (s.n + kForceNodes - 1) / kForceNodes), dim3(32, kForceNodes), 0, st>>>(
      s, c, p->model, Yc, E, Ai, w.G, p->d_tau, w.tails, w.EX[w.live]);
  if (ev) cudaEventRecord(ev[3], st);
  if (use_split(p)) {
    // exact digit products on the bf16 tensor cores
    e = launch_contract_split(p, s, c, w.G, Yc, Yn, R32, s.order == 2 ? SPLIT_SECOND_ORDER : SPLIT_FIRST_ORDER, st);
    if (e != cudaSuccess) return e;
  } else {
    // persistent FP64 contraction: contract_ctas_per_sm CTAs of kSplit warps per SM
    const long long tiles = (long long)(s.rows_pad / 16) * ((s.A + 7) / 8);
    const long long blocks =
        std::max<long long>(1, std::min<long long>(sm_ctas(p, p->tune.contract_ctas_per_sm), tiles));
    k_contract<<<(unsigned)blocks, 32 * kSplit, 0, st>>>(s, c, p->d_K, w.G, Yc, Yn, R32);
  }
  if (branches) {
    e = cudaStreamWaitEvent(st, p->branch_ev[1], 0);
    if (e != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[4], st);
  // one warp per CTA: the control work (resolution tests) spreads over all SMs
  k_control<<<blocks_for(s.A, 32), 32, 0, st>>>(s, c, w.tails, Yn, w.ints);
  if (ev) cudaEventRecord(ev[5], st);
  p->acc_launches += s.mixed ? (s.refine ? 6 : 5) : 4;
  return cudaGetLastError();
}

cudaError_t launch_repack(const pc_plan *p, const Sweep &s, int cur, cudaStream_t st) {
  const Workspace &w = p->ws;
  if (s.A <= 0) return cudaSuccess;
  const int a = w.live, b = w.live ^ 1;
  cudaError_t e = cudaMemsetAsync(w.ints + 4, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.list_cnt + s.list_cur, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.l64_cnt + s.list_cur, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.lc_cnt + s.list_cur, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const unsigned nb = blocks_for(s.A, kThreads);
  k_repack_pos<<<nb, kThreads, 0, st>>>(s.A, w.ctl[a].phase, w.pos, w.ints + 4);
  const long long n = p->n, B = p->model.B;
  const dim3 g(nb, 64);
  k_repack_rows<double><<<g, kThreads, 0, st>>>(s.A, s.ld, n * 6, w.pos, w.Y[cur], w.Y[cur ^ 1]);
  if (B > 0) k_repack_rows<double><<<g, kThreads, 0, st>>>(s.A, s.ld, n * B * 3, w.pos, w.E[a], w.E[b]);
  k_repack_rows<double><<<g, kThreads, 0, st>>>(s.A, s.ld, n * 3, w.pos, w.Aind[a], w.Aind[b]);
  if (w.EX[a])
    k_repack_rows<double><<<g, kThreads, 0, st>>>(s.A, s.ld, n * eih_stride((int)B), w.pos, w.EX[a], w.EX[b]);
  if (s.refine) k_repack_rows<float><<<g, kThreads, 0, st>>>(s.A, s.ld, n * 6, w.pos, w.R32[a], w.R32[b]);
  k_repack_ctl<<<nb, kThreads, 0, st>>>(s, w.ctl[a], w.ctl[b], w.pos);
  p->acc_launches += 4 + (B > 0) + (s.refine ? 1 : 0) + (w.EX[a] ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_abort(const pc_plan *p, const Sweep &s, cudaStream_t st) {
  if (s.A <= 0) return cudaSuccess;
  k_abort<<<blocks_for(s.A, kThreads), kThreads, 0, st>>>(s, p->ws.ctl[p->ws.live]);
  p->acc_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_eval_ephemeris(const pc_plan *p, long long n, const double *t, double *rb, cudaStream_t st) {
  k_eval_ephem<<<blocks_for(n, kThreads), kThreads, 0, st>>>(p->model, n, t, rb);
  return cudaGetLastError();
}

cudaError_t launch_eval_warm(const pc_plan *p, long long n, const double *x0, const double *dt, double *x,
                             cudaStream_t st) {
  k_eval_warm<<<blocks_for(n, kThreads), kThreads, 0, st>>>(p->model, n, x0, dt, x);
  return cudaGetLastError();
}

// Dynamics at n points with the same device functions as the sweep
// (ephemeris, indirect term, acceleration); omega2 = 1.
cudaError_t launch_eval_dynamics(const pc_plan *p, long long n, const double *t, const double *y, double *f,
                                 cudaStream_t st) {
  k_eval_dyn<<<blocks_for(n, kThreads), kThreads, 0, st>>>(p->model, n, t, y, f);
  return cudaGetLastError();
}

cudaError_t launch_apply_operator(const pc_plan *p, long long n_ic, int ld, const double *x0, const double *G,
                                  double *Y, cudaStream_t st) {
  const Workspace &w = p->ws;
  Sweep s{};
  s.N = p->N;
  s.n = p->n;
  s.kpad = p->kpad;
  s.rows_pad = p->rows_pad;
  s.n_ic = n_ic;
  s.ld = ld;
  Ctl c = w.ctl[w.live];
  c.x = const_cast<double *>(x0);
  if (use_split(p)) {
    const cudaError_t e = prepare_split(p);
    if (e != cudaSuccess) return e;
    return launch_contract_split(p, s, c, const_cast<double *>(G), nullptr, Y, nullptr, SPLIT_DIAG, st);
  }
  const long long tiles = (long long)(s.rows_pad / 16) * ((n_ic + 7) / 8);
  k_contract_diag<<<(unsigned)std::min<long long>(tiles, sm_ctas(p, 8)), 32 * kSplit, 0, st>>>(s, c, p->d_K, G, Y);
  return cudaGetLastError();
}

}  // namespace pcx
