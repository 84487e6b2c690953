// Plan creation: operator construction (host, extended precision), model
// upload, workspace management, status strings.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "pc_internal.h"

using namespace pcx;

namespace {

// T_m(tau_j) on the CGL nodes tau_j = -cos(j pi/N): with theta_j = pi - j pi/N,
// T_m(tau_j) = cos(m theta_j) = (-1)^m cos(m j pi / N).  The angle m*j is
// reduced modulo 2N in integers before the cosine, so every entry is the
// correctly reduced extended-precision value.
long double cheb_at_node(int m, int j, int N) {
  const long double pi = 3.141592653589793238462643383279502884L;
  long long q = ((long long)m * (long long)j) % (2LL * N);
  long double c = cosl(pi * (long double)q / (long double)N);
  return (m & 1) ? -c : c;
}

// The PC operator, built column by column.  Column k is the map from a unit
// force at node k to the state increments: the Lagrange basis polynomial l_k
// on the CGL nodes has Chebyshev coefficients
//   a_m = (2/N) * T_m(tau_k) / (c_k c_m),   c_0 = c_N = 2, otherwise 1,
// its integral from -1 has coefficients b_1 = a_0 - a_2/2,
// b_m = (a_{m-1} - a_{m+1})/(2m) (m >= 2, a_{N+1} = a_{N+2} = 0) and b_0 fixed
// by the integral vanishing at tau = -1, and K[j][k] = sum_m b_m T_m(tau_j).
// This is the paper's chain of matrix products (A, S, C) collapsed into one
// (N+1) x (N+1) matrix acting on omega2-scaled forces.
void build_operator(int N, int truncated, double *K /* (N+1)^2 */) {
  const int n = N + 1;
  std::vector<long double> a(N + 3), b(N + 2);
  std::vector<long double> T((size_t)(N + 2) * n);
  for (int m = 0; m <= N + 1; m++)
    for (int j = 0; j < n; j++) T[(size_t)m * n + j] = cheb_at_node(m, j, N);
  for (int k = 0; k < n; k++) {
    const long double ck = (k == 0 || k == N) ? 2.0L : 1.0L;
    for (int m = 0; m <= N + 2; m++) a[m] = 0.0L;
    for (int m = 0; m <= N; m++) {
      const long double cm = (m == 0 || m == N) ? 2.0L : 1.0L;
      a[m] = 2.0L / (long double)N * T[(size_t)m * n + k] / (ck * cm);
    }
    b[1] = a[0] - 0.5L * a[2];
    for (int m = 2; m <= N + 1; m++) b[m] = (a[m - 1] - a[m + 1]) / (2.0L * (long double)m);
    if (truncated) b[N + 1] = 0.0L;
    long double s = 0.0L;
    for (int m = 1; m <= N + 1; m++) s += (m & 1) ? -b[m] : b[m];  // value at tau = -1
    b[0] = -s;
    for (int j = 0; j < n; j++) {
      long double y = 0.0L;
      for (int m = 0; m <= N + 1; m++) y += b[m] * T[(size_t)m * n + j];
      K[(size_t)j * n + k] = (double)y;
    }
  }
  for (int k = 0; k < n; k++) K[k] = 0.0;  // node 0 is the initial condition itself
}

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
  return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

}  // namespace

extern "C" pc_status pc_options_default(pc_options *o) {
  if (!o) return PC_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-13;
  o->relative = 1;
  o->max_iters = 60;
  o->max_depth = 8;
  o->warm_start = 1;
  o->seg_mode = 0;
  o->truncated = 0;
  o->stall_sweeps = 5;
  o->stall_factor = 1e3;
  o->div_limit = 1e3;
  o->trunc_tol = 1e-13;
  o->precision = PC_PREC_FP64;
  o->switch_tol = 0.0;
  o->max_rounds = 0;
  o->refine32 = 1;
  o->contraction = PC_CONTRACT_SPLIT;
  o->order = 1;
  o->fp32_mma = 0;
  return PC_OK;
}

static pc_status check_options(const pc_options &o) {
  if (!(o.tol >= 0.0) || o.max_iters < 1 || o.max_depth < 0 || o.max_depth > 30 || o.stall_sweeps < 1 ||
      !(o.stall_factor >= 0.0) || !(o.div_limit > 0.0) || (o.seg_mode != 0 && o.seg_mode != 1) ||
      (o.precision != PC_PREC_FP64 && o.precision != PC_PREC_MIXED) || o.max_rounds < 0 ||
      !(o.switch_tol >= 0.0) || (o.refine32 != 0 && o.refine32 != 1) ||
      (o.contraction != PC_CONTRACT_DMMA && o.contraction != PC_CONTRACT_SPLIT) || (o.order != 1 && o.order != 2) ||
      (o.order == 2 && o.contraction != PC_CONTRACT_SPLIT) || (o.fp32_mma != 0 && o.fp32_mma != 1))
    return PC_EINVAL;
  return PC_OK;
}

extern "C" pc_status pc_plan_create(int N, int segments, const pc_force_model *force, const pc_ephemeris *ephem,
                                    const pc_options *opt, pc_plan **out) {
  if (!out) return PC_EINVAL;
  *out = nullptr;
  if (N < 2 || N > kMaxN || segments < 1 || !force) return PC_EINVAL;
  const int B = force->n_bodies;
  if (B < 0 || B > kMaxBodies || !(force->mu_central > 0.0) || (B > 0 && !force->mu) || !(force->c_light >= 0.0))
    return PC_EINVAL;
  if (B > 0) {
    if (!ephem || ephem->n_bodies != B || !(ephem->granule_s > 0.0) || ephem->degree < 0 || ephem->degree > 63 ||
        ephem->n_granules < 1 || !ephem->coef)
      return PC_EINVAL;
  }
  pc_options o;
  pc_options_default(&o);
  if (opt) o = *opt;
  if (check_options(o) != PC_OK) return PC_EINVAL;
  if (o.precision == PC_PREC_MIXED && N + 1 > 32 * kMaxNpl) return PC_EINVAL;
  if (o.order == 2 && N > 255) return PC_EINVAL;  // the second-order sweep runs on the split contraction

  pc_plan *p = new (std::nothrow) pc_plan();
  if (!p) return PC_ENOMEM;
  p->N = N;
  p->n = N + 1;
  p->kpad = (p->n + 3) / 4 * 4;
  p->rows_pad = (N + 15) / 16 * 16;
  p->segments = segments;
  p->opt = o;
  cudaGetDevice(&p->device);

  const int n = p->n;
  p->h_K = (double *)std::malloc(sizeof(double) * n * n);
  p->h_tau = (double *)std::malloc(sizeof(double) * n);
  if (!p->h_K || !p->h_tau) { pc_plan_destroy(p); return PC_ENOMEM; }
  build_operator(N, o.truncated, p->h_K);
  // tau_j = -cos(j pi/N) written as sin(pi (2j - N)/(2N)): exactly antisymmetric, 0 in the middle
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int j = 0; j < n; j++) p->h_tau[j] = (double)sinl(pi * (long double)(2 * j - N) / (long double)(2 * N));

  // Device operator: rows = nodes 1..N, zero-padded to rows_pad x kpad.
  std::vector<double> Kd((size_t)p->rows_pad * p->kpad, 0.0);
  for (int r = 0; r < N; r++)
    for (int k = 0; k < n; k++) Kd[(size_t)r * p->kpad + k] = p->h_K[(size_t)(r + 1) * n + k];
  cudaError_t e = dalloc(&p->d_K, Kd.size());
  if (e == cudaSuccess) e = cudaMemcpy(p->d_K, Kd.data(), sizeof(double) * Kd.size(), cudaMemcpyHostToDevice);
  // FP32 operator for the mixed-precision kernels: K32T[k][j] = K[j][k]
  // for output nodes j = 0..N laid out as 32 lanes x npl, zero elsewhere.
  if (N + 1 <= 32 * kMaxNpl) {
    p->npl = (N + 32) / 32;
    const int np = 32 * p->npl;
    std::vector<float> Kt((size_t)n * np, 0.0f);
    for (int k = 0; k < n; k++)
      for (int j = 0; j <= N; j++) Kt[(size_t)k * np + j] = (float)p->h_K[(size_t)j * n + k];
    if (e == cudaSuccess) e = dalloc(&p->d_K32T, Kt.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_K32T, Kt.data(), sizeof(float) * Kt.size(), cudaMemcpyHostToDevice);
    // the same operator for the tiled FP32 kernels: K32R[k][r] = K[r+1][k] for
    // output rows r = 0..N-1 (nodes 1..N; row 0 of K is zero), rows32 floats
    // per k, zero-padded
    p->rows32 = (N + 31) / 32 * 32;
    std::vector<float> Kr((size_t)n * p->rows32, 0.0f);
    for (int k = 0; k < n; k++)
      for (int r = 0; r < N; r++) Kr[(size_t)k * p->rows32 + r] = (float)p->h_K[(size_t)(r + 1) * n + k];
    if (e == cudaSuccess) e = dalloc(&p->d_K32R, Kr.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_K32R, Kr.data(), sizeof(float) * Kr.size(), cudaMemcpyHostToDevice);
  }
  // Warm-start interpolation: Lagrange weights of the 17 nodes tau_{i N/16}
  // (Chebyshev-Lobatto nodes of degree 16) at every node, in long double,
  // stored as FP32 pairs hi + lo (L[j][i] then the remainders at offset
  // n x 17); rows of the 17 nodes themselves are exact unit vectors.
  if (N % 16 == 0 && N >= 32) {
    p->kep_stride = N / 16;
    std::vector<float> L(2 * (size_t)n * kKepNodes, 0.0f);
    for (int j = 0; j < n; j++) {
      if (j % p->kep_stride == 0) {
        L[(size_t)j * kKepNodes + j / p->kep_stride] = 1.0f;
        continue;
      }
      const long double x = (long double)p->h_tau[j];
      for (int i = 0; i < kKepNodes; i++) {
        const long double xi = (long double)p->h_tau[i * p->kep_stride];
        long double l = 1.0L;
        for (int k = 0; k < kKepNodes; k++)
          if (k != i) l *= (x - (long double)p->h_tau[k * p->kep_stride]) / (xi - (long double)p->h_tau[k * p->kep_stride]);
        const float hi = (float)l;
        L[(size_t)j * kKepNodes + i] = hi;
        L[((size_t)n + j) * kKepNodes + i] = (float)(l - (long double)hi);
      }
    }
    if (e == cudaSuccess) e = dalloc(&p->d_Lint, L.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_Lint, L.data(), sizeof(float) * L.size(), cudaMemcpyHostToDevice);
  }
  // Split-digit contraction: each operator row (node r+1) cut into 7 digits
  // against its largest exponent, packed as bf16 mma B fragments (B[k][n] =
  // K[node n][k]; lane (g, t) holds k = 2t, 2t+1 and 2t+8, 2t+9 of node g)
  if (N <= 255) {
    p->split_nt = (N + 7) / 8;
    p->split_ks = (n + 15) / 16;
    std::vector<int> kexp(N, 0), dig((size_t)N * kSplitDigits * p->split_ks * 16, 0);
    for (int r = 0; r < N; r++) {
      const double *row = p->h_K + (size_t)(r + 1) * n;
      int bmax = 0;
      for (int k = 0; k < n; k++) {
        unsigned long long b;
        std::memcpy(&b, row + k, sizeof(b));
        bmax = std::max(bmax, (int)((b >> 52) & 0x7ff));
      }
      kexp[r] = bmax;
      for (int k = 0; k < n; k++) {
        int d[kSplitDigits];
        split_digits7(row[k], bmax, d);
        for (int a = 0; a < kSplitDigits; a++) dig[((size_t)r * kSplitDigits + a) * p->split_ks * 16 + k] = d[a];
      }
    }
    auto bf16_bits = [](int v) -> unsigned {
      const float f = (float)v;  // |v| <= 128: exact, and so is its bf16 (the top 16 bits)
      unsigned u;
      std::memcpy(&u, &f, sizeof(u));
      return u >> 16;
    };
    auto digit = [&](int r, int a, int k) -> int {
      return (r < N && k < n) ? dig[((size_t)r * kSplitDigits + a) * p->split_ks * 16 + k] : 0;
    };
    std::vector<unsigned> frag((size_t)p->split_nt * p->split_ks * kSplitDigits * 32 * 2);
    for (int nt = 0; nt < p->split_nt; nt++)
      for (int ks = 0; ks < p->split_ks; ks++)
        for (int a = 0; a < kSplitDigits; a++)
          for (int lane = 0; lane < 32; lane++) {
            const int g = lane >> 2, t = lane & 3, r = nt * 8 + g, k0 = ks * 16 + 2 * t;
            unsigned *f = frag.data() + ((((size_t)nt * p->split_ks + ks) * kSplitDigits + a) * 32 + lane) * 2;
            f[0] = bf16_bits(digit(r, a, k0)) | (bf16_bits(digit(r, a, k0 + 1)) << 16);
            f[1] = bf16_bits(digit(r, a, k0 + 8)) | (bf16_bits(digit(r, a, k0 + 9)) << 16);
          }
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_Kdig, sizeof(unsigned) * frag.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_Kdig, frag.data(), sizeof(unsigned) * frag.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_Kexp, sizeof(int) * N);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_Kexp, kexp.data(), sizeof(int) * N, cudaMemcpyHostToDevice);
  }
  // Adjoint operator: K transposed without its zero row 0, KTp[j][k'] = K[k'+1][j].
  p->adj_mpad = (n + 15) / 16 * 16;
  p->adj_kpad = (N + 3) / 4 * 4;
  {
    std::vector<double> KT((size_t)p->adj_mpad * p->adj_kpad, 0.0);
    for (int j = 0; j < n; j++)
      for (int k = 0; k < N; k++) KT[(size_t)j * p->adj_kpad + k] = p->h_K[(size_t)(k + 1) * n + j];
    if (e == cudaSuccess) e = dalloc(&p->d_KTp, KT.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_KTp, KT.data(), sizeof(double) * KT.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e == cudaSuccess) e = dalloc(&p->d_tau, n);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_tau, p->h_tau, sizeof(double) * n, cudaMemcpyHostToDevice);
  Model &m = p->model;
  m.B = B;
  m.mu_c = force->mu_central;
  m.indirect = force->indirect ? 1 : 0;
  m.c_light = force->c_light;
  if (B > 0) {
    m.t_begin = ephem->t_begin;
    m.granule = ephem->granule_s;
    m.deg = ephem->degree;
    m.n_gr = ephem->n_granules;
    size_t nc = (size_t)B * ephem->n_granules * 3 * (ephem->degree + 1);
    if (e == cudaSuccess) e = dalloc(&p->d_mu, B);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_mu, force->mu, sizeof(double) * B, cudaMemcpyHostToDevice);
    std::vector<float> mu32(B);
    for (int b = 0; b < B; b++) mu32[b] = (float)force->mu[b];
    if (e == cudaSuccess) e = dalloc(&p->d_mu32, B);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_mu32, mu32.data(), sizeof(float) * B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dalloc(&p->d_coef, nc);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_coef, ephem->coef, sizeof(double) * nc, cudaMemcpyHostToDevice);
  } else {
    m.t_begin = 0.0;
    m.granule = 1.0;
    m.deg = 0;
    m.n_gr = 1;
  }
  m.mu = p->d_mu;
  m.coef = p->d_coef;
  if (e != cudaSuccess) {
    pc_plan_destroy(p);
    return e == cudaErrorMemoryAllocation ? PC_ENOMEM : PC_ECUDA;
  }
  *out = p;
  return PC_OK;
}

namespace {
// Carves one control block (kCtlDoubles doubles, one u64, one i64 and kCtlInts
// 4-byte fields per slot) into the Ctl arrays.
void carve_ctl(void *block, long long ld, Ctl &t) {
  char *c = (char *)block;
  auto take = [&](size_t each) { char *r = c; c += each * ld; return r; };
  t.x = (double *)take(8 * 6);
  t.t0 = (double *)take(8);
  t.tf = (double *)take(8);
  t.total = (double *)take(8);
  t.sgn = (double *)take(8);
  t.hbase = (double *)take(8);
  t.ta = (double *)take(8);
  t.tb = (double *)take(8);
  t.w1 = (double *)take(8);
  t.w2 = (double *)take(8);
  t.e_best = (double *)take(8);
  t.err = (unsigned long long *)take(8);
  t.p = (long long *)take(8);
  t.depth = (int *)take(4);
  t.phase = (int *)take(4);
  t.status = (int *)take(4);
  t.sweeps = (int *)take(4);
  t.seg_sweeps = (int *)take(4);
  t.nstall = (int *)take(4);
  t.nseg = (int *)take(4);
  t.need_setup = (int *)take(4);
  t.last = (int *)take(4);
  t.ic = (int *)take(4);
  t.err32 = (unsigned *)take(4);
  t.ncorr = (int *)take(4);
  t.kc = (double *)take(8 * kKeplerConsts);
}
}  // namespace

pc_status pcx::ensure_workspace(pc_plan *p, long long n_ic, int mixed) {
  Workspace &w = p->ws;
  if (n_ic <= w.cap && w.Y[0] && (!mixed || w.mixed)) return PC_OK;
  free_workspace(p);
  const long long ld = (n_ic + 7) / 8 * 8;
  if (ld > (1LL << 30)) return PC_EINVAL;
  const size_t n = p->n, kpad = p->kpad, B = p->model.B;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; b++) e = dalloc(&w.Y[b], n * 6 * ld);
  if (e == cudaSuccess) e = dalloc(&w.G, kpad * 6 * ld);
  if (e == cudaSuccess) e = cudaMemset(w.G, 0, sizeof(double) * kpad * 6 * ld);
  if (e == cudaSuccess) e = dalloc(&w.tails, (n + 7) / 8 * 14 * ld);
  const size_t ctl_bytes = (size_t)ld * (kCtlDoubles * 8 + 8 + 8 + kCtlInts * 4) + 256;
  for (int b = 0; b < 2 && e == cudaSuccess; b++) {
    if (B > 0) e = dalloc(&w.E[b], n * B * 3 * ld);
    if (e == cudaSuccess) e = dalloc(&w.Aind[b], n * 3 * ld);
    if (e == cudaSuccess) e = cudaMemset(w.Aind[b], 0, sizeof(double) * n * 3 * ld);
    if (e == cudaSuccess && p->model.c_light > 0.0) e = dalloc(&w.EX[b], n * (size_t)eih_stride((int)B) * ld);
    if (e == cudaSuccess) e = cudaMalloc(&w.ctl_block[b], ctl_bytes);
    if (e == cudaSuccess) e = cudaMemset(w.ctl_block[b], 0, ctl_bytes);
  }
  if (mixed && e == cudaSuccess) {
    e = dalloc(&w.YK, n * 6 * ld);
    if (e == cudaSuccess) e = dalloc(&w.X32, n * (size_t)x32_stride((int)B) * ld);
    for (int b = 0; b < 2 && e == cudaSuccess; b++) e = dalloc(&w.R32[b], n * 6 * ld);
  }
  if (p->kep_stride > 0 && e == cudaSuccess) e = dalloc(&w.YK17, 2 * (size_t)kKepNodes * 6 * ld);
  if (B > 0 && e == cudaSuccess) {
    // ephemeris cache: a table of at least twice the list capacity, and room
    // for up to 32768 distinct node-time grids per round
    long long sz = 1024;
    while (sz < 2 * ld) sz *= 2;
    w.eh_size = (int)sz;
    w.eh_cap = (int)std::min<long long>(ld, 32768);
    e = dalloc(&w.eh_tab, 4 * (size_t)sz);
    if (e == cudaSuccess) e = dalloc(&w.eh_ent, (size_t)ld);
    if (e == cudaSuccess) e = dalloc(&w.eh_own, (size_t)w.eh_cap);
    if (e == cudaSuccess) e = dalloc(&w.EC, n * (3 * B + 3) * (size_t)w.eh_cap);
  }
  if (e == cudaSuccess) e = dalloc(&w.lists, 6 * ld);
  if (e == cudaSuccess) e = dalloc(&w.pos, ld);
  if (e == cudaSuccess) e = dalloc(&w.cnt64, 2);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&w.h_cnt64, sizeof(unsigned long long) * 2);
  if (e == cudaSuccess) e = dalloc(&w.ints, 16);
  if (e == cudaSuccess) e = cudaMemset(w.ints, 0, sizeof(int) * 16);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&w.h_ints, sizeof(int) * 24);
  for (int i = 0; i < 2 && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&w.ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_workspace(p);
    return e == cudaErrorMemoryAllocation ? PC_ENOMEM : PC_ECUDA;
  }
  for (int b = 0; b < 2; b++) carve_ctl(w.ctl_block[b], ld, w.ctl[b]);
  w.cap = ld;
  w.ld = (int)ld;
  w.live = 0;
  w.mixed = mixed;
  return PC_OK;
}

void pcx::free_workspace(pc_plan *p) {
  Workspace &w = p->ws;
  for (int b = 0; b < 2; b++) {
    cudaFree(w.Y[b]);
    cudaFree(w.E[b]);
    cudaFree(w.Aind[b]);
    cudaFree(w.EX[b]);
    cudaFree(w.ctl_block[b]);
  }
  cudaFree(w.YK);
  cudaFree(w.YK17);
  cudaFree(w.eh_tab);
  cudaFree(w.eh_ent);
  cudaFree(w.eh_own);
  cudaFree(w.EC);
  cudaFree(w.X32);
  for (int b = 0; b < 2; b++) cudaFree(w.R32[b]);
  cudaFree(w.G);
  cudaFree(w.tails);
  cudaFree(w.lists);
  cudaFree(w.pos);
  cudaFree(w.ints);
  cudaFree(w.cnt64);
  if (w.h_ints) cudaFreeHost(w.h_ints);
  if (w.h_cnt64) cudaFreeHost(w.h_cnt64);
  for (int i = 0; i < 2; i++)
    if (w.ev[i]) cudaEventDestroy(w.ev[i]);
  if (w.graph) cudaGraphExecDestroy(w.graph);
  w = Workspace();
}

extern "C" void pc_plan_destroy(pc_plan *p) {
  if (!p) return;
  free_workspace(p);
  free_adjoint_workspace(p);
  for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
  if (p->own_stream) cudaStreamDestroy(p->own_stream);
  if (p->fork_ev) cudaEventDestroy(p->fork_ev);
  if (p->side_stream) cudaStreamDestroy(p->side_stream);
  for (int k = 0; k < 2; k++)
    if (p->branch_ev[k]) cudaEventDestroy(p->branch_ev[k]);
  cudaFree(p->d_K);
  cudaFree(p->d_KTp);
  cudaFree(p->d_K32T);
  cudaFree(p->d_K32R);
  cudaFree(p->d_Kdig);
  cudaFree(p->d_Lint);
  cudaFree(p->d_Kexp);
  cudaFree(p->d_tau);
  cudaFree(p->d_mu);
  cudaFree(p->d_mu32);
  cudaFree(p->d_coef);
  std::free(p->h_K);
  std::free(p->h_tau);
  delete p;
}

extern "C" pc_status pc_plan_operator(const pc_plan *p, double *K, double *tau) {
  if (!p) return PC_EINVAL;
  if (K) std::memcpy(K, p->h_K, sizeof(double) * p->n * p->n);
  if (tau) std::memcpy(tau, p->h_tau, sizeof(double) * p->n);
  return PC_OK;
}

extern "C" const char *pc_status_string(pc_status s) {
  switch (s) {
    case PC_OK: return "success";
    case PC_EINVAL: return "invalid argument";
    case PC_ENOMEM: return "out of memory";
    case PC_ECUDA: return "CUDA runtime error";
    case PC_ENOTCONV: return "some trajectories stopped before the end of the arc";
    case PC_ENONFINITE: return "non-finite value";
  }
  return "unknown status";
}
