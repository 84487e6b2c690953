// Reverse mode through the converged Picard-Chebyshev segments, and the
// b-plane of a flyby with its Jacobian.
//
// Forward, a segment's converged nodes satisfy (Eq. 2 in matrix form)
//   Y = 1 x0^T + omega2 K G(Y),   G_j = f(y_j, t_j),
// and the segment hands y_N to the next one.  Differentiating the fixed point,
// a cotangent ybar on y_N reaches x0 as
//   x0bar = sum_j lambda_j,   lambda = Ybar + J^T (omega2 K^T lambda),
// with Ybar = ybar at node N only and J = blockdiag(df/dy at the nodes):
// (J^T m)_r = A_j m_v, (J^T m)_v = m_r, A_j the gravity gradient at node j.
// The adjoint equation is linear with the same contraction factor as the
// forward sweep, so it is swept the same way until lambda stops changing.
// The nodes come from the tape the forward pass recorded: every accepted
// segment's converged states, so no iterate is stored and nothing is
// recomputed.  Segments are taken in reverse, one launch per step back; all
// trajectories with at least that many segments go in the same launch,
// ordered by segment count so the tiles stay full.
//
// k_adjoint keeps a tile of T trajectories in shared memory for all sweeps of
// its segment (lambda, K^T lambda and the gravity gradients): a sweep reads
// only the operator, from L2, and runs its (N+1) x N x 6T product on the FP64
// tensor cores.
#include <algorithm>
#include <vector>

#include "pc_device.cuh"

namespace pcx {
namespace {

struct Adj {
  int N, n, mpad, kpad;      // degree, nodes, padded rows (nodes) and k extent (nodes 1..N)
  long long n_ic;
  const int *perm;           // trajectories by segment count, descending
  const int *nseg;           // [n_ic]
  int max_seg;
  const double *tape;        // [n_ic][max_seg][2 + 6n]
  double *xb;                // [6][n_ic] cotangent: of the segment end in, of its start out
  int relative, max_iters, stall_sweeps;
  double tol, stall_factor, div_limit;
  int *status, *iters;       // [n_ic] or nullptr (OR-ed / summed over segments)
  int *fail;                 // trajectories whose adjoint sweep failed
};

// Adds the gradient of -mu d/|d|^3 with respect to d,
// -mu (I/|d|^3 - 3 d d^T/|d|^5), as (xx, xy, xz, yy, yz, zz).
__device__ __forceinline__ void add_point_gradient(double mu, double dx, double dy, double dz, double A[6]) {
  const double d2 = dx * dx + dy * dy + dz * dz;
  const double ir = rsqrt(d2);
  const double i3 = mu * ir * ir * ir;
  const double i5 = 3.0 * i3 / d2;
  A[0] += dx * dx * i5 - i3;
  A[1] += dx * dy * i5;
  A[2] += dx * dz * i5;
  A[3] += dy * dy * i5 - i3;
  A[4] += dy * dz * i5;
  A[5] += dz * dz * i5 - i3;
}

template <int T>
struct AdjTile {
  static constexpr int NT = (6 * T + 7) / 8;  // 8-column MMA tiles over the 6T columns
  static constexpr int STR = 8 * NT + 4;      // shared row stride (doubles): conflict-free B fragments
};

template <int T>
__host__ __device__ constexpr int adj_max_threads() {
  return T >= 8 ? 512 : (T >= 4 ? 768 : 1024);
}

template <int T>
__global__ void __launch_bounds__(adj_max_threads<T>()) k_adjoint(const Adj a, const Model md,
                                                                   const double *__restrict__ KTp,
                                                                   const double *__restrict__ tau, int r, int count) {
  constexpr int NT = AdjTile<T>::NT, STR = AdjTile<T>::STR;
  extern __shared__ double sm[];
  double *hB = sm;                                  // [kpad][STR]  lambda_j, row j-1 for nodes 1..N
  double *mu = hB + (size_t)a.kpad * STR;           // [mpad][STR]  (K^T lambda)_j
  double *As = mu + (size_t)a.mpad * STR;           // [T][n][6]    gravity gradients
  __shared__ double h0[T][6], seed[T][6], w2s[T], ebest[T];
  __shared__ unsigned long long red[T][4];
  __shared__ int icx[T], done[T], flags[T], sweeps[T], nstall[T], any_left;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int n = a.n, N = a.N;
  const int tiles = (count + T - 1) / T;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    // ---- tile set-up: trajectories, segment lengths, incoming cotangents
    if (tid < T) {
      const int pidx = tile * T + tid;
      const int ic = pidx < count ? a.perm[pidx] : -1;
      icx[tid] = ic;
      done[tid] = ic < 0;
      flags[tid] = 0;
      sweeps[tid] = 0;
      nstall[tid] = 0;
      ebest[tid] = __longlong_as_double(0x7FF0000000000000LL);
      double w2 = 0.0;
      if (ic >= 0) {
        const double *rec = a.tape + ((size_t)ic * a.max_seg + (a.nseg[ic] - 1 - r)) * (size_t)tape_rec(n);
        w2 = dmul(0.5, dsub(rec[1], rec[0]));
      }
      w2s[tid] = w2;
      for (int q = 0; q < 6; q++) {
        seed[tid][q] = ic >= 0 ? a.xb[(size_t)q * a.n_ic + ic] : 0.0;
        h0[tid][q] = 0.0;
      }
      for (int q = 0; q < 4; q++) red[tid][q] = 0ULL;
    }
    for (int i = tid; i < a.kpad * STR; i += nth) hB[i] = 0.0;
    __syncthreads();
    // ---- gravity gradient at the converged nodes (same node times and body
    // positions as the forward sweep); lambda starts as the seed at node N
    for (int it = tid; it < T * n; it += nth) {
      const int i = it / n, j = it - i * n;
      double A[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      const int ic = icx[i];
      if (ic >= 0) {
        const double *rec = a.tape + ((size_t)ic * a.max_seg + (a.nseg[ic] - 1 - r)) * (size_t)tape_rec(n);
        const double w1 = dmul(0.5, dadd(rec[1], rec[0])), w2 = dmul(0.5, dsub(rec[1], rec[0]));
        const double tj = dadd(w1, dmul(w2, tau[j]));
        const double *y = rec + 2 + 6 * j;
        add_point_gradient(md.mu_c, y[0], y[1], y[2], A);
        if (md.B > 0) {
          const EphemLoc L = ephem_locate(md, tj);
          for (int b = 0; b < md.B; b++) {
            double rb[3];
            ephem_body(md, L, b, rb);
            add_point_gradient(md.mu[b], y[0] - rb[0], y[1] - rb[1], y[2] - rb[2], A);
          }
        }
        if (j == N)
          for (int q = 0; q < 6; q++) hB[(size_t)(N - 1) * STR + 6 * i + q] = seed[i][q];
      }
      double *Ad = As + (size_t)it * 6;
      for (int q = 0; q < 6; q++) Ad[q] = A[q];
    }
    __syncthreads();
    // ---- adjoint sweeps
    for (;;) {
      // mu = K^T lambda on the FP64 tensor cores; warp w takes row tiles w, w + nwarps, ...
      for (int mt = warp; mt < a.mpad / 16; mt += nwarps) {
        double acc[NT][4];
#pragma unroll
        for (int q = 0; q < NT; q++) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.0;
        const double *ka = KTp + (size_t)(mt * 16 + g) * a.kpad + t;
        const double *kb = ka + (size_t)8 * a.kpad;
        for (int ks = 0; ks < a.kpad; ks += 4) {
          const double a0 = __ldg(ka + ks), a1 = __ldg(kb + ks);
          const double *hb = hB + (size_t)(ks + t) * STR + g;
#pragma unroll
          for (int q = 0; q < NT; q++) dmma16x8x4(acc[q], a0, a1, hb[q * 8]);
        }
        double *m0 = mu + (size_t)(mt * 16 + g) * STR + 2 * t;
#pragma unroll
        for (int q = 0; q < NT; q++) {
          m0[q * 8] = acc[q][0];
          m0[q * 8 + 1] = acc[q][1];
          m0[(size_t)8 * STR + q * 8] = acc[q][2];
          m0[(size_t)8 * STR + q * 8 + 1] = acc[q][3];
        }
      }
      __syncthreads();
      // lambda_j = Ybar_j + J_j^T (omega2 mu_j); change and size per trajectory
      for (int it = tid; it < T * n; it += nth) {
        const int i = it / n, j = it - i * n;
        if (done[i]) continue;
        const double w2 = w2s[i];
        const double *mj = mu + (size_t)j * STR + 6 * i;
        const double *A = As + (size_t)it * 6;
        const double m3 = w2 * mj[3], m4 = w2 * mj[4], m5 = w2 * mj[5];
        double h[6];
        h[0] = A[0] * m3 + A[1] * m4 + A[2] * m5;
        h[1] = A[1] * m3 + A[3] * m4 + A[4] * m5;
        h[2] = A[2] * m3 + A[4] * m4 + A[5] * m5;
        h[3] = w2 * mj[0];
        h[4] = w2 * mj[1];
        h[5] = w2 * mj[2];
        if (j == N)
          for (int q = 0; q < 6; q++) h[q] += seed[i][q];
        double *old = (j == 0) ? h0[i] : hB + (size_t)(j - 1) * STR + 6 * i;
        double dr = 0.0, nr = 0.0, dv = 0.0, nv = 0.0;
        for (int q = 0; q < 3; q++) {
          const double d = h[q] - old[q], e = h[3 + q] - old[3 + q];
          dr += d * d;
          nr += h[q] * h[q];
          dv += e * e;
          nv += h[3 + q] * h[3 + q];
        }
        for (int q = 0; q < 6; q++) old[q] = h[q];
        atomicMax(&red[i][0], err_bits(sqrt(dr)));
        atomicMax(&red[i][1], err_bits(sqrt(nr)));
        atomicMax(&red[i][2], err_bits(sqrt(dv)));
        atomicMax(&red[i][3], err_bits(sqrt(nv)));
      }
      __syncthreads();
      // per-trajectory stopping: the forward rules (blow-up, tolerance, stall, cap)
      // on max_j |d lambda_r| / max_j |lambda_r| and the same for the v part
      if (tid < T) {
        const int i = tid;
        if (!done[i]) {
          sweeps[i] += 1;
          double er = __longlong_as_double((long long)red[i][0]), ev = __longlong_as_double((long long)red[i][2]);
          const double nr = __longlong_as_double((long long)red[i][1]), nv = __longlong_as_double((long long)red[i][3]);
          if (a.relative) {
            if (nr > 0.0) er = er / nr;
            if (nv > 0.0) ev = ev / nv;
          }
          const double e = nanmax(er, ev);
          if (!(e <= a.div_limit)) {
            flags[i] |= PC_IC_NONFINITE;
            done[i] = 1;
          } else if (e < a.tol) {
            done[i] = 1;
          } else {
            if (e < ebest[i]) {
              ebest[i] = e;
              nstall[i] = 0;
            } else {
              nstall[i] += 1;
            }
            if (nstall[i] >= a.stall_sweeps && ebest[i] < a.stall_factor * a.tol) {
              flags[i] |= PC_IC_STALLED;
              done[i] = 1;
            } else if (sweeps[i] >= a.max_iters) {
              flags[i] |= PC_IC_NOT_CONVERGED;
              done[i] = 1;
            }
          }
        }
        for (int q = 0; q < 4; q++) red[i][q] = 0ULL;
      }
      __syncthreads();
      if (tid == 0) {
        int left = 0;
        for (int i = 0; i < T; i++) left |= !done[i];
        any_left = left;
      }
      __syncthreads();
      if (!any_left) break;
    }
    // ---- cotangent of the segment's start: x0bar = sum_j lambda_j (fixed order)
    if (tid < 6 * T) {
      const int i = tid / 6, q = tid - 6 * (tid / 6);
      if (icx[i] >= 0) {
        double s = h0[i][q];
        for (int k = 0; k < N; k++) s += hB[(size_t)k * STR + 6 * i + q];
        a.xb[(size_t)q * a.n_ic + icx[i]] = s;
      }
    }
    if (tid < T && icx[tid] >= 0) {
      if (a.status) a.status[icx[tid]] |= flags[tid];
      if (a.iters) a.iters[icx[tid]] += sweeps[tid];
      if (flags[tid] & (PC_IC_NONFINITE | PC_IC_NOT_CONVERGED)) atomicAdd(a.fail, 1);
    }
    __syncthreads();  // shared memory is reused by the next tile
  }
}

// ---------------------------------------------------------------------------
// b-plane.  The flyby body's velocity is the time derivative of its table
// series: with f = sum_k c_k T_k(sigma), f' = c'_0/2 + sum_{k>=1} c'_k T_k where
// c'_{deg} = c'_{deg+1} = 0 and c'_{k-1} = c'_{k+1} + 2k c_k, evaluated by
// Clenshaw and scaled by dsigma/dt = 2/L.
// ---------------------------------------------------------------------------
__device__ void ephem_body_velocity(const Model &md, EphemLoc L, int b, double v[3]) {
  const int deg = md.deg;
  for (int ax = 0; ax < 3; ax++) {
    const double *cf = md.coef + (((size_t)b * md.n_gr + L.g) * 3 + ax) * (deg + 1);
    // Clenshaw over the derivative coefficients, generated from the top down
    double dk1 = 0.0, dk2 = 0.0;  // c'_k, c'_{k+1} at the top of iteration k
    double b1 = 0.0, b2 = 0.0;
    double d0 = 0.0;
    for (int k = deg; k >= 1; k--) {
      const double dkm1 = dk2 + 2.0 * k * cf[k];  // c'_{k-1}
      // Clenshaw step for index k-1 (c'_{k-1}), skipping the constant term
      if (k - 1 >= 1) {
        const double bn = dkm1 + 2.0 * L.sig * b1 - b2;
        b2 = b1;
        b1 = bn;
      } else {
        d0 = dkm1;
      }
      dk2 = dk1;
      dk1 = dkm1;
    }
    v[ax] = (0.5 * d0 + L.sig * b1 - b2) * (2.0 / md.granule);
  }
}

// Forward-mode dual number with six tangent directions (the 6 state components).
struct D6 {
  double v, d[6];
};
__device__ __forceinline__ D6 dconst(double x) {
  D6 r;
  r.v = x;
  for (int q = 0; q < 6; q++) r.d[q] = 0.0;
  return r;
}
__device__ __forceinline__ D6 operator+(const D6 &a, const D6 &b) {
  D6 r;
  r.v = a.v + b.v;
  for (int q = 0; q < 6; q++) r.d[q] = a.d[q] + b.d[q];
  return r;
}
__device__ __forceinline__ D6 operator-(const D6 &a, const D6 &b) {
  D6 r;
  r.v = a.v - b.v;
  for (int q = 0; q < 6; q++) r.d[q] = a.d[q] - b.d[q];
  return r;
}
__device__ __forceinline__ D6 operator*(const D6 &a, const D6 &b) {
  D6 r;
  r.v = a.v * b.v;
  for (int q = 0; q < 6; q++) r.d[q] = a.d[q] * b.v + a.v * b.d[q];
  return r;
}
__device__ __forceinline__ D6 operator*(double s, const D6 &a) {
  D6 r;
  r.v = s * a.v;
  for (int q = 0; q < 6; q++) r.d[q] = s * a.d[q];
  return r;
}
__device__ __forceinline__ D6 operator/(const D6 &a, const D6 &b) {
  D6 r;
  r.v = a.v / b.v;
  for (int q = 0; q < 6; q++) r.d[q] = (a.d[q] - r.v * b.d[q]) / b.v;
  return r;
}
__device__ __forceinline__ D6 dsqrt(const D6 &a) {
  D6 r;
  r.v = sqrt(a.v);
  for (int q = 0; q < 6; q++) r.d[q] = a.d[q] / (2.0 * r.v);
  return r;
}
__device__ __forceinline__ void dcross(const D6 a[3], const D6 b[3], D6 c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ D6 ddot(const D6 a[3], const D6 b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// b-plane of the body-relative state rel (see pc.h for the construction).
// Returns false when the relative orbit is not a hyperbola.
__device__ bool bplane_dual(double mu, const double rel[6], D6 out[2]) {
  D6 r[3], v[3];
  for (int q = 0; q < 3; q++) {
    r[q] = dconst(rel[q]);
    r[q].d[q] = 1.0;
    v[q] = dconst(rel[3 + q]);
    v[q].d[3 + q] = 1.0;
  }
  const D6 rn = dsqrt(ddot(r, r)), v2 = ddot(v, v), rv = ddot(r, v);
  const D6 vinf2 = v2 - dconst(2.0 * mu) / rn;
  if (!(vinf2.v > 0.0)) return false;
  const D6 vinf = dsqrt(vinf2);
  D6 h[3], ev[3], P[3], hh[3], Q[3], S[3], T[3], R[3], Bv[3];
  dcross(r, v, h);
  const D6 hn = dsqrt(ddot(h, h));
  const D6 c1 = v2 - dconst(mu) / rn;
  for (int q = 0; q < 3; q++) ev[q] = (1.0 / mu) * (c1 * r[q] - rv * v[q]);
  const D6 e = dsqrt(ddot(ev, ev));
  if (!(e.v > 1.0)) return false;
  for (int q = 0; q < 3; q++) {
    P[q] = ev[q] / e;
    hh[q] = h[q] / hn;
  }
  dcross(hh, P, Q);
  const D6 se = dsqrt(e * e - dconst(1.0)) / e;
  for (int q = 0; q < 3; q++) S[q] = P[q] / e + se * Q[q];
  // T = S x z / |S x z| with z = (0, 0, 1): S x z = (S_y, -S_x, 0)
  const D6 tn = dsqrt(S[0] * S[0] + S[1] * S[1]);
  T[0] = S[1] / tn;
  T[1] = dconst(0.0) - S[0] / tn;
  T[2] = dconst(0.0);
  dcross(S, T, R);
  dcross(S, h, Bv);
  for (int q = 0; q < 3; q++) Bv[q] = Bv[q] / vinf;
  out[0] = ddot(Bv, T);
  out[1] = ddot(Bv, R);
  return true;
}

__global__ void k_bplane(Model md, int body, double mu_body, long long n, const double *__restrict__ t,
                         const double *__restrict__ x, double *__restrict__ out, double *__restrict__ jac,
                         const double *__restrict__ obar, double *__restrict__ xbar, int *bad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const EphemLoc L = ephem_locate(md, t[i]);
  double rb[3], vb[3], rel[6];
  ephem_body(md, L, body, rb);
  ephem_body_velocity(md, L, body, vb);
  for (int q = 0; q < 3; q++) {
    rel[q] = x[(size_t)q * n + i] - rb[q];
    rel[3 + q] = x[(size_t)(3 + q) * n + i] - vb[q];
  }
  D6 o[2];
  const bool ok = bplane_dual(mu_body, rel, o);
  if (!ok) {
    atomicAdd(bad, 1);
    for (int k = 0; k < 2; k++) o[k] = dconst(__longlong_as_double(0x7FF8000000000000LL));
  }
  if (out)
    for (int k = 0; k < 2; k++) out[(size_t)k * n + i] = o[k].v;
  if (jac)
    for (int k = 0; k < 2; k++)
      for (int q = 0; q < 6; q++) jac[(size_t)(6 * k + q) * n + i] = o[k].d[q];
  if (obar && xbar) {
    const double b0 = obar[i], b1 = obar[(size_t)n + i];
    for (int q = 0; q < 6; q++) xbar[(size_t)q * n + i] = b0 * o[0].d[q] + b1 * o[1].d[q];
  }
}

pc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PC_OK;
  return e == cudaErrorMemoryAllocation ? PC_ENOMEM : PC_ECUDA;
}

template <class U>
cudaError_t dalloc(U **p, size_t count) {
  return cudaMalloc((void **)p, sizeof(U) * (count > 0 ? count : 1));
}

pc_status ensure_adjoint_workspace(pc_plan *p, long long n_ic) {
  AdjWorkspace &w = p->adj;
  if (w.cap >= n_ic && w.perm) return PC_OK;
  const long long cap = std::max<long long>(n_ic, 64);
  cudaFree(w.perm);
  cudaFree(w.xb);
  cudaFree(w.xf);
  cudaFree(w.nseg);
  w.perm = nullptr;
  w.xb = w.xf = nullptr;
  w.nseg = nullptr;
  w.cap = 0;
  cudaError_t e = dalloc(&w.perm, cap);
  if (e == cudaSuccess) e = dalloc(&w.xb, 6 * cap);
  if (e == cudaSuccess) e = dalloc(&w.xf, 6 * cap);
  if (e == cudaSuccess) e = dalloc(&w.nseg, cap);
  if (e == cudaSuccess && !w.fail) e = dalloc(&w.fail, 1);
  if (e == cudaSuccess && !w.h_fail) e = cudaMallocHost((void **)&w.h_fail, sizeof(int));
  if (e != cudaSuccess) return cuda_status(e);
  w.cap = cap;
  return PC_OK;
}

template <int T>
size_t adjoint_smem(const pc_plan *p) {
  return sizeof(double) * ((size_t)(p->adj_kpad + p->adj_mpad) * AdjTile<T>::STR + (size_t)T * p->n * 6);
}

template <int T>
cudaError_t launch_adjoint_t(const pc_plan *p, const Adj &a, int r, int count, cudaStream_t st) {
  const size_t smem = adjoint_smem<T>(p);
  cudaError_t e = cudaFuncSetAttribute(k_adjoint<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int warps = std::min(p->adj_mpad / 16, adj_max_threads<T>() / 32);
  const int tiles = (count + T - 1) / T;
  const int grid = std::max(1, std::min(tiles, p->num_sms > 0 ? p->num_sms : 152));
  k_adjoint<T><<<grid, 32 * warps, smem, st>>>(a, p->model, p->d_KTp, p->d_tau, r, count);
  p->acc_launches += 1;
  return cudaGetLastError();
}

// Trajectories per tile: the largest of 8, 4, 2 whose shared memory fits.
int adjoint_tile(const pc_plan *p) {
  constexpr size_t kLimit = 200 * 1024;
  if (adjoint_smem<8>(p) <= kLimit) return 8;
  if (adjoint_smem<4>(p) <= kLimit) return 4;
  if (adjoint_smem<2>(p) <= 226 * 1024) return 2;
  return 0;
}

}  // namespace

void free_adjoint_workspace(pc_plan *p) {
  AdjWorkspace &w = p->adj;
  cudaFree(w.perm);
  cudaFree(w.xb);
  cudaFree(w.xf);
  cudaFree(w.nseg);
  cudaFree(w.fail);
  cudaFree(w.tape);
  if (w.h_fail) cudaFreeHost(w.h_fail);
  w = AdjWorkspace();
}

}  // namespace pcx

using namespace pcx;

extern "C" pc_status pc_propagate_tape(pc_plan *p, long long n_ic, const double *x0, const double *t0,
                                       const double *tf, const int *segments, double tol, double *xf, int *status,
                                       int *nseg, int max_seg, double *tape, void *stream) {
  // reverse mode differentiates the Newtonian force only
  if (!p || n_ic < 0 || p->model.c_light > 0.0) return PC_EINVAL;
  if (n_ic == 0) return PC_OK;
  if (!x0 || !t0 || !tf || !xf || !nseg || !tape || max_seg < 1 || n_ic > (1LL << 30)) return PC_EINVAL;
  return propagate_with_tape(p, n_ic, x0, 0.0, 0.0, t0, tf, segments, tol, xf, status, nullptr, nseg, max_seg, tape,
                             (cudaStream_t)stream);
}

extern "C" pc_status pc_adjoint_tape(pc_plan *p, long long n_ic, const int *nseg, int max_seg, const double *tape,
                                     const double *xf_bar, double tol, double *x0_bar, int *status, int *iters,
                                     void *stream) {
  // reverse mode differentiates the Newtonian force only
  if (!p || n_ic < 0 || p->model.c_light > 0.0) return PC_EINVAL;
  if (n_ic == 0) return PC_OK;
  if (!nseg || !tape || !xf_bar || !x0_bar || max_seg < 1 || n_ic > (1LL << 30)) return PC_EINVAL;
  const int T = adjoint_tile(p);
  if (T == 0) return PC_EINVAL;
  pc_status ps = ensure_adjoint_workspace(p, n_ic);
  if (ps != PC_OK) return ps;
  AdjWorkspace &w = p->adj;
  cudaStream_t st = (cudaStream_t)stream;
  // segment counts to the host: they set the number of reverse steps and the order
  std::vector<int> h_nseg((size_t)n_ic);
  cudaError_t e = cudaMemcpyAsync(h_nseg.data(), nseg, sizeof(int) * n_ic, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  int top = 0;
  for (long long i = 0; i < n_ic; i++) {
    if (h_nseg[i] < 0 || h_nseg[i] > max_seg) return PC_EINVAL;
    top = std::max(top, h_nseg[i]);
  }
  // counting sort by segment count, descending; count[r] = #(nseg > r)
  std::vector<long long> bucket((size_t)top + 2, 0);
  for (long long i = 0; i < n_ic; i++) bucket[(size_t)h_nseg[i]]++;
  std::vector<int> count((size_t)top + 1, 0);
  {
    long long above = 0;
    for (int r = top; r >= 0; r--) {
      count[(size_t)r] = (int)above;  // trajectories with nseg > r
      above += bucket[(size_t)r];
    }
  }
  std::vector<int> perm((size_t)n_ic);
  {
    std::vector<long long> start((size_t)top + 1, 0);
    long long pos = 0;
    for (int v = top; v >= 0; v--) {
      start[(size_t)v] = pos;
      pos += bucket[(size_t)v];
    }
    for (long long i = 0; i < n_ic; i++) perm[(size_t)start[(size_t)h_nseg[i]]++] = (int)i;
  }
  e = cudaMemcpyAsync(w.perm, perm.data(), sizeof(int) * n_ic, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.xb, xf_bar, sizeof(double) * 6 * n_ic, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.fail, 0, sizeof(int), st);
  if (e == cudaSuccess && status) e = cudaMemsetAsync(status, 0, sizeof(int) * n_ic, st);
  if (e == cudaSuccess && iters) e = cudaMemsetAsync(iters, 0, sizeof(int) * n_ic, st);
  const pc_options &o = p->opt;
  Adj a{};
  a.N = p->N;
  a.n = p->n;
  a.mpad = p->adj_mpad;
  a.kpad = p->adj_kpad;
  a.n_ic = n_ic;
  a.perm = w.perm;
  a.nseg = nseg;
  a.max_seg = max_seg;
  a.tape = tape;
  a.xb = w.xb;
  a.relative = o.relative;
  a.max_iters = 2 * o.max_iters;  // lambda starts cold (no Keplerian guess): twice the forward cap
  a.stall_sweeps = o.stall_sweeps;
  a.tol = tol > 0.0 ? tol : o.tol;
  a.stall_factor = o.stall_factor;
  a.div_limit = o.div_limit;
  a.status = status;
  a.iters = iters;
  a.fail = w.fail;
  for (int r = 0; r < top && e == cudaSuccess; r++) {
    const int c = count[(size_t)r];
    if (c <= 0) break;
    if (T == 8) e = launch_adjoint_t<8>(p, a, r, c, st);
    else if (T == 4) e = launch_adjoint_t<4>(p, a, r, c, st);
    else e = launch_adjoint_t<2>(p, a, r, c, st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(x0_bar, w.xb, sizeof(double) * 6 * n_ic, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.h_fail, w.fail, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  return *w.h_fail > 0 ? PC_ENOTCONV : PC_OK;
}

extern "C" pc_status pc_propagate_adjoint(pc_plan *p, long long n_ic, const double *x0, double t0, double tf,
                                          double tol, const double *xf_bar, double *x0_bar, void *stream) {
  // reverse mode differentiates the Newtonian force only
  if (!p || n_ic < 0 || p->model.c_light > 0.0) return PC_EINVAL;
  if (n_ic == 0) return PC_OK;
  if (!x0 || !xf_bar || !x0_bar || n_ic > (1LL << 30)) return PC_EINVAL;
  pc_status ps = ensure_adjoint_workspace(p, n_ic);
  if (ps != PC_OK) return ps;
  AdjWorkspace &w = p->adj;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t rec = (size_t)tape_rec(p->n);
  int cap = w.tape_hint > 0 ? w.tape_hint : std::max(16, 2 * p->segments + 8);
  pc_status fwd = PC_OK;
  for (int attempt = 0; attempt < 2; attempt++) {
    const size_t bytes = sizeof(double) * rec * (size_t)cap * (size_t)n_ic;
    if (bytes > w.tape_bytes) {
      cudaFree(w.tape);
      w.tape = nullptr;
      w.tape_bytes = 0;
      cudaError_t e = cudaMalloc((void **)&w.tape, bytes);
      if (e != cudaSuccess) return cuda_status(e);
      w.tape_bytes = bytes;
    }
    fwd = propagate_with_tape(p, n_ic, x0, t0, tf, nullptr, nullptr, nullptr, tol, w.xf, nullptr, nullptr, w.nseg,
                              cap, w.tape, st);
    if (fwd != PC_OK && fwd != PC_ENOTCONV) return fwd;
    std::vector<int> h_nseg((size_t)n_ic);
    cudaError_t e = cudaMemcpyAsync(h_nseg.data(), w.nseg, sizeof(int) * n_ic, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    const int top = *std::max_element(h_nseg.begin(), h_nseg.end());
    if (top <= cap) break;
    cap = top;  // the tape was too short: run again with room for every segment
    if (attempt == 1) return PC_ECUDA;
  }
  w.tape_hint = cap;
  ps = pc_adjoint_tape(p, n_ic, w.nseg, cap, w.tape, xf_bar, tol, x0_bar, nullptr, nullptr, stream);
  if (ps != PC_OK) return ps;
  return fwd;
}

extern "C" pc_status pc_bplane(pc_plan *p, int body, double mu_body, long long n, const double *t, const double *x,
                               double *out, double *jac, const double *out_bar, double *x_bar, void *stream) {
  if (!p || n < 0) return PC_EINVAL;
  if (n == 0) return PC_OK;
  if (body < 0 || body >= p->model.B || !(mu_body > 0.0) || !t || !x || (!out && !jac && !x_bar) ||
      ((out_bar == nullptr) != (x_bar == nullptr)))
    return PC_EINVAL;
  pc_status ps = ensure_adjoint_workspace(p, 1);
  if (ps != PC_OK) return ps;
  AdjWorkspace &w = p->adj;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(w.fail, 0, sizeof(int), st);
  const int threads = 128;
  const long long blocks = (n + threads - 1) / threads;
  if (e == cudaSuccess) {
    k_bplane<<<(unsigned)blocks, threads, 0, st>>>(p->model, body, mu_body, n, t, x, out, jac, out_bar, x_bar, w.fail);
    p->acc_launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.h_fail, w.fail, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  return *w.h_fail > 0 ? PC_ENONFINITE : PC_OK;
}
