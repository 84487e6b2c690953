// FP64 operator contraction by exact digit products on the bf16 tensor cores
// (PC_CONTRACT_SPLIT): Y' = 1 x0^T + K G over the round's FP64 list, the
// same product as k_contract (Section "Matrix form for vectorized and
// parallel computation", the operators collapsed into one (N+1)x(N+1) K),
// fused with the per-trajectory change and the residual.
//
// GB300's FP64 pipe (DFMA and the .f64 mma shapes alike) runs at about
// 1 TFLOP/s, its bf16 tensor cores two orders of magnitude faster.  Every
// operator row and every force column is cut into 7 signed 8-bit digits
// against its own largest exponent (split_digits7): K~ = sum_a d_a 2^-8a,
// G~ = sum_b e_b 2^-8b.  For each anti-diagonal d = a + b <= 8 (28 digit
// pairs) the tensor cores sum d_a e_b over the nodes in FP32 -- exactly,
// since every term and partial sum is an integer below 2^24 -- and the seven
// sums are combined in 64-bit integers, converted once to FP64 and scaled by
// the two exponents.  The pairs with a + b > 8 are below 2^-64 of the scale
// and dropped; the result's error is below that of an FP64 dot product.
//
// One CTA (4 warps) takes a column tile of 8 trajectories x 6 components (16 x
// 3 in a pass of the second-order sweep) from a counter: it writes the tile's
// digits to shared memory as 7 x 48 rows of bf16 (row q*8 + tt: component q
// of trajectory tt), then each warp runs
// node tiles of 8 output nodes: C[(q, tt)][node] = sum_k G~[k][(q, tt)]
// K~[node][k] with the force digits as the A operand (ldmatrix from shared
// memory) and the operator digits as the B operand (fragments precomputed by
// the plan, 64-bit loads from L2).  A thread's accumulators then hold every
// component of its trajectories at two nodes, which is what the epilogue (new
// iterate, change, residual) needs.
#include <cuda_bf16.h>

#include <algorithm>

#include "pc_device.cuh"
#include "pc_internal.h"

namespace pcx {
namespace {

constexpr int kSplitThreads = 128;
constexpr int kSplitCtasPerSm = 2;

// Epilogues: EPI_FULL the first-order sweep (new iterate, change, residual),
// EPI_DIAG the kernel-level product, and the two passes of a second-order
// sweep: EPI_VEL (velocities V' = v0 + K A; also omega2 V' into the velocity
// rows of G for the next pass) and EPI_POS (positions R' = r0 + K (omega2 V'),
// then the change and residual of the whole state).
enum : int { EPI_FULL = 0, EPI_DIAG = 1, EPI_VEL = 2, EPI_POS = 3 };

// k extent of a digit row in shared memory: 16 per k-step plus 8 (304 bytes
// at 9 k-steps, so the 8 rows of an ldmatrix phase hit distinct banks)
__host__ __device__ inline int split_ksp(int n_ks) { return 16 * n_ks + 8; }
// digit rows per slice: 48 = 3 tiles of 16 rows, 8 trajectories x 6 components
// or 16 trajectories x 3 components
constexpr int kSplitRows = 48;
__host__ __device__ constexpr int split_traj(int nc) { return kSplitRows / nc; }
__host__ __device__ inline size_t split_smem_bytes(int n_ks) {
  return sizeof(__nv_bfloat16) * (size_t)kSplitDigits * kSplitRows * split_ksp(n_ks);
}

struct SplitOp {
  const uint2 *kfrag;  // [n_nt][n_ks][7][32] B fragments of the operator digits
  const int *kexp;     // [N] largest biased exponent of each operator row
  int n_nt, n_ks;
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p) {
  const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// 2^e (exact; ldexp outside the normal exponent range)
__device__ __forceinline__ double pow2i(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

// NC components (6: the first-order sweep; 3: one pass of the second-order
// sweep) starting at component Q0 of G, for TRAJ = 48 / NC trajectories per
// tile.  Digit row q*TRAJ + tt holds component Q0 + q of the tile's
// trajectory tt; a thread's accumulators hold all NC components of
// trajectories g + 8h (h < TRAJ / 8) at two nodes.
template <int NC, int Q0, int EPI>
__global__ void __launch_bounds__(kSplitThreads, kSplitCtasPerSm)
    k_contract_split(Sweep s, Ctl c, SplitOp op, double *__restrict__ G, const double *__restrict__ Yold,
                     double *__restrict__ Ynew, float *__restrict__ R32) {
  constexpr bool DIAG = EPI == EPI_DIAG;
  constexpr int TRAJ = split_traj(NC);             // trajectories per tile
  constexpr int TPT = TRAJ / 8;                    // of them per thread
  constexpr int kRows = kSplitRows, MT = 3, kRowsPad = kSplitRows;
  extern __shared__ __align__(16) unsigned char split_sm[];
  __nv_bfloat16 *Gd = reinterpret_cast<__nv_bfloat16 *>(split_sm);  // [7][48][ksp]
  __shared__ int colB[kRows];            // largest biased exponent of each column
  __shared__ int colm[TRAJ];             // the tile's trajectories (slots), -1 past the end
  __shared__ int bad[TRAJ];              // an inf or NaN in one of the trajectory's columns
  __shared__ unsigned long long emax_sh[TRAJ];
  __shared__ int tile_sh;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int N = s.N, n = s.n, ld = s.ld;
  const int ksp = split_ksp(op.n_ks), kext = 16 * op.n_ks;
  const int ncols = DIAG ? (int)s.n_ic : s.l64_cnt[s.list_cur];
  const int *map = DIAG ? nullptr : s.l64[s.list_cur];
  const int n_tiles = (ncols + TRAJ - 1) / TRAJ;
  if (tid < kRows) colB[tid] = 0;
  if (tid < TRAJ) {
    bad[tid] = 0;
    emax_sh[tid] = 0ULL;
  }
  for (int iter = 0;; iter++) {
    int tile;
    if (DIAG) {
      tile = blockIdx.x + iter * gridDim.x;
    } else {
      if (tid == 0) tile_sh = atomicAdd(EPI == EPI_POS ? s.tile_ctr2 : s.tile_ctr, 1);
      __syncthreads();
      tile = tile_sh;
    }
    if (tile >= n_tiles) break;
    const int e0 = tile * TRAJ;
    if (tid < TRAJ) colm[tid] = (e0 + tid < ncols) ? (DIAG ? e0 + tid : map[e0 + tid]) : -1;
    __syncthreads();
    // ---- column exponents (shared-memory max over the nodes)
    for (int i = tid; i < kRows * n; i += kSplitThreads) {
      const int col = i % kRows, k = i / kRows;
      const int m = colm[col % TRAJ];
      if (m >= 0) {
        const unsigned long long b =
            (unsigned long long)__double_as_longlong(G[((size_t)k * 6 + Q0 + col / TRAJ) * ld + m]);
        atomicMax(&colB[col], (int)((b >> 52) & 0x7ff));
      }
    }
    // node 0 of the new iterate is the segment's initial state
    if (tid < kRows) {
      const int q = Q0 + tid / TRAJ, m = colm[tid % TRAJ];
      if (m >= 0) Ynew[(size_t)q * ld + m] = c.x[(size_t)q * ld + m];
    }
    __syncthreads();
    // ---- digits, two nodes per thread and step (bf16 pairs along k)
    for (int i = tid; i < kRows * (kext / 2); i += kSplitThreads) {
      const int k = 2 * (i % (kext / 2)), col = i / (kext / 2);
      const int m = colm[col % TRAJ], q = Q0 + col / TRAJ, Bc = colB[col];
      if (Bc == 0x7ff && (i % (kext / 2)) == 0) bad[col % TRAJ] = 1;
      int d0[kSplitDigits], d1[kSplitDigits];
      split_digits7((m >= 0 && k < n) ? G[((size_t)k * 6 + q) * ld + m] : 0.0, Bc, d0);
      split_digits7((m >= 0 && k + 1 < n) ? G[((size_t)(k + 1) * 6 + q) * ld + m] : 0.0, Bc, d1);
#pragma unroll
      for (int a = 0; a < kSplitDigits; a++)
        *reinterpret_cast<__nv_bfloat162 *>(Gd + ((size_t)a * kRowsPad + col) * ksp + k) =
            __halves2bfloat162(__int2bfloat16_rn(d0[a]), __int2bfloat16_rn(d1[a]));
    }
    __syncthreads();
    // ---- node tiles: 28 digit-pair products per k-step on the tensor cores
    const int g = lane >> 2, t = lane & 3;
    const int arow = (lane & 7) + ((lane >> 3) & 1) * 8, acol = (lane >> 4) * 8;
    for (int nt = w; nt < op.n_nt; nt += kSplitThreads / 32) {
      float acc[MT][kSplitDigits][4];
#pragma unroll
      for (int mt = 0; mt < MT; mt++)
#pragma unroll
        for (int dd = 0; dd < kSplitDigits; dd++)
#pragma unroll
          for (int i = 0; i < 4; i++) acc[mt][dd][i] = 0.0f;
      const uint2 *kf = op.kfrag + (size_t)nt * op.n_ks * kSplitDigits * 32 + lane;
      for (int ks = 0; ks < op.n_ks; ks++) {
        uint2 bf[kSplitDigits];
#pragma unroll
        for (int b = 0; b < kSplitDigits; b++) bf[b] = __ldg(kf + ((size_t)ks * kSplitDigits + b) * 32);
#pragma unroll
        for (int a = 0; a < kSplitDigits; a++) {
          unsigned af[MT][4];
#pragma unroll
          for (int mt = 0; mt < MT; mt++)
            ldsm_x4(af[mt], Gd + ((size_t)a * kRowsPad + mt * 16 + arow) * ksp + ks * 16 + acol);
#pragma unroll
          for (int b = 0; b < kSplitDigits - a; b++)
#pragma unroll
            for (int mt = 0; mt < MT; mt++) mma_bf16_16816(acc[mt][a + b], af[mt], bf[b]);
        }
      }
      // ---- epilogue: trajectories g + 8h of the tile at nodes 1 + nt*8 + 2t + {0, 1}
#pragma unroll
      for (int h = 0; h < TPT; h++) {
        const int tt = g + 8 * h, m = colm[tt];
        double e2 = 0.0;
#pragma unroll
        for (int e = 0; e < 2; e++) {
          const int r = nt * 8 + 2 * t + e, j = r + 1;
          if (m < 0 || j > N) continue;
          const int kx = op.kexp[r];
          const size_t base = (size_t)j * 6 * ld + m;
          double yq[NC];
#pragma unroll
          for (int q = 0; q < NC; q++) {
            const int row = q * TRAJ + tt;  // digit row; g < 8, so its tile and half are compile-time
            const int mt = (q * TRAJ + 8 * h) >> 4, idx = (((q * TRAJ + 8 * h) >> 3) & 1) * 2 + e;
            long long S[kSplitDigits];
#pragma unroll
            for (int dd = 0; dd < kSplitDigits; dd++) S[dd] = (long long)__float2int_rn(acc[mt][dd][idx]);
            const long long vhi = S[0] * (1LL << 24) + S[1] * (1LL << 16) + S[2] * (1LL << 8) + S[3];
            const long long vlo = S[4] * (1LL << 16) + S[5] * (1LL << 8) + S[6];
            // x0 + v 2^e in one rounding (the power-of-two scaling is exact)
            yq[q] = fma(fma((double)vlo, 0x1p-24, (double)vhi), pow2i(kx + colB[row] - 2042 - 40),
                        c.x[(size_t)(Q0 + q) * ld + m]);
          }
          if (bad[tt])
#pragma unroll
            for (int q = 0; q < NC; q++) yq[q] = __longlong_as_double(0x7FF8000000000000LL);
#pragma unroll
          for (int q = 0; q < NC; q++) Ynew[base + (size_t)(Q0 + q) * ld] = yq[q];
          if (EPI == EPI_VEL) {
            // omega2 V' is what the position pass integrates
            const double w2 = c.w2[m];
#pragma unroll
            for (int q = 0; q < 3; q++) G[base + (size_t)q * ld] = w2 * yq[q];
          }
          if (EPI == EPI_FULL || EPI == EPI_POS) {
            double yn[6];
#pragma unroll
            for (int q = 0; q < 6; q++) yn[q] = (q < NC) ? yq[q] : Ynew[base + (size_t)q * ld];
            // the sweep's change, rounded to FP32: the residual an FP32
            // correction solve starts from next round, and (scaled by the
            // new iterate's |r| and |v|) the convergence measure, whose
            // decisions need a few digits, not FP64 -- GB300's FP64 pipe is
            // this epilogue's bound
            float df[6];
#pragma unroll
            for (int q = 0; q < 6; q++) df[q] = (float)(yn[q] - Yold[base + (size_t)q * ld]);
            if (R32)
#pragma unroll
              for (int q = 0; q < 6; q++) R32[base + (size_t)q * ld] = df[q];
            float sr = 1.0f, sv = 1.0f;
            if (s.relative) {
              const float nr = (float)fma(yn[2], yn[2], fma(yn[1], yn[1], yn[0] * yn[0]));
              const float nv = (float)fma(yn[5], yn[5], fma(yn[4], yn[4], yn[3] * yn[3]));
              sr = (nr > 0.0f && nr <= 3.0e38f) ? rsqrtf(nr) : 1.0f;
              sv = (nv > 0.0f && nv <= 3.0e38f) ? rsqrtf(nv) : 1.0f;
            }
            // squared change of |r| and |v| relative to the new iterate (one
            // square root per trajectory, after the maximum)
            const float r0 = df[0] * sr, r1 = df[1] * sr, r2 = df[2] * sr;
            const float v0 = df[3] * sv, v1 = df[4] * sv, v2 = df[5] * sv;
            const float dr = r0 * r0 + r1 * r1 + r2 * r2, dv = v0 * v0 + v1 * v1 + v2 * v2;
            e2 = nanmax(e2, (double)nanmaxf(dr, dv));
          }
        }
        if (EPI == EPI_FULL || EPI == EPI_POS) {
          e2 = nanmax(e2, __shfl_xor_sync(0xffffffffu, e2, 1));
          e2 = nanmax(e2, __shfl_xor_sync(0xffffffffu, e2, 2));
          if (t == 0 && m >= 0) atomicMax(&emax_sh[tt], err_bits(e2));
        }
      }
    }
    __syncthreads();
    // the tile holds every node of its trajectories: the maximum is final
    if (tid < TRAJ) {
      const int m = colm[tid];
      if ((EPI == EPI_FULL || EPI == EPI_POS) && m >= 0)
        c.err[m] = err_bits(sqrt(__longlong_as_double((long long)emax_sh[tid])));
      bad[tid] = 0;
      emax_sh[tid] = 0ULL;
    }
    if (tid < kRows) colB[tid] = 0;
    __syncthreads();  // shared memory is reused by the next tile
  }
}

template <int NC, int Q0, int EPI>
cudaError_t split_attr(const pc_plan *p) {
  return cudaFuncSetAttribute(k_contract_split<NC, Q0, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)split_smem_bytes(p->split_ks));
}

template <int NC, int Q0, int EPI>
void split_launch(const pc_plan *p, const Sweep &s, const Ctl &c, double *G, const double *Yold, double *Ynew,
                  float *R32, long long cols, cudaStream_t st) {
  SplitOp op{reinterpret_cast<const uint2 *>(p->d_Kdig), p->d_Kexp, p->split_nt, p->split_ks};
  const long long tiles = (cols + split_traj(NC) - 1) / split_traj(NC);
  const int sms = p->num_sms > 0 ? p->num_sms : 152;
  const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((long long)sms * kSplitCtasPerSm, tiles));
  k_contract_split<NC, Q0, EPI><<<blocks, kSplitThreads, split_smem_bytes(p->split_ks), st>>>(s, c, op, G, Yold, Ynew,
                                                                                             R32);
}

}  // namespace

bool split_supported(const pc_plan *p) { return p->d_Kdig != nullptr; }

cudaError_t prepare_split(const pc_plan *p) {
  if (!split_supported(p)) return cudaSuccess;
  cudaError_t e = split_attr<6, 0, EPI_FULL>(p);
  if (e == cudaSuccess) e = split_attr<6, 0, EPI_DIAG>(p);
  if (e == cudaSuccess) e = split_attr<3, 3, EPI_VEL>(p);
  if (e == cudaSuccess) e = split_attr<3, 0, EPI_POS>(p);
  return e;
}

cudaError_t launch_contract_split(const pc_plan *p, const Sweep &s, const Ctl &c, double *G, const double *Yold,
                                  double *Ynew, float *R32, int mode, cudaStream_t st) {
  switch (mode) {
    case SPLIT_DIAG: split_launch<6, 0, EPI_DIAG>(p, s, c, G, nullptr, Ynew, nullptr, s.n_ic, st); break;
    case SPLIT_SECOND_ORDER:
      // velocities first; the position pass reads omega2 V' from G's velocity rows
      split_launch<3, 3, EPI_VEL>(p, s, c, G, nullptr, Ynew, nullptr, s.A, st);
      split_launch<3, 0, EPI_POS>(p, s, c, G, Yold, Ynew, R32, s.A, st);
      break;
    default: split_launch<6, 0, EPI_FULL>(p, s, c, G, Yold, Ynew, R32, s.A, st); break;
  }
  return cudaGetLastError();
}

}  // namespace pcx
