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
// One CTA (4 warps) takes a column tile of 8 trajectories x 6 components from
// a counter: it writes the tile's digits to shared memory as 7 x 48 rows of
// bf16 (row q*8 + tt: component q of trajectory tt), then each warp runs
// node tiles of 8 output nodes: C[(q, tt)][node] = sum_k G~[k][(q, tt)]
// K~[node][k] with the force digits as the A operand (ldmatrix from shared
// memory) and the operator digits as the B operand (fragments precomputed by
// the plan, 128-bit loads from L2).  A thread's accumulators then hold all six
// components of one trajectory at two nodes, which is what the epilogue
// (new iterate, change, residual) needs.
#include <cuda_bf16.h>

#include <algorithm>

#include "pc_device.cuh"
#include "pc_internal.h"

namespace pcx {
namespace {

constexpr int kSplitThreads = 128;
constexpr int kSplitTraj = 8;                   // trajectories per column tile
constexpr int kSplitRows = 6 * kSplitTraj;      // digit rows per slice
constexpr int kSplitCtasPerSm = 2;

// k extent of a digit row in shared memory: 16 per k-step plus 8 (304 bytes
// at 9 k-steps, so the 8 rows of an ldmatrix phase hit distinct banks)
__host__ __device__ inline int split_ksp(int n_ks) { return 16 * n_ks + 8; }
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

template <bool DIAG>
__global__ void __launch_bounds__(kSplitThreads, kSplitCtasPerSm)
    k_contract_split(Sweep s, Ctl c, SplitOp op, const double *__restrict__ G, const double *__restrict__ Yold,
                     double *__restrict__ Ynew, float *__restrict__ R32) {
  extern __shared__ __align__(16) unsigned char split_sm[];
  __nv_bfloat16 *Gd = reinterpret_cast<__nv_bfloat16 *>(split_sm);  // [7][48][ksp]
  __shared__ int colB[kSplitRows];       // largest biased exponent of each column
  __shared__ int colm[kSplitTraj];       // the tile's trajectories (slots), -1 past the end
  __shared__ int bad[kSplitTraj];        // an inf or NaN in one of the trajectory's columns
  __shared__ unsigned long long emax_sh[kSplitTraj];
  __shared__ int tile_sh;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int N = s.N, n = s.n, ld = s.ld;
  const int ksp = split_ksp(op.n_ks), kext = 16 * op.n_ks;
  const int ncols = DIAG ? (int)s.n_ic : s.l64_cnt[s.list_cur];
  const int *map = DIAG ? nullptr : s.l64[s.list_cur];
  const int n_tiles = (ncols + kSplitTraj - 1) / kSplitTraj;
  if (tid < kSplitRows) colB[tid] = 0;
  if (tid < kSplitTraj) {
    bad[tid] = 0;
    emax_sh[tid] = 0ULL;
  }
  for (int iter = 0;; iter++) {
    int tile;
    if (DIAG) {
      tile = blockIdx.x + iter * gridDim.x;
    } else {
      if (tid == 0) tile_sh = atomicAdd(s.tile_ctr, 1);
      __syncthreads();
      tile = tile_sh;
    }
    if (tile >= n_tiles) break;
    const int e0 = tile * kSplitTraj;
    if (tid < kSplitTraj) colm[tid] = (e0 + tid < ncols) ? (DIAG ? e0 + tid : map[e0 + tid]) : -1;
    __syncthreads();
    // ---- column exponents (shared-memory max over the nodes)
    for (int i = tid; i < kSplitRows * n; i += kSplitThreads) {
      const int col = i % kSplitRows, k = i / kSplitRows;
      const int m = colm[col & 7];
      if (m >= 0) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(G[((size_t)k * 6 + (col >> 3)) * ld + m]);
        atomicMax(&colB[col], (int)((b >> 52) & 0x7ff));
      }
    }
    // node 0 of the new iterate is the segment's initial state
    if (tid < kSplitRows) {
      const int q = tid >> 3, m = colm[tid & 7];
      if (m >= 0) Ynew[(size_t)q * ld + m] = c.x[(size_t)q * ld + m];
    }
    __syncthreads();
    // ---- digits, two nodes per thread and step (bf16 pairs along k)
    for (int i = tid; i < kSplitRows * (kext / 2); i += kSplitThreads) {
      const int k = 2 * (i % (kext / 2)), col = i / (kext / 2);
      const int m = colm[col & 7], q = col >> 3, Bc = colB[col];
      if (Bc == 0x7ff && (i % (kext / 2)) == 0) bad[col & 7] = 1;
      int d0[kSplitDigits], d1[kSplitDigits];
      split_digits7((m >= 0 && k < n) ? G[((size_t)k * 6 + q) * ld + m] : 0.0, Bc, d0);
      split_digits7((m >= 0 && k + 1 < n) ? G[((size_t)(k + 1) * 6 + q) * ld + m] : 0.0, Bc, d1);
#pragma unroll
      for (int a = 0; a < kSplitDigits; a++)
        *reinterpret_cast<__nv_bfloat162 *>(Gd + ((size_t)a * kSplitRows + col) * ksp + k) =
            __halves2bfloat162(__int2bfloat16_rn(d0[a]), __int2bfloat16_rn(d1[a]));
    }
    __syncthreads();
    // ---- node tiles: 28 digit-pair products per k-step on the tensor cores
    const int g = lane >> 2, t = lane & 3;
    const int arow = (lane & 7) + ((lane >> 3) & 1) * 8, acol = (lane >> 4) * 8;
    for (int nt = w; nt < op.n_nt; nt += kSplitThreads / 32) {
      float acc[3][kSplitDigits][4];
#pragma unroll
      for (int mt = 0; mt < 3; mt++)
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
          unsigned af[3][4];
#pragma unroll
          for (int mt = 0; mt < 3; mt++)
            ldsm_x4(af[mt], Gd + ((size_t)a * kSplitRows + mt * 16 + arow) * ksp + ks * 16 + acol);
#pragma unroll
          for (int b = 0; b < kSplitDigits - a; b++)
#pragma unroll
            for (int mt = 0; mt < 3; mt++) mma_bf16_16816(acc[mt][a + b], af[mt], bf[b]);
        }
      }
      // ---- epilogue: trajectory g of the tile at nodes 1 + nt*8 + 2t + {0, 1}
      const int m = colm[g];
      double e2 = 0.0;
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int r = nt * 8 + 2 * t + e, j = r + 1;
        if (m < 0 || j > N) continue;
        const int kx = op.kexp[r];
        double yn[6];
#pragma unroll
        for (int q = 0; q < 6; q++) {
          const int mt = q >> 1, idx = (q & 1) * 2 + e;
          long long S[kSplitDigits];
#pragma unroll
          for (int dd = 0; dd < kSplitDigits; dd++) S[dd] = (long long)__float2int_rn(acc[mt][dd][idx]);
          const long long vhi = S[0] * (1LL << 24) + S[1] * (1LL << 16) + S[2] * (1LL << 8) + S[3];
          const long long vlo = S[4] * (1LL << 16) + S[5] * (1LL << 8) + S[6];
          const double v = fma((double)vlo, 0x1p-24, (double)vhi) * pow2i(kx + colB[q * 8 + g] - 2042 - 40);
          yn[q] = c.x[(size_t)q * ld + m] + v;
        }
        if (bad[g])
#pragma unroll
          for (int q = 0; q < 6; q++) yn[q] = __longlong_as_double(0x7FF8000000000000LL);
        const size_t base = (size_t)j * 6 * ld + m;
#pragma unroll
        for (int q = 0; q < 6; q++) Ynew[base + (size_t)q * ld] = yn[q];
        if (!DIAG) {
          double d[6];
#pragma unroll
          for (int q = 0; q < 6; q++) d[q] = yn[q] - Yold[base + (size_t)q * ld];
          if (R32)  // the sweep's residual, for an FP32 correction solve next round
#pragma unroll
            for (int q = 0; q < 6; q++) R32[base + (size_t)q * ld] = (float)d[q];
          // squared change of |r| and |v| relative to the new iterate (one
          // square root per trajectory, after the maximum)
          double dr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          double dv = d[3] * d[3] + d[4] * d[4] + d[5] * d[5];
          if (s.relative) {
            const double nr = yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2];
            const double nv = yn[3] * yn[3] + yn[4] * yn[4] + yn[5] * yn[5];
            if (nr > 0.0) dr = dr / nr;
            if (nv > 0.0) dv = dv / nv;
          }
          e2 = nanmax(e2, nanmax(dr, dv));
        }
      }
      if (!DIAG) {
        e2 = nanmax(e2, __shfl_xor_sync(0xffffffffu, e2, 1));
        e2 = nanmax(e2, __shfl_xor_sync(0xffffffffu, e2, 2));
        if (t == 0 && m >= 0) atomicMax(&emax_sh[g], err_bits(e2));
      }
    }
    __syncthreads();
    // the tile holds every node of its trajectories: the maximum is final
    if (tid < kSplitTraj) {
      const int m = colm[tid];
      if (!DIAG && m >= 0) c.err[m] = err_bits(sqrt(__longlong_as_double((long long)emax_sh[tid])));
      bad[tid] = 0;
      emax_sh[tid] = 0ULL;
    }
    if (tid < kSplitRows) colB[tid] = 0;
    __syncthreads();  // shared memory is reused by the next tile
  }
}

}  // namespace

bool split_supported(const pc_plan *p) { return p->d_Kdig != nullptr; }

cudaError_t prepare_split(const pc_plan *p) {
  if (!split_supported(p)) return cudaSuccess;
  const int bytes = (int)split_smem_bytes(p->split_ks);
  cudaError_t e = cudaFuncSetAttribute(k_contract_split<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_contract_split<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t launch_contract_split(const pc_plan *p, const Sweep &s, const Ctl &c, const double *G, const double *Yold,
                                  double *Ynew, float *R32, int diag, cudaStream_t st) {
  SplitOp op{reinterpret_cast<const uint2 *>(p->d_Kdig), p->d_Kexp, p->split_nt, p->split_ks};
  const long long cols = diag ? s.n_ic : s.A;
  const long long tiles = (cols + kSplitTraj - 1) / kSplitTraj;
  const int sms = p->num_sms > 0 ? p->num_sms : 152;
  const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((long long)sms * kSplitCtasPerSm, tiles));
  const size_t smem = split_smem_bytes(p->split_ks);
  if (diag)
    k_contract_split<true><<<blocks, kSplitThreads, smem, st>>>(s, c, op, G, nullptr, Ynew, nullptr);
  else
    k_contract_split<false><<<blocks, kSplitThreads, smem, st>>>(s, c, op, G, Yold, Ynew, R32);
  return cudaGetLastError();
}

}  // namespace pcx
