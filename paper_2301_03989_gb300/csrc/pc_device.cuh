// Device helpers shared by the sweep kernels (pc_sweep.cu) and the adjoint
// kernels (pc_adjoint.cu): exactly rounded FP64 operations, NaN-propagating
// maxima, the ephemeris evaluation and the FP64 tensor-core MMA.
#pragma once

#include "pc_internal.h"

namespace pcx {
namespace {

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// NaN-propagating maximum of non-negative values.
__device__ __forceinline__ double nanmax(double a, double b) { return (b > a || b != b) ? b : a; }
__device__ __forceinline__ float nanmaxf(float a, float b) { return (b > a || b != b) ? b : a; }

// Non-negative doubles / floats order like their bit patterns; NaN maps to the largest.
__device__ __forceinline__ unsigned long long err_bits(double e) {
  if (e != e) return 0x7FF8000000000000ULL;
  return (unsigned long long)__double_as_longlong(e);
}
__device__ __forceinline__ unsigned err_bits32(float e) {
  if (e != e) return 0x7FC00000u;
  return __float_as_uint(e);
}

// ---------------------------------------------------------------------------
// Ephemeris: Clenshaw evaluation of body b at time t,
//   b_k = c_k + 2 sigma b_{k+1} - b_{k+2},  r = c_0 + sigma b_1 - b_2.
// Every operation is rounded on its own (no fused multiply-add), so the body
// positions are the exactly rounded results of this recurrence: near a body
// the force amplifies a position rounding difference by |r| / |r - r_b|.
// ---------------------------------------------------------------------------
struct EphemLoc {
  int g;
  double sig;
};

__device__ __forceinline__ EphemLoc ephem_locate(const Model &md, double t) {
  int g = (int)floor((t - md.t_begin) / md.granule);
  g = g < 0 ? 0 : (g > md.n_gr - 1 ? md.n_gr - 1 : g);
  const double tg = dadd(md.t_begin, dmul((double)g, md.granule));
  return {g, dsub(dmul(2.0, dsub(t, tg)) / md.granule, 1.0)};
}

__device__ __forceinline__ void ephem_body(const Model &md, EphemLoc L, int b, double r[3]) {
  const double s2 = dmul(2.0, L.sig);
  const int nc = md.deg + 1;
  for (int ax = 0; ax < 3; ax++) {
    const double *cf = md.coef + (((size_t)b * md.n_gr + L.g) * 3 + ax) * nc;
    double b1 = 0.0, b2 = 0.0;
    for (int k = nc - 1; k >= 1; k--) {
      const double b0 = dsub(dadd(cf[k], dmul(s2, b1)), b2);
      b2 = b1;
      b1 = b0;
    }
    r[ax] = dsub(dadd(cf[0], dmul(L.sig, b1)), b2);
  }
}

// FP64 tensor-core MMA, mma.sync m16n8k4 .f64 (PTX ISA).  Fragment layouts,
// with g = lane/4 and t = lane%4:  A: a0 = A[g][t], a1 = A[g+8][t];
// B: b0 = B[t][g];  C/D: d0,d1 = C[g][2t..2t+1], d2,d3 = C[g+8][2t..2t+1].
__device__ __forceinline__ void dmma16x8x4(double (&d)[4], double a0, double a1, double b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
      : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
      : "d"(a0), "d"(a1), "d"(b0));
}

}  // namespace
}  // namespace pcx
