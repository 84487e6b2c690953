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
// Ephemeris: the table's Chebyshev series r = sum_k c_k T_k(sigma) at the
// granule holding t.  T_0 = 1, T_1 = sigma, T_{k+1} = fma(2 sigma, T_k, -T_{k-1})
// are formed once per time and shared by every body and axis; each coordinate
// is then summed from the top degree down with one fused multiply-add per
// term.  This differs from Clenshaw's recurrence only in rounding: both agree
// to a few ulps of sum_k |c_k|.
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

constexpr int kEphemRegCoefs = 16;  // degrees up to 15 keep T_k in registers
constexpr int kEphemMaxCoefs = 64;  // degrees up to 63

// Calls out(b, r) for every body b in order with its position r[3].
template <class Out>
__device__ __forceinline__ void ephem_all(const Model &md, EphemLoc L, Out out);

// Same for the bodies b_lo <= b < b_hi.
template <class Out>
__device__ __forceinline__ void ephem_range(const Model &md, EphemLoc L, int b_lo, int b_hi, Out out) {
  Model sub = md;
  sub.coef = md.coef + (size_t)b_lo * md.n_gr * 3 * (md.deg + 1);
  sub.B = b_hi - b_lo;
  ephem_all(sub, L, [&](int b, const double r[3]) { out(b_lo + b, r); });
}

template <class Out>
__device__ __forceinline__ void ephem_all(const Model &md, EphemLoc L, Out out) {
  const int nc = md.deg + 1;
  const double s2 = 2.0 * L.sig;
  if (nc <= kEphemRegCoefs) {
    double T[kEphemRegCoefs];
    T[0] = 1.0;
    T[1] = L.sig;
#pragma unroll
    for (int k = 2; k < kEphemRegCoefs; k++) T[k] = fma(s2, T[k - 1], -T[k - 2]);
    for (int b = 0; b < md.B; b++) {
      const double *cf = md.coef + ((size_t)b * md.n_gr + L.g) * 3 * nc;
      double r[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int k = kEphemRegCoefs - 1; k >= 0; k--)
        if (k < nc)
#pragma unroll
          for (int ax = 0; ax < 3; ax++) r[ax] = fma(cf[ax * nc + k], T[k], r[ax]);
      out(b, r);
    }
  } else {
    double T[kEphemMaxCoefs];
    const int m = nc < kEphemMaxCoefs ? nc : kEphemMaxCoefs;
    T[0] = 1.0;
    T[1] = L.sig;
    for (int k = 2; k < m; k++) T[k] = fma(s2, T[k - 1], -T[k - 2]);
    for (int b = 0; b < md.B; b++) {
      const double *cf = md.coef + ((size_t)b * md.n_gr + L.g) * 3 * nc;
      double r[3] = {0.0, 0.0, 0.0};
      for (int k = m - 1; k >= 0; k--)
        for (int ax = 0; ax < 3; ax++) r[ax] = fma(cf[ax * nc + k], T[k], r[ax]);
      out(b, r);
    }
  }
}

// One body's position (same arithmetic as ephem_all).
__device__ __forceinline__ void ephem_body(const Model &md, EphemLoc L, int body, double r[3]) {
  Model one = md;
  one.coef = md.coef + (size_t)body * md.n_gr * 3 * (md.deg + 1);
  one.B = 1;
  ephem_all(one, L, [&](int, const double p[3]) {
    r[0] = p[0];
    r[1] = p[1];
    r[2] = p[2];
  });
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
