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

// Body velocities: the time derivative of the table's series,
// (2 / granule) sum_{k>=1} c_k k U_{k-1}(sigma), with the Chebyshev
// polynomials of the second kind U_0 = 1, U_1 = 2 sigma, U_{k+1} = 2 sigma
// U_k - U_{k-1} formed once per time; out(b, v) for every body.
template <class Out>
__device__ __forceinline__ void ephem_vel_all(const Model &md, EphemLoc L, Out out) {
  const int nc = md.deg + 1;
  const int m = nc < kEphemMaxCoefs ? nc : kEphemMaxCoefs;
  double U[kEphemMaxCoefs];
  U[0] = 1.0;
  if (m > 1) U[1] = 2.0 * L.sig;
  for (int k = 2; k < m; k++) U[k] = fma(2.0 * L.sig, U[k - 1], -U[k - 2]);
  const double sc = 2.0 / md.granule;
  for (int b = 0; b < md.B; b++) {
    const double *cf = md.coef + ((size_t)b * md.n_gr + L.g) * 3 * nc;
    double v[3] = {0.0, 0.0, 0.0};
    for (int k = m - 1; k >= 1; k--)
      for (int ax = 0; ax < 3; ax++) v[ax] = fma(cf[ax * nc + k] * (double)k, U[k - 1], v[ax]);
    for (int ax = 0; ax < 3; ax++) v[ax] *= sc;
    out(b, v);
  }
}

// Einstein-Infeld-Hoffmann data of the bodies at one time, from their
// heliocentric positions rb and velocities vb [B][3] (the central body at the
// origin): X[7j + 0..2] the barycentric velocity of body j (0 central, 1..B the
// table's), X[7j + 3..5] its Newtonian acceleration and X[7j + 6] its
// Newtonian potential from the other bodies.
__device__ __noinline__ void eih_bodies(const Model &md, const double *rb, const double *vb, double *X) {
  const int B = md.B, nb = B + 1;
  double msum = md.mu_c, vs[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < B; b++) {
    msum += md.mu[b];
    for (int q = 0; q < 3; q++) vs[q] -= md.mu[b] * vb[3 * b + q];
  }
  for (int q = 0; q < 3; q++) vs[q] /= msum;
  for (int j = 0; j < nb; j++) {
    double a[3] = {0.0, 0.0, 0.0}, phi = 0.0;
    for (int k = 0; k < nb; k++) {
      if (k == j) continue;
      double d[3];
      for (int q = 0; q < 3; q++) d[q] = (k ? rb[3 * (k - 1) + q] : 0.0) - (j ? rb[3 * (j - 1) + q] : 0.0);
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2);
      const double mk = k ? md.mu[k - 1] : md.mu_c;
      phi += mk / r;
      for (int q = 0; q < 3; q++) a[q] += mk * d[q] / (r2 * r);
    }
    for (int q = 0; q < 3; q++) {
      X[7 * j + q] = (j ? vb[3 * (j - 1) + q] : 0.0) + vs[q];
      X[7 * j + 3 + q] = a[q];
    }
    X[7 * j + 6] = phi;
  }
}

// The 1/c^2 terms of the EIH acceleration of a massless particle at the
// heliocentric state (r, v) among the central body and the table's bodies
// (positions Eb[(3b + axis) * es], EIH data Xb[f * es] as eih_bodies lays it
// out), velocities taken in the barycentric frame:
//   sum_j mu_j d_j/r_j^3 [ -4 phi - Phi_j + W.W + 2 V_j.V_j - 4 W.V_j
//                          - 3/2 (n_j.V_j)^2 + 1/2 d_j.A_j ] / c^2
// + sum_j mu_j/r_j^3 [ (-d_j).(4 W - 3 V_j) ] (W - V_j) / c^2
// + 7/2 sum_j mu_j A_j / r_j / c^2,
// d_j = P_j - r, n_j = -d_j/r_j, phi = sum_j mu_j/r_j, W = v + V_central.
__device__ __noinline__ void eih_terms(const Model &md, const double *Eb, const double *Xb, size_t es,
                                       const double r[3], const double v[3], double out[3]) {
  const int B = md.B;
  const double c2 = md.c_light * md.c_light;
  const double W[3] = {v[0] + Xb[0], v[1] + Xb[es], v[2] + Xb[2 * es]};
  double phi = 0.0;
  for (int j = 0; j <= B; j++) {
    double d[3];
    for (int q = 0; q < 3; q++) d[q] = (j ? Eb[(size_t)(3 * (j - 1) + q) * es] : 0.0) - r[q];
    phi += (j ? md.mu[j - 1] : md.mu_c) / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  }
  const double ww = W[0] * W[0] + W[1] * W[1] + W[2] * W[2];
  out[0] = out[1] = out[2] = 0.0;
  for (int j = 0; j <= B; j++) {
    double d[3], Vj[3], Aj[3];
    for (int q = 0; q < 3; q++) {
      d[q] = (j ? Eb[(size_t)(3 * (j - 1) + q) * es] : 0.0) - r[q];
      Vj[q] = Xb[(size_t)(7 * j + q) * es];
      Aj[q] = Xb[(size_t)(7 * j + 3 + q) * es];
    }
    const double Phij = Xb[(size_t)(7 * j + 6) * es];
    const double mu = j ? md.mu[j - 1] : md.mu_c;
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], rr = sqrt(r2), r3 = r2 * rr;
    const double vv = Vj[0] * Vj[0] + Vj[1] * Vj[1] + Vj[2] * Vj[2];
    const double wv = W[0] * Vj[0] + W[1] * Vj[1] + W[2] * Vj[2];
    const double nv = -(d[0] * Vj[0] + d[1] * Vj[1] + d[2] * Vj[2]) / rr;
    const double da = d[0] * Aj[0] + d[1] * Aj[1] + d[2] * Aj[2];
    const double br = -4.0 * phi - Phij + ww + 2.0 * vv - 4.0 * wv - 1.5 * nv * nv + 0.5 * da;
    double sdot = 0.0;
    for (int q = 0; q < 3; q++) sdot += -d[q] * (4.0 * W[q] - 3.0 * Vj[q]);
    for (int q = 0; q < 3; q++)
      out[q] += (mu * d[q] / r3 * br + mu / r3 * sdot * (W[q] - Vj[q]) + 3.5 * mu * Aj[q] / rr) / c2;
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
