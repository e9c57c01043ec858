// Closed-form wedge (vertex-pyramid) integrals of the M4 kernel.
//
// Section II-B splits a cell into vertex pyramids characterised by r0 (the
// particle's distance to the face plane), R0 (the in-plane distance from the
// projection point p to the edge line) and phi (the angle at p between the
// foot q of that perpendicular and a vertex).  With h = 1, dOmega = r0 dA/r^3
// reduces one pyramid to
//     I(r0,R0,phi) = r0 int_0^phi [H(U) - H(r0)] dphi',
//     U(phi') = sqrt(r0^2 + R0^2 sec^2 phi'),  H' = F/u^2,
// with 4 pi F(u) the kernel mass inside radius u.
//
// This library writes H = H_far + E, where H_far is the value the kernel would
// have as a point mass (E vanishes for u >= 2).  Then
//     I = Omega/(4 pi) - C,  C = r0 E(r0) phi - J(phi),  J = r0 int_0^phi E(U) dphi'.
// Summed over a closed cell, the solid-angle parts give 1 when the particle
// is inside the cell and 0 otherwise, and the r0 E(r0) phi parts of one face
// give 2 pi r0 E(r0) when p lies inside that face's polygon.  What is left is
// one integral per edge, over the signed along-edge coordinate s of the
// exit point (s = R0 tan phi'):
//     K = int_{a_a}^{a_b} r0 E(U(s)) R0/(R0^2 + s^2) ds,  U = sqrt(r0^2 + R0^2 + s^2),
// so that  f = [inside] - sum_faces s_f (2 pi r0 E(r0) [p in face] - sum_edges s_e K).
// Faces with r0 >= 2 and edges with r0^2 + R0^2 >= 4 contribute nothing.
//
// E is piecewise: for u < 1
//     4 pi E(u) = 1/u - 7/5 + 2u^2/3 - 3u^4/10 + u^5/10,
// for 1 <= u < 2
//     120 pi E(u) = (2-u)^5 (1+u)/u = 32/u - 48 + 40u^2 - 30u^3 + 9u^4 - u^5.
// The antiderivatives in s use the elementary integrals of U^k dphi
// (k = -1, 2, 3, 4, 5): with Phi = atan2(s, R0), A = atan2(r0 s, R0 U),
// L = asinh(s/c), c^2 = r0^2 + R0^2:
//     r0 int dphi/U = A,   int U^2 = r0^2 Phi + R0 s,
//     int U^3 = R0 s U/2 + R0 (c^2/2 + r0^2) L + r0^3 A,
//     int U^4 = r0^4 Phi + 2 r0^2 R0 s + R0^3 s + R0 s^3/3,
//     int U^5 = R0 s U^3/4 + 3/8 c^2 R0 s U + 3/8 c^4 R0 L + r0^2 int U^3.
// All are odd in s, so signed s needs no case split.
//
// FP32 (mixed build): in 1 <= u < 2 the monomial form above cancels by two to
// three decimal orders (E is tiny near u = 2), which costs ~1e-7 absolute per
// edge in FP32.  There the mixed build integrates instead
//     r0 E(U) R0/(R0^2+s^2) = [p(r0) + N(s)] R0/(R0^2+s^2) / (120 pi),
//     p(u) = (2-u)^5 (1+u),  N(s) = r0 p(U)/U - p(r0),
// taking the pole term exactly (p(r0) dPhi) and the smooth remainder
// N(s)/(R0^2+s^2) by 6-point Gauss-Legendre; the remainder's only
// singularities are the branch points s = +-i c, at distance >= 1 from the
// interval, so six nodes reach ~1e-8.
#pragma once

#include <cuda_runtime.h>

namespace wedge {

// Work tally (per thread) used for the algorithmic operation count.
struct WorkCount {
  int faces = 0;  // face tests
  int edges = 0;  // edge records read (faces within the support)
  int terms = 0;  // edge integrals evaluated
  int inner = 0;  // inner-piece antiderivative evaluations
  int mid = 0;    // middle-piece intervals (closed form: 2 evaluations; mixed: one GL-6 interval)
};

// ------------------------------------------------------------------ math wrappers
__device__ __forceinline__ float xsqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double xsqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float xatan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double xatan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float xasinh(float v) { return asinhf(v); }
__device__ __forceinline__ double xasinh(double v) { return asinh(v); }

// 2 pi r0 E(r0): the face term when p lies inside the face polygon.
template <typename T>
__device__ __forceinline__ T face_term(T r0) {
  if (r0 < T(1)) {
    T r2 = r0 * r0, r3 = r2 * r0;
    return T(0.5) * (T(1) - T(1.4) * r0 + (T(2) / T(3)) * r3 - T(0.3) * r3 * r2 + T(0.1) * r3 * r3);
  }
  if (r0 < T(2)) {
    T t = T(2) - r0, t2 = t * t;
    return t2 * t2 * t * (T(1) + r0) * (T(1) / T(60));
  }
  return T(0);
}

// Antiderivative pieces at signed s.  Returns 4 pi G_in (inner) and
// 120 pi G_mid (middle) where G = r0 int E dphi from 0 to s.
template <typename T, bool WANT_IN, bool WANT_MID>
__device__ __forceinline__ void antider(T r0, T R0, T c2, T c, T s, T& gin, T& gmid) {
  T U = xsqrt(c2 + s * s);
  T Phi = xatan2(s, R0);
  T A = xatan2(r0 * s, R0 * U);
  T L = xasinh(s / c);
  T r02 = r0 * r0, r03 = r02 * r0;
  T R0s = R0 * s;
  T P2 = r02 * Phi + R0s;
  T P3 = T(0.5) * R0s * U + R0 * (T(0.5) * c2 + r02) * L + r03 * A;
  T P4 = r02 * r02 * Phi + T(2) * r02 * R0s + R0 * R0 * R0s + R0s * s * s * (T(1) / T(3));
  T P5 = T(0.25) * R0s * U * U * U + T(0.375) * c2 * R0s * U + T(0.375) * c2 * c2 * R0 * L + r02 * P3;
  if (WANT_IN) gin = A - T(1.4) * r0 * Phi + (T(2) / T(3)) * r0 * P2 - T(0.3) * r0 * P4 + T(0.1) * r0 * P5;
  if (WANT_MID)
    gmid = T(32) * A - T(48) * r0 * Phi + T(40) * r0 * P2 - T(30) * r0 * P3 + T(9) * r0 * P4 - r0 * P5;
}

template <typename T>
__device__ __forceinline__ T pmid(T u) {
  T t = T(2) - u, t2 = t * t;
  return t2 * t2 * t * (T(1) + u);
}

// 120 pi * int_lo^hi r0 E_mid(U) R0/(R0^2+s^2) ds by pole subtraction + 6-point Gauss-Legendre.
template <typename T>
__device__ __forceinline__ T mid_gl(T r0, T R0, T c2, T lo, T hi) {
  const T gx[3] = {T(0.2386191860831969086305017), T(0.6612093864662645136613996), T(0.9324695142031520278123016)};
  const T gw[3] = {T(0.4679139345726910473898703), T(0.3607615730481386075698335), T(0.1713244923791703450402961)};
  T pr0 = pmid(r0);
  T dphi = xatan2((hi - lo) * R0, R0 * R0 + lo * hi);
  T half = T(0.5) * (hi - lo), ctr = T(0.5) * (hi + lo);
  T R02 = R0 * R0;
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      T s = ctr + T(sgn) * half * gx[k];
      T U = xsqrt(c2 + s * s);
      T N = r0 * pmid(U) / U - pr0;
      T den = R02 + s * s;
      acc += gw[k] * (den > T(0) ? N / den : T(0));
    }
  }
  return pr0 * dphi + R0 * half * acc;
}

// Edge integral K (see the file header) for one face edge: r0 > 0 is the
// particle's distance to the face plane, R0 >= 0 the projection point's
// distance to the edge line, a_a < a_b the signed along-edge coordinates of
// the edge's vertices measured from the foot q.  All lengths in units of h.
// MIXED selects the FP32 scheme for the middle piece.
template <typename T, bool MIXED>
__device__ __forceinline__ T edge_integral(T r0, T R0, T a_a, T a_b, WorkCount& wc) {
  T c2 = r0 * r0 + R0 * R0;
  if (!(r0 > T(0)) || c2 >= T(4)) return T(0);
  T s2 = xsqrt(T(4) - c2);
  T x0 = a_a > -s2 ? a_a : -s2;
  T x1 = a_b < s2 ? a_b : s2;
  if (!(x1 > x0)) return T(0);
  T c = xsqrt(c2);
  T acc_in = T(0), acc_mid = T(0);
  if (c2 < T(1)) {
    T s1 = xsqrt(T(1) - c2);
    T lo = x0 > -s1 ? x0 : -s1;
    T hi = x1 < s1 ? x1 : s1;
    if (hi > lo) {
      T g1, g0, d;
      antider<T, true, false>(r0, R0, c2, c, hi, g1, d);
      antider<T, true, false>(r0, R0, c2, c, lo, g0, d);
      acc_in = g1 - g0;
      wc.inner += 2;
    }
    if (x0 < -s1) {
      ++wc.mid;
      T hi2 = x1 < -s1 ? x1 : -s1;
      if (MIXED) {
        acc_mid += mid_gl<T>(r0, R0, c2, x0, hi2);
      } else {
        T g1, g0, d;
        antider<T, false, true>(r0, R0, c2, c, hi2, d, g1);
        antider<T, false, true>(r0, R0, c2, c, x0, d, g0);
        acc_mid += g1 - g0;
      }
    }
    if (x1 > s1) {
      ++wc.mid;
      T lo2 = x0 > s1 ? x0 : s1;
      if (MIXED) {
        acc_mid += mid_gl<T>(r0, R0, c2, lo2, x1);
      } else {
        T g1, g0, d;
        antider<T, false, true>(r0, R0, c2, c, x1, d, g1);
        antider<T, false, true>(r0, R0, c2, c, lo2, d, g0);
        acc_mid += g1 - g0;
      }
    }
  } else {
    ++wc.mid;
    if (MIXED) {
      acc_mid = mid_gl<T>(r0, R0, c2, x0, x1);
    } else {
      T g1, g0, d;
      antider<T, false, true>(r0, R0, c2, c, x1, d, g1);
      antider<T, false, true>(r0, R0, c2, c, x0, d, g0);
      acc_mid = g1 - g0;
    }
  }
  return acc_in * T(1.0 / (4.0 * 3.14159265358979323846)) + acc_mid * T(1.0 / (120.0 * 3.14159265358979323846));
}

}  // namespace wedge
