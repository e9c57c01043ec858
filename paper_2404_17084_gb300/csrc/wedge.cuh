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
// This library writes H = H_far + E, H_far being the value the kernel would
// have as a point mass (E vanishes for u >= 2).  Then for one pyramid
//     I = Omega/(4 pi) - r0 int_0^phi [E(r0) - E(U)] dphi'.
// Summed over a closed cell, the solid angles give 1 when the particle is
// inside the cell and 0 otherwise.  What is left is one integral per face
// edge, over the signed along-edge coordinate s of the exit point
// (s = R0 tan phi', U = sqrt(r0^2 + R0^2 + s^2)):
//     K'_e = int_{a_a}^{a_b} r0 [E(U) - E(r0)] R0/(R0^2 + s^2) ds,
//     f = [inside] + sum_faces sum_edges s_f s_e K'_e,
// with s_f = +1 when the particle is on the inner side of the face plane,
// s_e = +1 when p is on the inner side of the edge line, and a_a < a_b the
// signed positions of the edge's vertices measured from the foot q.  Faces
// with r0 >= 2 contribute nothing.  The integrand vanishes at the foot when
// R0 -> 0 (U -> r0), so K' is insensitive to rounding of R0 and of the
// along-edge coordinates near edges and vertices.
//
// E is piecewise: for u < 1
//     4 pi E(u) = 1/u - 7/5 + 2u^2/3 - 3u^4/10 + u^5/10,
// for 1 <= u < 2
//     120 pi E(u) = (2-u)^5 (1+u)/u = 32/u - 48 + 40u^2 - 30u^3 + 9u^4 - u^5,
// and 0 beyond.  Antiderivatives in s use Phi = atan2(s, R0),
// A = atan2(r0 s, R0 U), L = asinh(s/c), c^2 = r0^2 + R0^2 and
//     r0 int dphi/U = A,   int U^2 = r0^2 Phi + R0 s,
//     int U^3 = R0 s U/2 + R0 (c^2/2 + r0^2) L + r0^3 A,
//     int U^4 = r0^4 Phi + 2 r0^2 R0 s + R0^3 s + R0 s^3/3,
//     int U^5 = R0 s U^3/4 + 3/8 c^2 R0 s U + 3/8 c^4 R0 L + r0^2 int U^3.
// Subtracting r0 E(r0) Phi, the Phi and A terms of the inner piece combine
// into the solid angle Omega = Phi - A, evaluated directly as
//     Omega = atan( s R0 (R0^2 + s^2) / ((U + r0)(R0^2 U + r0 s^2)) ),
// and every other term carries a factor R0:
//     4 pi G'_in = -(1 + r0^6/10) Omega + r0 (2/3 P2 - 3/10 P4 + 1/10 P5),
//     120 pi G''_mid = -(32 - 30 r0^4 - r0^6) Omega + r0 (40 P2 - 30 P3 + 9 P4 - P5)
// with P_k the parts of int U^k free of Phi and A; the middle piece adds
// kappa * dPhi, kappa = (2-r0)^5 (1+r0)/(120 pi) - r0 E(r0) (zero for r0 >= 1),
// and the part of the edge beyond the support adds -r0 E(r0) dPhi.
//
// FP32 (mixed build): in 1 <= u < 2 the monomial form cancels by two to three
// decimal orders near u = 2 (E is tiny there), ~1e-7 absolute per edge in
// FP32.  There the mixed build integrates
//     r0 [E(U) - E(r0)] = N(s)/(120 pi) + kappa,  N = r0 p(U)/U - p(r0),
//     p(u) = (2-u)^5 (1+u),
// taking N R0/(R0^2+s^2) by 6-point Gauss-Legendre.  N vanishes at the poles
// s = +-i R0 and tends to zero with (2-U)^5 at the support, so the integrand
// keeps its relative accuracy where the kernel is small; its only
// singularities are the branch points s = +-i c.  An interval longer than c
// that straddles the foot s = 0 is split there, so that each part starts or
// ends level with the branch points: unsplit, an interval of length 2 sqrt 3
// at c = 1 loses 1e-4 relative; split, the rule's truncation stays below
// ~8e-8 absolute, and an interval no longer than c stays below ~6e-9 unsplit.
#pragma once

#include <cuda_runtime.h>

namespace wedge {

// Work tally (per thread) used for the algorithmic operation count.
struct WorkCount {
  int faces = 0;  // face tests
  int edges = 0;  // edge records read (faces within the support)
  int terms = 0;  // edges contributing a nonzero K'
  int inner = 0;  // inner-piece antiderivative evaluations
  int mid = 0;    // middle-piece intervals
  int outer = 0;  // beyond-the-support intervals
};

// ------------------------------------------------------------------ math wrappers
// FP32 atan2 of this library: octant reduction to t = min(|x|,|y|)/max(|x|,|y|)
// in [0, 1], atan(t) = t P(t^2) with P a degree-8 polynomial fitted here by
// iteratively reweighted least squares on Chebyshev nodes (relative error
// 1.2e-8 in exact arithmetic, ~2 ulp evaluated in FP32), then
// atan2 = (pi/2 - atan) when |y| > |x|, (pi - .) when x is negative (sign
// bit, so that atan2(+-0, -0) = +-pi), sign of y; the two corrections are
// fused multiply-adds with sign factors +-1 (one rounding each, as a
// subtraction).  The quotient uses the hardware reciprocal (2 ulp).
__device__ __forceinline__ float atan2_fast(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  // (the floor FLT_MIN only keeps 0/0 out: t = 0 when x = y = 0)
  const float mx = fmaxf(fmaxf(ax, ay), 1.17549435e-38f), mn = fminf(ax, ay);
  const float t = __fdividef(mn, mx);
  const float u = t * t;
  float p = 0.0028498810715973377f;
  p = fmaf(p, u, -0.0160685945302248f);
  p = fmaf(p, u, 0.042691461741924286f);
  p = fmaf(p, u, -0.07504289597272873f);
  p = fmaf(p, u, 0.10640931874513626f);
  p = fmaf(p, u, -0.14203643798828125f);
  p = fmaf(p, u, 0.1999261975288391f);
  p = fmaf(p, u, -0.3333307206630707f);
  p = fmaf(p, u, 1.0f);
  // the octant and half-plane corrections as sign multiplies:
  // r <- pi/2 - r when |y| > |x| (s1 = -1), r <- pi - r when x is negative
  const float s1 = copysignf(1.f, ax - ay), s2 = copysignf(1.f, x);
  float r = t * p;
  r = fmaf(r, s1, fmaf(-0.785398163397448310f, s1, 0.785398163397448310f));
  r = fmaf(r, s2, fmaf(-1.57079632679489662f, s2, 1.57079632679489662f));
  return copysignf(r, y);
}

__device__ __forceinline__ float xsqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double xsqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float xatan2(float y, float x) { return atan2_fast(y, x); }
__device__ __forceinline__ double xatan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float xasinh(float v) { return asinhf(v); }
__device__ __forceinline__ double xasinh(double v) { return asinh(v); }

constexpr double INV_4PI = 1.0 / (4.0 * 3.14159265358979323846);
constexpr double INV_120PI = 1.0 / (120.0 * 3.14159265358979323846);

// c0 = r0 E(r0)
// (both branches evaluated and selected: no divergence between lanes)
template <typename T>
__device__ __forceinline__ T c0_of(T r0) {
  const T r2 = r0 * r0, r3 = r2 * r0;
  const T a = (T(1) - T(1.4) * r0 + (T(2) / T(3)) * r3 - T(0.3) * r3 * r2 + T(0.1) * r3 * r3) * T(INV_4PI);
  const T t = T(2) - r0, t2 = t * t;
  const T b = t2 * t2 * t * (T(1) + r0) * T(INV_120PI);
  return r0 < T(1) ? a : (r0 < T(2) ? b : T(0));
}

template <typename T>
__device__ __forceinline__ T pmid(T u) {
  const T t = T(2) - u, t2 = t * t;
  return t2 * t2 * t * (T(1) + u);
}

// kappa = r0 E_mid(r0) - r0 E(r0): zero for r0 >= 1 (so only the inner
// branch of r0 E(r0) is needed)
template <typename T>
__device__ __forceinline__ T kappa_of(T r0) {
  const T r2 = r0 * r0, r3 = r2 * r0;
  const T a = (T(1) - T(1.4) * r0 + (T(2) / T(3)) * r3 - T(0.3) * r3 * r2 + T(0.1) * r3 * r3) * T(INV_4PI);
  return r0 < T(1) ? pmid(r0) * T(INV_120PI) - a : T(0);
}

// Phi(hi) - Phi(lo), Phi = atan2(s, R0), in one atan2 (exact for any order of lo, hi)
template <typename T>
__device__ __forceinline__ T dphi(T lo, T hi, T R0) {
  return xatan2((hi - lo) * R0, R0 * R0 + lo * hi);
}

// Solid-angle term Omega = Phi - A at s (atan of num/den with den > 0).
template <typename T>
__device__ __forceinline__ T omega(T r0, T R0, T s, T U) {
  const T den = (U + r0) * (R0 * R0 * U + r0 * s * s);
  return den > T(0) ? xatan2(s * R0 * (R0 * R0 + s * s), den) : T(0);
}

// 4 pi G'_in (WANT_IN) and 120 pi G''_mid (WANT_MID) at s.
// (WITH_L = false: the terms in L left out, for a caller that adds them itself)
template <typename T, bool WANT_IN, bool WANT_MID, bool WITH_L = true>
__device__ __forceinline__ void antider(T r0, T R0, T c2, T c, T s, T& gin, T& gmid) {
  const T U = xsqrt(c2 + s * s);
  const T Om = omega(r0, R0, s, U);
  const T L = WITH_L ? xasinh(s / c) : T(0);
  const T r02 = r0 * r0;
  const T R0s = R0 * s;
  const T P2 = R0s;
  const T P3 = T(0.5) * R0s * U + R0 * (T(0.5) * c2 + r02) * L;
  const T P4 = T(2) * r02 * R0s + R0 * R0 * R0s + R0s * s * s * (T(1) / T(3));
  const T P5 = T(0.25) * R0s * U * U * U + T(0.375) * c2 * R0s * U + T(0.375) * c2 * c2 * R0 * L + r02 * P3;
  const T r06 = r02 * r02 * r02;
  if (WANT_IN) gin = -(T(1) + T(0.1) * r06) * Om + r0 * ((T(2) / T(3)) * P2 - T(0.3) * P4 + T(0.1) * P5);
  if (WANT_MID)
    gmid = -(T(32) - T(30) * r02 * r02 - r06) * Om + r0 * (T(40) * P2 - T(30) * P3 + T(9) * P4 - P5);
}

// Node arithmetic of the Gauss-Legendre rule and the breakpoints.  FP32:
// sqrt(x), x > 0, from the hardware reciprocal square root and one Newton step
// (y <- y + r (x - y^2) / 2, ~1 ulp), and the quotient as a product with the
// hardware reciprocal (2 ulp); FP64: the correctly rounded operations.
__device__ __forceinline__ float gl_sqrt(float x) {
  const float r = rsqrtf(x);
  const float y = x * r;
  return fmaf(0.5f * r, fmaf(-y, y, x), y);
}
__device__ __forceinline__ double gl_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float gl_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double gl_div(double a, double b) { return a / b; }

// 120 pi int_lo^hi r0 [E_mid(U) - E_mid(r0)] R0/(R0^2+s^2) ds by 6-point Gauss-Legendre.
template <typename T>
__device__ __forceinline__ T mid_gl(T r0, T R0, T c2, T lo, T hi) {
  const T gx[3] = {T(0.2386191860831969086305017), T(0.6612093864662645136613996), T(0.9324695142031520278123016)};
  const T gw[3] = {T(0.4679139345726910473898703), T(0.3607615730481386075698335), T(0.1713244923791703450402961)};
  const T pr0 = pmid(r0);
  const T half = T(0.5) * (hi - lo), ctr = T(0.5) * (hi + lo);
  const T R02 = R0 * R0;
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      const T s = ctr + T(sgn) * half * gx[k];
      const T U = gl_sqrt(c2 + s * s);  // >= 1 on a middle piece
      const T den = U * (R02 + s * s);
      acc += gw[k] * (den > T(0) ? gl_div(r0 * pmid(U) - pr0 * U, den) : T(0));
    }
  }
  return R0 * half * acc;
}

// FP32 pairs in one instruction (Blackwell's two-lane FP32 arithmetic,
// round-to-nearest per lane, the same results as two scalar operations).
struct f2 { float x, y; };
__device__ __forceinline__ unsigned long long f2_bits(f2 a) {
  return (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ f2 f2_from(unsigned long long b) {
  return f2{__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32))};
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
  return f2_from(d);
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(d);
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(d);
}
__device__ __forceinline__ f2 sp(float v) { return f2{v, v}; }

// The FP32 rule with the nodes +x_k and -x_k of each pair in one two-lane
// operation.  Per node it differs from the scalar form above in two places:
// the Newton step is taken as y (3/2 - r y/2) (no negated operand; ~1.5 ulp
// instead of ~1), and den carries + 1e-30 in its last FMA instead of a
// floor (the same guard, see below).
template <>
__device__ __forceinline__ float mid_gl<float>(float r0, float R0, float c2, float lo, float hi) {
  const float gx[3] = {0.2386191860831969086305017f, 0.6612093864662645136613996f, 0.9324695142031520278123016f};
  const float gw[3] = {0.4679139345726910473898703f, 0.3607615730481386075698335f, 0.1713244923791703450402961f};
  const float pr0 = pmid(r0);
  const float half = 0.5f * (hi - lo), ctr = 0.5f * (hi + lo);
  const float R02 = R0 * R0;
  f2 acc = sp(0.f);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float hg = half * gx[k];
    const f2 s = add2(sp(ctr), f2{hg, -hg});
    const f2 s2 = mul2(s, s);
    const f2 u2 = add2(sp(c2), s2);
    // square root from the reciprocal square root
    const f2 r = f2{rsqrtf(u2.x), rsqrtf(u2.y)};
    const f2 y = mul2(u2, r);
    // one Newton step, y + r (u2 - y^2)/2 = y (3/2 - r y/2)
    const f2 U = mul2(y, fma2(mul2(sp(-0.5f), r), y, sp(1.5f)));
    // p(U) = (2 - U)^5 (1 + U)
    const f2 t = fma2(U, sp(-1.f), sp(2.f));
    const f2 t2 = mul2(t, t);
    const f2 t5 = mul2(mul2(t2, t2), t);
    const f2 pm = mul2(t5, add2(sp(1.f), U));
    const f2 num = fma2(sp(r0), pm, mul2(sp(-pr0), U));
    // den = 0 only with R0 = 0 (and a node at the foot), where the panel's
    // factor R0 makes the piece 0: 1e-30 added keeps q finite
    const f2 den = fma2(U, add2(sp(R02), s2), sp(1e-30f));
    const f2 q = f2{__fdividef(num.x, den.x), __fdividef(num.y, den.y)};
    acc = fma2(sp(gw[k]), q, acc);
  }
  return R0 * half * (acc.x + acc.y);
}

// ------------------------------------------------------------------ piece evaluators
// Each returns the contribution of one piece of K' over [lo, hi] (lo > hi
// gives the negated value, which carries the sign s_f s_e).

template <typename T>
__device__ __forceinline__ T piece_inner(T r0, T R0, T lo, T hi) {
  const T c2 = r0 * r0 + R0 * R0, c = xsqrt(c2);
  T g1, g0, d;
  antider<T, true, false>(r0, R0, c2, c, hi, g1, d);
  antider<T, true, false>(r0, R0, c2, c, lo, g0, d);
  return (g1 - g0) * T(INV_4PI);
}

// FP32: the L terms of both ends in one logarithm,
//     L(hi) - L(lo) = ln(E(hi) / E(lo)),  E(x) = x + sqrt(c^2 + x^2),
// with E(x) = c^2 / (sqrt(c^2 + x^2) - x) for x < 0 (no cancellation), and
// L's coefficient in 4 pi G'_in, r0/10 (3/8 c^4 + r0^2 (c^2/2 + r0^2)) R0,
// applied once.  The hardware logarithm's absolute error (~2e-7) times that
// coefficient (< 0.2 for an inner piece, c^2 < 1) stays below 3e-9 per piece.
template <>
__device__ __forceinline__ float piece_inner<float>(float r0, float R0, float lo, float hi) {
  const float c2 = r0 * r0 + R0 * R0;
  float g1, g0, d;
  antider<float, true, false, false>(r0, R0, c2, 0.f, hi, g1, d);
  antider<float, true, false, false>(r0, R0, c2, 0.f, lo, g0, d);
  const float U1 = xsqrt(c2 + hi * hi), U0 = xsqrt(c2 + lo * lo);
  const float E1 = hi >= 0.f ? hi + U1 : __fdividef(c2, U1 - hi);
  const float E0 = lo >= 0.f ? lo + U0 : __fdividef(c2, U0 - lo);
  const float dL = __logf(__fdividef(E1, E0));
  const float r02 = r0 * r0;
  const float kL = 0.1f * r0 * R0 * (0.375f * c2 * c2 + r02 * (0.5f * c2 + r02));
  return (g1 - g0 + kL * dL) * float(INV_4PI);
}

// Mixed build: a middle interval straddles the foot s = 0 only when it is no
// longer than c (a longer one is split there), so every call is one
// Gauss-Legendre panel; kappa
// dPhi is evaluated unconditionally (kappa = 0 for r0 >= 1), keeping the
// lanes of a warp on one path.
template <typename T, bool MIXED>
__device__ __forceinline__ T piece_mid(T r0, T R0, T lo, T hi) {
  const T c2 = r0 * r0 + R0 * R0;
  if (MIXED) return mid_gl<T>(r0, R0, c2, lo, hi) * T(INV_120PI) + kappa_of(r0) * dphi(lo, hi, R0);
  const T c = xsqrt(c2);
  T g1, g0, d;
  antider<T, false, true>(r0, R0, c2, c, hi, d, g1);
  antider<T, false, true>(r0, R0, c2, c, lo, d, g0);
  const T v = (g1 - g0) * T(INV_120PI);
  const T k = kappa_of(r0);
  return k != T(0) ? v + k * dphi(lo, hi, R0) : v;
}

template <typename T>
__device__ __forceinline__ T piece_outer(T r0, T R0, T lo, T hi) {
  return -c0_of(r0) * dphi(lo, hi, R0);
}

// Split one edge into pieces, branch-free: with c^2 = r0^2 + R0^2 and the
// breakpoints s2 = sqrt(4 - c^2) (U = 2) and s1 = sqrt(1 - c^2) (U = 1), taken
// as 0 where they do not exist, the edge [aa, ab] gives
//   beyond the support: [aa, min(ab, -s2)] and [max(aa, s2), ab]
//                       (the whole edge as one piece when c^2 >= 4),
//   middle:             [x0, min(x1, -s1)] and [max(x0, s1), x1],
//   inner:              [max(x0, -s1), min(x1, s1)],
// with x0 = max(aa, -s2), x1 = min(ab, s2), each kept when non-empty.  For
// c^2 >= 1 (s1 = 0) a middle interval longer than c is split at the foot
// s = 0, so that each part starts or ends level with the branch points of
// the middle-piece integrand (FP32 only: in FP64 the interval stays whole).
// Every lane runs the same instructions.  The
// breakpoints use the fast square root in FP32: E is smooth across u = 1 and
// u = 2, so moving a breakpoint by an ulp changes K' only at third order.
// Pieces are returned as (lo, hi) with the sign pos folded into the direction
// (lo > hi for pos == false).  r0 > 0 and r0 < 2 are assumed.
template <typename T>
struct EdgeSplit {
  T aa, ab, s1, s2, x0, x1;
  bool far, pos, split;
  bool whole;  // FP64: a middle interval with c^2 >= 1 stays one piece (piece 1)
  unsigned v;  // bit i: piece i non-empty (0 inner, 1-2 middle, 3-4 beyond the support)

  // bounds of piece i (0..4), direction folded in
  __device__ __forceinline__ void get(int i, T& lo, T& hi) const {
    T l, h;
    switch (i) {
      case 0: l = x0 > -s1 ? x0 : -s1; h = x1 < s1 ? x1 : s1; break;
      case 1: l = x0; h = (whole || x1 < -s1) ? x1 : -s1; break;
      case 2: l = x0 > s1 ? x0 : s1; h = x1; break;
      case 3: l = aa; h = far ? ab : (ab < -s2 ? ab : -s2); break;
      default: l = aa > s2 ? aa : s2; h = ab; break;
    }
    lo = pos ? l : h;
    hi = pos ? h : l;
  }
  // bounds of piece i, unfolded (lo <= hi for a non-empty piece)
  __device__ __forceinline__ void get_raw(int i, T& l, T& h) const {
    switch (i) {
      case 0: l = x0 > -s1 ? x0 : -s1; h = x1 < s1 ? x1 : s1; break;
      case 1: l = x0; h = (whole || x1 < -s1) ? x1 : -s1; break;
      case 2: l = x0 > s1 ? x0 : s1; h = x1; break;
      case 3: l = aa; h = far ? ab : (ab < -s2 ? ab : -s2); break;
      default: l = aa > s2 ? aa : s2; h = ab; break;
    }
  }
};

template <typename T>
__device__ __forceinline__ EdgeSplit<T> split_edge_flat(T r0, T R0, T aa, T ab, bool pos, bool on) {
  const T c2 = r0 * r0 + R0 * R0;
  EdgeSplit<T> P;
  P.far = c2 >= T(4);
  if constexpr (sizeof(T) == 4) {
    // both square roots in two-lane arithmetic (gl_sqrt's steps per lane)
    const f2 xs = f2{4.f - c2, 1.f - c2};
    const f2 r = f2{rsqrtf(xs.x), rsqrtf(xs.y)};
    const f2 y = mul2(xs, r);
    const f2 q = fma2(mul2(sp(0.5f), r), fma2(f2{-y.x, -y.y}, y, xs), y);
    P.s2 = P.far ? T(0) : q.x;
    P.s1 = c2 < T(1) ? q.y : T(0);
  } else {
    P.s2 = P.far ? T(0) : gl_sqrt(T(4) - c2);
    P.s1 = c2 < T(1) ? gl_sqrt(T(1) - c2) : T(0);
  }
  P.aa = aa;
  P.ab = ab;
  P.pos = pos;
  P.x0 = aa > -P.s2 ? aa : -P.s2;
  P.x1 = ab < P.s2 ? ab : P.s2;
  // the foot split serves the FP32 quadrature only, and only for a long
  // interval: with the branch points at s = +-ic, a 6-node panel over
  // [x0, x1] of length at most c keeps its truncation below ~6e-9 wherever
  // the interval lies (the Bernstein ellipse of the centred, worst case has
  // rho >= 2 + sqrt 5), under the split pieces' own ~8e-8; the FP64 closed
  // form takes the middle interval whole
  {
    const T len = P.x1 - P.x0;
    P.whole = !(c2 < T(1)) && (sizeof(T) == 8 || len * len <= c2);
  }
  const T s1 = P.s1, s2 = P.s2, x0 = P.x0, x1 = P.x1;
  const bool v0 = (x1 < s1 ? x1 : s1) > (x0 > -s1 ? x0 : -s1);
  const bool v1 = ((P.whole || x1 < -s1) ? x1 : -s1) > x0;
  const bool v2 = !P.whole && x1 > (x0 > s1 ? x0 : s1);
  const bool v3 = (P.far ? ab : (ab < -s2 ? ab : -s2)) > aa;
  const bool v4 = !P.far && ab > (aa > s2 ? aa : s2);
  P.v = on ? (unsigned)v0 | ((unsigned)v1 << 1) | ((unsigned)v2 << 2) | ((unsigned)v3 << 3) | ((unsigned)v4 << 4) : 0u;
  P.split = on && v1 && v2 && !(c2 < T(1));
  return P;
}

// The same split through callbacks (in-thread evaluation).
template <typename T, typename FIn, typename FMid, typename FOut>
__device__ __forceinline__ void split_edge(T r0, T R0, T aa, T ab, bool pos, FIn fin, FMid fmid, FOut fout) {
  const EdgeSplit<T> P = split_edge_flat<T>(r0, R0, aa, ab, pos, true);
  T lo, hi;
  if (P.v & 1u) { P.get(0, lo, hi); fin(lo, hi); }
  if (P.v & 2u) { P.get(1, lo, hi); fmid(lo, hi); }
  if (P.v & 4u) { P.get(2, lo, hi); fmid(lo, hi); }
  if (P.v & 8u) { P.get(3, lo, hi); fout(lo, hi); }
  if (P.v & 16u) { P.get(4, lo, hi); fout(lo, hi); }
}

// K' of one edge evaluated in this thread.
template <typename T, bool MIXED>
__device__ __forceinline__ T kprime_edge(T r0, T R0, T aa, T ab, WorkCount& wc) {
  T acc = T(0);
  split_edge<T>(r0, R0, aa, ab, true,
                [&](T lo, T hi) { acc += piece_inner<T>(r0, R0, lo, hi); wc.inner += 2; },
                [&](T lo, T hi) { acc += piece_mid<T, MIXED>(r0, R0, lo, hi); wc.mid++; },
                [&](T lo, T hi) { acc += piece_outer<T>(r0, R0, lo, hi); wc.outer++; });
  return acc;
}

}  // namespace wedge
