// nemd_device.cuh -- device helpers used by the wrap and force kernels.
#pragma once

#include "nemd_internal.cuh"

namespace nemd {

// Verlet list packing: a 10-bit signed field per component (brick images) and
// an 8-bit signed cell offset per component of a list entry.
__device__ __forceinline__ int vl_pack3(int x, int y, int z) {
  return (x & 1023) | ((y & 1023) << 10) | ((z & 1023) << 20);
}
__device__ __forceinline__ int vl_unpack3(int v, int a) {  // sign-extended 10-bit field a
  const int f = (v >> (10 * a)) & 1023;
  return f >= 512 ? f - 1024 : f;
}
__device__ __forceinline__ int vl_pack_k(int x, int y, int z) {
  return (x & 255) | ((y & 255) << 8) | ((z & 255) << 16);
}
__device__ __forceinline__ int vl_unpack_k(int v, int a) { return (int)(signed char)((v >> (8 * a)) & 255); }

__device__ __forceinline__ int floordiv_dev(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
  return q;
}

// Fractional coordinates in the unit cell (Sec. 2, Omega = {sum lambda_i v_i,
// 0 <= lambda_i < 1}): s = L^-1 q, s -= floor(s), and s = 1 (possible after the
// subtraction for tiny negative s) becomes 0.  Every operation is a separate
// IEEE round-to-nearest step in this order, without fused multiply-add, so the
// wrapped position is a fixed function of (L^-1, q).
__device__ __forceinline__ void frac_wrap(const double *Li, double x, double y, double z, double s[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    double v = __dadd_rn(__dadd_rn(__dmul_rn(Li[3 * a], x), __dmul_rn(Li[3 * a + 1], y)), __dmul_rn(Li[3 * a + 2], z));
    v = __dsub_rn(v, floor(v));
    if (v >= 1.0) v = 0.0;
    s[a] = v;
  }
}

// Cartesian position of fractional s: q' = L s, same operation order rules.
__device__ __forceinline__ void frac_to_cart(const double *L, const double s[3], double qp[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++)
    qp[a] = __dadd_rn(__dadd_rn(__dmul_rn(L[3 * a], s[0]), __dmul_rn(L[3 * a + 1], s[1])), __dmul_rn(L[3 * a + 2], s[2]));
}

// ---- float-float arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2 ----
// Built from error-free transformations: TwoSum (Knuth), Fast2Sum (Dekker) and
// TwoProduct through a fused multiply-add.  Every step is an explicit
// round-to-nearest intrinsic, so no compiler contraction changes a result and
// the same inputs give the same bits in every kernel.  Relative error of one
// operation is about 2^-45 of its operands' magnitudes.
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_of(float2 v) { return {v.x, v.y}; }

__device__ __forceinline__ ff fast2sum(float a, float b) {  // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float bb = __fsub_rn(s, x.hi);
  float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  return fast2sum(s, e);
}

__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast2sum(p, e);
}

__device__ __forceinline__ ff ff_mul_f(ff x, float b) {
  const float p = __fmul_rn(x.hi, b);
  float e = __fmaf_rn(x.hi, b, -p);
  e = __fmaf_rn(x.lo, b, e);
  return fast2sum(p, e);
}

// floor(hi + lo) as a float: floor(hi), one lower when hi is an integer and lo < 0
// (a non-integer hi is at least ulp(hi) from every integer, more than |lo|)
__device__ __forceinline__ float ff_floor(ff x) {
  const float f = floorf(x.hi);
  return (f == x.hi && x.lo < 0.f) ? __fsub_rn(f, 1.f) : f;
}

// Float-float split of s in [0, 1) from its bits, integer operations only: hi
// keeps the leading 24 significant bits, lo the next 29 (rounded to 24), then
// the pair is renormalised; values below 2^-74 lose lo (below 2^-126 also hi),
// an error under 2^-98.
__device__ __forceinline__ ff split_unit(double s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(s);
  const int e = (int)(b >> 52);  // biased exponent; s >= 0
  if (e < 1023 - 126) return {0.f, 0.f};
  const unsigned int m_hi = (unsigned int)(b >> 29) & 0x7fffffu;
  const float hi = __int_as_float(((e - 1023 + 127) << 23) | (int)m_hi);
  if (e < 949) return {hi, 0.f};
  const unsigned int m_lo = (unsigned int)b & 0x1fffffffu;
  const float scale = __int_as_float((e - 1075 + 127) << 23);  // 2^(e - 1075), normal for e >= 949
  return fast2sum(hi, __fmul_rn(__uint2float_rn(m_lo), scale));
}

// Float-float split of any double x from its bits (integer operations only):
// exact to 2^-48 relative for 2^-100 <= |x| < 2^100; below, zero (an error
// under 2^-100); at or above, ok is cleared (the caller takes float64).
__device__ __forceinline__ ff split_double(double x, bool &ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e < 1023 - 100) return {0.f, 0.f};
  if (e >= 1023 + 100) {
    ok = false;
    return {0.f, 0.f};
  }
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const unsigned int m_hi = (unsigned int)(b >> 29) & 0x7fffffu;
  const float hi = __uint_as_float(sign | ((unsigned int)(e - 1023 + 127) << 23) | m_hi);
  if (e < 949) return {hi, 0.f};
  const unsigned int m_lo = (unsigned int)b & 0x1fffffffu;
  const float lo = __fmul_rn(__uint2float_rn(m_lo), __int_as_float((e - 1075 + 127) << 23));
  return fast2sum(hi, sign ? -lo : lo);
}

// Fractional coordinates for binning, s = L^-1 q - floor(L^-1 q), in
// float-float.  The float64 definition (frac_wrap) is followed exactly: each
// v_a = (L^-1 q)_a is formed in float-float (within 2^-43 sum_b |L^-1_ab q_b|
// of the float64 value, itself within 2^-51 of that sum of the exact one), and
// whenever v_a lies within 2^-42 (sum + 1) of an integer, the sum reaches 16
// (a position far outside the unit cell), or the inputs are out of range, the
// particle takes the float64 path instead.  So floor(v_a)
// is always the float64 definition's, the wrapped image agrees with the
// canonical one, and s is within tol_a = 2^-42 (sum + 1) of the canonical s.
// exact reports that the float64 path was taken (s64 then holds the canonical s).
__device__ __forceinline__ void frac_wrap_ff(const Geo *g, double x, double y, double z, ff sf[3], double s64[3],
                                             bool &exact, float tol[3]) {
  bool ok = true;
  const ff X = split_double(x, ok), Y = split_double(y, ok), Z = split_double(z, ok);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const ff l0 = ff_of(g->Linvff[3 * a]), l1 = ff_of(g->Linvff[3 * a + 1]), l2 = ff_of(g->Linvff[3 * a + 2]);
    const ff v = ff_add(ff_add(ff_mul(l0, X), ff_mul(l1, Y)), ff_mul(l2, Z));
    const float mag = fmaf(fabsf(l2.hi), fabsf(Z.hi), fmaf(fabsf(l1.hi), fabsf(Y.hi), fabsf(l0.hi) * fabsf(X.hi)));
    const float r = rintf(v.hi);
    const float d = __fadd_rn(__fsub_rn(v.hi, r), v.lo);  // v - r: v.hi - r is exact for |v.hi| < 2^22
    tol[a] = 2.2737368e-13f * (mag * 1.0001f + 1.0f);  // 2^-42 (sum + 1)
    ok = ok && mag < 16.f && fabsf(d) > tol[a];  // (mag < 16 also bounds |v.hi| for the exact v.hi - r)
    const float fl = d < 0.f ? __fsub_rn(r, 1.f) : r;
    sf[a] = ff_add(v, ff{-fl, 0.f});
  }
  exact = !ok;
  if (!ok) {
    frac_wrap(g->Linv, x, y, z, s64);
    sf[0] = split_unit(s64[0]);
    sf[1] = split_unit(s64[1]);
    sf[2] = split_unit(s64[2]);
  }
}

// Rectangular rearrangement of the rotated box (Sec. 4.2) in float-float: the
// point R s is moved by lattice vectors into the brick [0,r11) x [0,r22) x
// [0,r33) -- first along z (shifting x and y by the third column of R), then y
// (shifting x by r12), then x modulo r11.  b = R (s - m).  Every caller (the
// wrap, and the image of a pair in the float64 guard band and the pair record)
// uses this one function on the same split of the same s, so the binning and
// the image of a pair agree even for points on a brick face (b may then lie a
// rounding outside the brick; the cell index is clamped).
__device__ __forceinline__ void brick_wrap_ff(const Geo *g, const ff s[3], ff b[3], int m[3]) {
  const ff r11 = ff_of(g->Rff[0]), r12 = ff_of(g->Rff[1]), r13 = ff_of(g->Rff[2]);
  const ff r22 = ff_of(g->Rff[4]), r23 = ff_of(g->Rff[5]), r33 = ff_of(g->Rff[8]);
  ff x = ff_add(ff_add(ff_mul(r11, s[0]), ff_mul(r12, s[1])), ff_mul(r13, s[2]));
  ff y = ff_add(ff_mul(r22, s[1]), ff_mul(r23, s[2]));
  ff z = ff_mul(r33, s[2]);
  // a shift by 0 lattice vectors leaves a float-float value bit for bit (its
  // hi is already the rounding of hi + lo), so it is skipped: z (s3 in [0, 1))
  // almost never moves
  const float m3 = ff_floor(ff_mul(z, ff_of(g->rinvff[2])));
  if (m3 != 0.f) {
    z = ff_add(z, ff_neg(ff_mul_f(r33, m3)));
    y = ff_add(y, ff_neg(ff_mul_f(r23, m3)));
    x = ff_add(x, ff_neg(ff_mul_f(r13, m3)));
  }
  const float m2 = ff_floor(ff_mul(y, ff_of(g->rinvff[1])));
  if (m2 != 0.f) {
    y = ff_add(y, ff_neg(ff_mul_f(r22, m2)));
    x = ff_add(x, ff_neg(ff_mul_f(r12, m2)));
  }
  const float m1 = ff_floor(ff_mul(x, ff_of(g->rinvff[0])));
  if (m1 != 0.f) x = ff_add(x, ff_neg(ff_mul_f(r11, m1)));
  b[0] = x;
  b[1] = y;
  b[2] = z;
  m[0] = (int)m1;
  m[1] = (int)m2;
  m[2] = (int)m3;
}

// Canonical float64 displacement of the pair (i, j, n):
//   d_a = (q'_j,a - q'_i,a) + ((n1 L_a0 + n2 L_a1) + n3 L_a2),  r2 = (d0^2 + d1^2) + d2^2
// with q' the wrapped positions.  This decides every pair whose float32 r^2
// falls in the guard band, so the pair set is exactly that of the definition.
__device__ __forceinline__ double canon_r2(const Geo *g, const double *q, int oi, int oj, int n1, int n2, int n3,
                                           double d[3]) {
  double si[3], sj[3], qi[3], qj[3];
  frac_wrap(g->Linv, q[3 * (size_t)oi], q[3 * (size_t)oi + 1], q[3 * (size_t)oi + 2], si);
  frac_wrap(g->Linv, q[3 * (size_t)oj], q[3 * (size_t)oj + 1], q[3 * (size_t)oj + 2], sj);
  frac_to_cart(g->L, si, qi);
  frac_to_cart(g->L, sj, qj);
  const double f1 = n1, f2 = n2, f3 = n3;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    double img = __dadd_rn(__dadd_rn(__dmul_rn(f1, g->L[3 * a]), __dmul_rn(f2, g->L[3 * a + 1])), __dmul_rn(f3, g->L[3 * a + 2]));
    d[a] = __dadd_rn(__dsub_rn(qj[a], qi[a]), img);
  }
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// Lattice image of particle oi's brick position relative to its wrapped
// fractional position (dynamic offset frame), recomputed from q.
__device__ __forceinline__ void brick_image(const Geo *g, const double *q, int oi, int m[3]) {
  double s64[3];
  ff sf[3];
  bool exact;
  float tol[3];
  frac_wrap_ff(g, q[3 * (size_t)oi], q[3 * (size_t)oi + 1], q[3 * (size_t)oi + 2], sf, s64, exact, tol);
  ff b[3];
  brick_wrap_ff(g, sf, b, m);
}

}  // namespace nemd
