// nemd_device.cuh -- device helpers used by the wrap and force kernels.
#pragma once

#include "nemd_internal.cuh"

namespace nemd {

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

// Rectangular rearrangement of the rotated box (Sec. 4.2): the point R s is
// moved by lattice vectors into the brick [0,r11) x [0,r22) x [0,r33) --
// first along z (shifting x and y by the third column of R), then y (shifting
// x by r12), then x modulo r11.  b = R (s - m).  The quotients use the
// reciprocals rinv = 1 / r_ii; every caller uses this one function, so the
// binning and the image of a pair agree even for points on a brick face (b
// may then lie a rounding outside the brick; the cell index is clamped).
__device__ __forceinline__ void brick_wrap(const double *R, const double *rinv, const double s[3], double b[3],
                                           int m[3]) {
  double x = R[0] * s[0] + R[1] * s[1] + R[2] * s[2];
  double y = R[4] * s[1] + R[5] * s[2];
  double z = R[8] * s[2];
  double m3 = floor(z * rinv[2]);
  z -= m3 * R[8];
  y -= m3 * R[5];
  x -= m3 * R[2];
  double m2 = floor(y * rinv[1]);
  y -= m2 * R[4];
  x -= m2 * R[1];
  double m1 = floor(x * rinv[0]);
  x -= m1 * R[0];
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
  double s[3], b[3];
  frac_wrap(g->Linv, q[3 * (size_t)oi], q[3 * (size_t)oi + 1], q[3 * (size_t)oi + 2], s);
  brick_wrap(g->R, g->rinv, s, b, m);
}

}  // namespace nemd
