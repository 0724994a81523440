// force_common.cuh -- pieces shared by the force kernels: potential constants,
// the per-block float64 partial sums, and the rare float64 guard-band decision.
#pragma once

#include "nemd_device.cuh"
#include "nemd_internal.cuh"

namespace nemd {

// LJ constants (Sec. 5 potential; WCA = LJ cut at 2^(1/6) sigma, shifted).
struct Pot {
  float eps4, eps24, sig2, ushift;
  double eps4d, eps24d, sig2d, ushiftd;
};

Pot make_pot(const nemd_ctx *c);

// FP64 reductions of the per-block partials (force.cu); half: the partials hold
// every unordered pair once (half neighbourhoods) instead of twice.

// Per-block sums of the per-thread values (float64, fixed order within the
// block) -> partials[blockIdx.x * kPartials + k].
template <int NT>
__device__ __forceinline__ void block_reduce_store(double (&v)[kPartials], double *out) {
  __shared__ double sh[NT / 32][kPartials];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kPartials; k++) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[warp][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < kPartials) {
    double x = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; w++) x += sh[w][threadIdx.x];
    out[(size_t)blockIdx.x * kPartials + threadIdx.x] = x;
  }
}

// Lattice image n of a pair met through stencil image (kx, ky, kz): for the
// dynamic offset frame the brick images of both particles are folded in
// (n = k + m_i - m_j).  Rare path (guard band, pair record): kept out of line.
static __device__ __noinline__ void pair_image(const Geo *g, const double *q, int oi, int oj, int kx, int ky,
                                               int kz, int n[3]) {
  n[0] = kx;
  n[1] = ky;
  n[2] = kz;
  if (g->variant == NEMD_DO) {
    int mi[3], mj[3];
    brick_image(g, q, oi, mi);
    brick_image(g, q, oj, mj);
    for (int a = 0; a < 3; a++) n[a] += mi[a] - mj[a];
  }
}

// Canonical float64 decision of a candidate whose float32 r^2 fell in the fine
// guard band (about 1e-7 of all candidates).  Kept out of line: its float64
// registers would otherwise lower the occupancy of every force kernel.
static __device__ __noinline__ bool guard_band_accept(const Geo *g, const double *q, int oi, int oj, int kx,
                                                      int ky, int kz) {
  int n[3];
  pair_image(g, q, oi, oj, kx, ky, kz, n);
  double d[3];
  return canon_r2(g, q, oi, oj, n[0], n[1], n[2], d) < g->rc2;
}

// Defer a fine-band candidate (sorted i, sorted j, stencil image) to the float64
// fix-up pass; an overflow of the list is reported as a capacity error.
__device__ __forceinline__ void defer_recheck(int4 *list, int *count, int *err, int ki, int j, int kx, int ky,
                                              int kz) {
  const int slot = atomicAdd(count, 1);
  if (slot < kRecheckCap)
    list[slot] = make_int4(ki, j, kx, (ky & 0xffff) | (kz << 16));
  else
    atomicOr(err, ERRB_CAPACITY);
}

// Record one unordered pair in canonical orientation (verification mode).
static __device__ __noinline__ void record_pair(const Geo *g, const double *q, int oi, int oj, int kx, int ky,
                                                int kz, int32_t *buf, unsigned long long *count, long long cap) {
  int n[3];
  pair_image(g, q, oi, oj, kx, ky, kz, n);
  bool canon = (oi < oj) || (oi == oj && (n[0] != 0 ? n[0] > 0 : (n[1] != 0 ? n[1] > 0 : n[2] > 0)));
  if (!canon) return;
  unsigned long long slot = atomicAdd(count, 1ull);
  if ((long long)slot < cap) {
    int32_t *p = buf + 5 * slot;
    p[0] = oi;
    p[1] = oj;
    p[2] = n[0];
    p[3] = n[1];
    p[4] = n[2];
  }
}

// Accumulators of one particle's pair terms (float32).
struct Acc {
  float fx, fy, fz, u, wxx, wyy, wzz, wxy, wxz, wyz;
  int npair;
  __device__ __forceinline__ void zero() {
    fx = fy = fz = u = wxx = wyy = wzz = wxy = wxz = wyz = 0.f;
    npair = 0;
  }
  // LJ force on i from j for displacement d = x_j - x_i (Sec. 5 potential):
  // F_i = -fr d, fr = 24 eps / r^2 [2 (sigma^2/r^2)^6 - (sigma^2/r^2)^3]
  __device__ __forceinline__ void add(const Pot &pp, float dx, float dy, float dz) {
    add_r2(pp, dx, dy, dz, fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
  }
  // the same with r^2 already formed; 1 / r^2 by the fast reciprocal (2 ulp)
  __device__ __forceinline__ void add_r2(const Pot &pp, float dx, float dy, float dz, float r2) {
    float gx, gy, gz;
    add_pair(pp, dx, dy, dz, r2, gx, gy, gz);
  }
  // ... also returning the force on the partner j, g = fr d (the force on i is -g)
  __device__ __forceinline__ void add_pair(const Pot &pp, float dx, float dy, float dz, float r2, float &gx,
                                           float &gy, float &gz) {
    const float inv = __fdividef(1.0f, r2);
    const float s2 = pp.sig2 * inv;
    const float s6 = s2 * s2 * s2;
    const float fr = pp.eps24 * inv * s6 * (2.0f * s6 - 1.0f);
    u += fmaf(pp.eps4 * s6, s6 - 1.0f, -pp.ushift);
    gx = fr * dx;
    gy = fr * dy;
    gz = fr * dz;
    fx -= gx;
    fy -= gy;
    fz -= gz;
    wxx = fmaf(gx, dx, wxx);
    wyy = fmaf(gy, dy, wyy);
    wzz = fmaf(gz, dz, wzz);
    wxy = fmaf(gx, dy, wxy);
    wxz = fmaf(gx, dz, wxz);
    wyz = fmaf(gy, dz, wyz);
    npair++;
  }
  // The same sums without the potential's constant factors, which the caller
  // applies once per particle: fr = (1/r^2) s6 (2 s6 - 1) for the force and
  // virial (times 24 eps) and s6 (s6 - 1) for the energy (times 4 eps, less
  // the shift per pair), s6 = (sigma^2 / r^2)^3.
  __device__ __forceinline__ void add_unscaled(float sig2, float dx, float dy, float dz, float r2) {
    const float inv = __fdividef(1.0f, r2);
    const float s2 = sig2 * inv;
    const float s6 = s2 * s2 * s2;
    const float fr = inv * s6 * fmaf(2.0f, s6, -1.0f);
    u = fmaf(s6, s6 - 1.0f, u);
    const float gx = fr * dx, gy = fr * dy, gz = fr * dz;
    fx -= gx;
    fy -= gy;
    fz -= gz;
    wxx = fmaf(gx, dx, wxx);
    wyy = fmaf(gy, dy, wyy);
    wzz = fmaf(gz, dz, wzz);
    wxy = fmaf(gx, dy, wxy);
    wxz = fmaf(gx, dz, wxz);
    wyz = fmaf(gy, dz, wyz);
    npair++;
  }
};

// t = x_i - (shift + n * step), exact for quantised operands (the fused
// multiply-add rounds once, and the exact result is a representable multiple
// of the quantum).
__device__ __forceinline__ float sub_offset(float x, float shift, int n, float step) {
  return fmaf(-(float)n, step, x - shift);
}

// Residual of t: r_i - (shift_r + n * step_r), float32 (only added back to d).
__device__ __forceinline__ float sub_residual(float r, float shift_r, int n, float step_r) {
  return fmaf(-(float)n, step_r, r - shift_r);
}

}  // namespace nemd
