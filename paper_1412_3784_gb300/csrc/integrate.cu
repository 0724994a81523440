// integrate.cu -- time integration under the flow (the step after the force
// evaluation): SLLOD equations of motion for unit mass in peculiar momenta,
//     dq/dt = p + A q,   dp/dt = F - A p,
// which make every periodic image (q + L_t n, p + A L_t n) of Sec. 2.1 carry
// the same peculiar momentum, integrated by a symmetric splitting:
//     p <- exp(-A h) (p + h F);  rescale;  q <- exp(A dt) q + Phi(dt) p;
//     t <- t + dt;  wrap q into the unit cell of L(t);  F <- F(q, t);
//     p <- h F + exp(-A h) p;  rescale                       (h = dt / 2)
// with Phi(dt) = int_0^dt exp(sA) ds (the drift is exact for fixed p: with
// p = 0 a particle moves affinely with the box, q = L_t s at fixed s).  The
// rescale multiplies p by sqrt(K0 / sum |p|^2) (isokinetic; K0 the initial
// sum), or is skipped.  Sums of |p|^2 are per-block float64 partials added in
// a fixed order by the last block of each kick, so a run repeats bit for bit.
// The paper gives no integrator: this is the reading stated with
// nemd_integrate in include/nemd.h.
//
// Arithmetic: the per-particle kernels (the kicks and the drift) read q and p
// as float64, work in float-float (pairs of float32 from error-free
// transformations, about 2^-47 relative per operation) and write float64, the
// propagators applied as x + (M - I) x so that the large part of x passes
// through exactly; one rounded float64 addition per stored component is their
// only float64 arithmetic (float64 runs at a small fraction of the float32
// rate here).  A value outside [2^-100, 2^100) in magnitude, or not finite,
// sends its particle through the same step in float64.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>

#include "nemd_device.cuh"

namespace nemd {

namespace {

constexpr int kIntThreads = 256;
// int_state layout (doubles); from kDff on, float-float copies (two floats in
// each double slot) of exp(A dt) - I, exp(-A dt/2) - I, Phi(dt), the rescale
// factor and h
constexpr int kE = 0, kEh = 9, kPhi = 18, kK0 = 27, kScale = 28, kH = 29, kThermo = 30, kT0 = 31, kDt = 32,
              kStep = 33, kTnow = 34, kTicket = 35, kDff = 36, kDhff = 45, kPhiff = 54, kScaleff = 63,
              kHff = 64, kIntState = 65;

// The flow matrix by value.
struct Mat9 {
  double a[9];
};

// float-float copy of a float64 value (one thread, set-up only)
__device__ __forceinline__ float2 int_ff2(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}

__device__ __forceinline__ ff st_ff(const double *st, int k) {
  const float2 v = reinterpret_cast<const float2 *>(st)[k];
  return {v.x, v.y};
}

__device__ __forceinline__ void st_set_ff(double *st, int k, double x) {
  reinterpret_cast<float2 *>(st)[k] = int_ff2(x);
}

// float32 to float64 from the bits (exact; zero and subnormal floats give 0,
// an error below 2^-126)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  const unsigned long long ex = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(((unsigned long long)(b & 0x80000000u) << 32) | (ex << 52) |
                                          ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// the float64 nearest to hi + lo: both exactly in float64, one rounded addition
__device__ __forceinline__ double ff_to_double(ff x) { return __dadd_rn(f2d_bits(x.hi), f2d_bits(x.lo)); }

// x + D x for a 3x3 float-float matrix D (row-major, in st from slot k) and
// float-float x: the products and their sums in float-float, x added last
__device__ __forceinline__ void ff_apply(const double *st, int k, const ff x[3], ff out[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const ff d = ff_add(ff_add(ff_mul(st_ff(st, k + 3 * a), x[0]), ff_mul(st_ff(st, k + 3 * a + 1), x[1])),
                        ff_mul(st_ff(st, k + 3 * a + 2), x[2]));
    out[a] = ff_add(x[a], d);
  }
}

// Phi x (float-float)
__device__ __forceinline__ void ff_matvec(const double *st, int k, const ff x[3], ff out[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++)
    out[a] = ff_add(ff_add(ff_mul(st_ff(st, k + 3 * a), x[0]), ff_mul(st_ff(st, k + 3 * a + 1), x[1])),
                    ff_mul(st_ff(st, k + 3 * a + 2), x[2]));
}

__device__ __forceinline__ ff ff_norm2(const ff x[3]) {
  return ff_add(ff_add(ff_mul(x[0], x[0]), ff_mul(x[1], x[1])), ff_mul(x[2], x[2]));
}

// the three components of row i of a float64 N x 3 array in float-float; ok
// is cleared when one is out of the split's range
__device__ __forceinline__ void load_ff3(const double *v, size_t i, ff x[3], bool &ok) {
#pragma unroll
  for (int a = 0; a < 3; a++) x[a] = split_double(v[3 * i + a], ok);
}

__device__ __forceinline__ void mat3(const double *a, const double *b, double *c) {
  double t[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) t[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
  for (int k = 0; k < 9; k++) c[k] = t[k];
}

// exp(B) and int_0^1 exp(sB) ds for a 3x3 B: scaling by 2^-s until
// |B|_1 <= 1/8, Taylor polynomials of degree 16 for both, then s doublings
// exp(2X) = exp(X)^2 and Phi(2X) = (I + exp(X)) Phi(X) (Phi scaled by the step).
__device__ void expm_phi(const double *B, double *E, double *Phi) {
  double nrm = 0.0;
  for (int j = 0; j < 3; j++) nrm = fmax(nrm, fabs(B[j]) + fabs(B[3 + j]) + fabs(B[6 + j]));
  int s = 0;
  if (nrm > 0.125) frexp(nrm * 8.0, &s);
  double X[9];
  for (int k = 0; k < 9; k++) X[k] = ldexp(B[k], -s);
  // Horner: E = I + X (I + X/2 (I + X/3 (...))); P = I + X/2 (I + X/3 (I + ...)) so Phi = P
  double Et[9], Pt[9];
  const int deg = 16;
  for (int k = 0; k < 9; k++) {
    Et[k] = (k % 4 == 0 ? 1.0 : 0.0) + X[k] / deg;
    Pt[k] = (k % 4 == 0 ? 1.0 : 0.0) + X[k] / (deg + 1);
  }
  for (int m = deg - 1; m >= 1; m--) {
    double T1[9], T2[9];
    mat3(X, Et, T1);
    mat3(X, Pt, T2);
    for (int k = 0; k < 9; k++) {
      Et[k] = (k % 4 == 0 ? 1.0 : 0.0) + T1[k] / m;
      Pt[k] = (k % 4 == 0 ? 1.0 : 0.0) + T2[k] / (m + 1);
    }
  }
  // Et = exp(X); Pt = sum_k X^k / (k+1)! = int_0^1 exp(sX) ds
  for (int r = 0; r < s; r++) {
    double T[9], Ip[9];
    for (int k = 0; k < 9; k++) Ip[k] = (k % 4 == 0 ? 1.0 : 0.0) + Et[k];
    mat3(Ip, Pt, T);  // int_0^1 exp(2 s X) ds = (I + exp(X)) int_0^1 exp(sX) ds / 2
    for (int k = 0; k < 9; k++) Pt[k] = 0.5 * T[k];
    mat3(Et, Et, Et);
  }
  for (int k = 0; k < 9; k++) {
    E[k] = Et[k];
    Phi[k] = Pt[k];
  }
}

// Propagators of the step: exp(A dt), exp(-A dt/2), Phi(dt) = dt int_0^1 exp(s dt A) ds;
// the clock: t_k = t0 + k dt, k = 0.
__global__ void k_int_setup(double *st, Mat9 A, double t0, double dt, int thermostat) {
  if (threadIdx.x != 0) return;
  double B[9], Bh[9], P[9], Ph[9];
  for (int k = 0; k < 9; k++) {
    B[k] = dt * A.a[k];
    Bh[k] = -0.5 * dt * A.a[k];
  }
  expm_phi(B, st + kE, P);
  for (int k = 0; k < 9; k++) st[kPhi + k] = dt * P[k];
  expm_phi(Bh, st + kEh, Ph);
  for (int k = 0; k < 9; k++) {
    const double id = (k % 4 == 0) ? 1.0 : 0.0;
    st_set_ff(st, kDff + k, st[kE + k] - id);
    st_set_ff(st, kDhff + k, st[kEh + k] - id);
    st_set_ff(st, kPhiff + k, st[kPhi + k]);
  }
  st_set_ff(st, kScaleff, 1.0);
  st_set_ff(st, kHff, 0.5 * dt);
  st[kScale] = 1.0;
  st[kH] = 0.5 * dt;
  st[kThermo] = thermostat;
  st[kT0] = t0;
  st[kDt] = dt;
  st[kStep] = 0.0;
  st[kTnow] = t0;
  *reinterpret_cast<unsigned long long *>(st + kTicket) = 0ull;
}

// Per-block partial of sum |p|^2 (fixed grid-stride order, shuffle tree).
__device__ __forceinline__ void block_p2(double x, double *part) {
  __shared__ double sh[kIntThreads / 32];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double y = 0.0;
    for (int w = 0; w < kIntThreads / 32; w++) y += sh[w];
    part[blockIdx.x] = y;
  }
}

__global__ void __launch_bounds__(kIntThreads) k_int_p2(const double *__restrict__ p, int n, double *part) {
  double x = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x += (p[3 * (size_t)i] * p[3 * (size_t)i] + p[3 * (size_t)i + 1] * p[3 * (size_t)i + 1]) +
         p[3 * (size_t)i + 2] * p[3 * (size_t)i + 2];
  block_p2(x, part);
}

// Sum of part[0..m) by all threads of one block in a fixed order: each thread
// adds the partials b = tid, tid + blockDim, ... in turn, then the shuffle
// tree of each warp and the warps' sums in warp order (a tree of depth
// ~log2(m) instead of m dependent float64 adds).  The result is in thread 0.
__device__ __forceinline__ double block_sum_fixed(const double *part, int m) {
  __shared__ double sh[kIntThreads / 32];
  double y = 0.0;
  for (int b = threadIdx.x; b < m; b += blockDim.x) y += __ldcg(part + b);
  for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = y;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
  return s;
}

// K0 = sum of the partials; no rescale before the first kick
__global__ void __launch_bounds__(kIntThreads) k_int_k0(double *st, const double *part, int nb) {
  const double y = block_sum_fixed(part, nb);
  if (threadIdx.x != 0) return;
  st[kK0] = y;
  st[kScale] = 1.0;
  st_set_ff(st, kScaleff, 1.0);
}

// After every block has written its partial of sum |p|^2: the last block to
// arrive (ticket in st, returned to zero) sets the rescale factor from the
// partials (block_sum_fixed) and, with tick, advances the clock one step,
// t = t0 + k dt (each operation rounded once).
template <bool TICK>
__device__ __forceinline__ void last_block_scale(double *st, const double *part) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    last = atomicAdd(reinterpret_cast<unsigned long long *>(st + kTicket), 1ull) == (unsigned long long)(gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const double y = block_sum_fixed(part, (int)gridDim.x);
  if (threadIdx.x != 0) return;
  st[kScale] = (st[kThermo] != 0.0 && y > 0.0) ? sqrt(st[kK0] / y) : 1.0;
  st_set_ff(st, kScaleff, st[kScale]);
  if (TICK) {
    const double k = st[kStep] + 1.0;
    st[kStep] = k;
    st[kTnow] = __dadd_rn(st[kT0], __dmul_rn(k, st[kDt]));
  }
  *reinterpret_cast<unsigned long long *>(st + kTicket) = 0ull;
}

__device__ __forceinline__ void mv3(const double *M, double x, double y, double z, double &ox, double &oy,
                                    double &oz) {
  ox = (M[0] * x + M[1] * y) + M[2] * z;
  oy = (M[3] * x + M[4] * y) + M[5] * z;
  oz = (M[6] * x + M[7] * y) + M[8] * z;
}

// first half: p <- exp(-A h) (scale p + h F); the new rescale factor, and the
// clock advanced to the step's end time
__global__ void __launch_bounds__(kIntThreads) k_int_kick1(double *__restrict__ p, const float *__restrict__ F,
                                                           int n, double *st, double *part) {
  const ff h = st_ff(st, kHff), sc = st_ff(st, kScaleff);
  ff x2 = {0.f, 0.f};
  double x2d = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bool ok = true;
    ff v[3], o[3];
    load_ff3(p, (size_t)i, v, ok);
    if (ok) {
#pragma unroll
      for (int a = 0; a < 3; a++) v[a] = ff_add(ff_mul(sc, v[a]), ff_mul_f(h, F[3 * (size_t)i + a]));
      ff_apply(st, kDhff, v, o);
#pragma unroll
      for (int a = 0; a < 3; a++) p[3 * (size_t)i + a] = ff_to_double(o[a]);
      x2 = ff_add(x2, ff_norm2(o));
    } else {
      const double hd = st[kH], sd = st[kScale];
      const double a0 = sd * p[3 * (size_t)i] + hd * (double)F[3 * (size_t)i];
      const double a1 = sd * p[3 * (size_t)i + 1] + hd * (double)F[3 * (size_t)i + 1];
      const double a2 = sd * p[3 * (size_t)i + 2] + hd * (double)F[3 * (size_t)i + 2];
      double ox, oy, oz;
      mv3(st + kEh, a0, a1, a2, ox, oy, oz);
      p[3 * (size_t)i] = ox;
      p[3 * (size_t)i + 1] = oy;
      p[3 * (size_t)i + 2] = oz;
      x2d += (ox * ox + oy * oy) + oz * oz;
    }
  }
  block_p2(ff_to_double(x2) + x2d, part);
  last_block_scale<true>(st, part);
}

// drift: p <- scale p; q <- exp(A dt) q + Phi p, then q wrapped into the unit
// cell of the lattice already evolved to the new time (g).  A particle whose
// fractional coordinates (estimated in float32, error ~1e-6) lie within
// [1e-3, 1 - 1e-3] is inside the cell already and keeps its drifted q; the
// others take the float64 wrap q = L frac(L^-1 q)
// (xf, yf, zf: the new position within a float32 ulp, for the inside test)
__device__ __forceinline__ void drift_store(double *__restrict__ q, size_t i, double xx, double yy, double zz,
                                            float xf, float yf, float zf, const Geo *g) {
  bool inside = true;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const float sa = fmaf(g->Linvff[3 * a + 2].x, zf, fmaf(g->Linvff[3 * a + 1].x, yf, g->Linvff[3 * a].x * xf));
    inside = inside && sa > 1e-3f && sa < 0.999f;
  }
  if (inside) {
    q[3 * i] = xx;
    q[3 * i + 1] = yy;
    q[3 * i + 2] = zz;
  } else {
    double s[3], qp[3];
    frac_wrap(g->Linv, xx, yy, zz, s);
    frac_to_cart(g->L, s, qp);
    q[3 * i] = qp[0];
    q[3 * i + 1] = qp[1];
    q[3 * i + 2] = qp[2];
  }
}

__global__ void __launch_bounds__(kIntThreads) k_int_drift(double *__restrict__ q, double *__restrict__ p, int n,
                                                           const double *__restrict__ st, const Geo *g) {
  const ff sc = st_ff(st, kScaleff);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bool ok = true;
    ff pv[3], qv[3];
    load_ff3(p, (size_t)i, pv, ok);
    load_ff3(q, (size_t)i, qv, ok);
    if (ok) {
      ff e[3], f[3];
#pragma unroll
      for (int a = 0; a < 3; a++) {
        pv[a] = ff_mul(sc, pv[a]);
        p[3 * (size_t)i + a] = ff_to_double(pv[a]);
      }
      // q + (exp(A dt) - I) q + Phi p: the increments first, q added last
      ff_matvec(st, kDff, qv, e);
      ff_matvec(st, kPhiff, pv, f);
      ff x[3];
#pragma unroll
      for (int a = 0; a < 3; a++) x[a] = ff_add(qv[a], ff_add(e[a], f[a]));
      drift_store(q, (size_t)i, ff_to_double(x[0]), ff_to_double(x[1]), ff_to_double(x[2]), x[0].hi, x[1].hi,
                  x[2].hi, g);
    } else {
      const double sd = st[kScale];
      const double px = sd * p[3 * (size_t)i], py = sd * p[3 * (size_t)i + 1], pz = sd * p[3 * (size_t)i + 2];
      p[3 * (size_t)i] = px;
      p[3 * (size_t)i + 1] = py;
      p[3 * (size_t)i + 2] = pz;
      double ex, ey, ez, fx, fy, fz;
      mv3(st + kE, q[3 * (size_t)i], q[3 * (size_t)i + 1], q[3 * (size_t)i + 2], ex, ey, ez);
      mv3(st + kPhi, px, py, pz, fx, fy, fz);
      const double xx = ex + fx, yy = ey + fy, zz = ez + fz;
      drift_store(q, (size_t)i, xx, yy, zz, __double2float_rn(xx), __double2float_rn(yy), __double2float_rn(zz), g);
    }
  }
}

// second half: p <- h F + exp(-A h) p; the new rescale factor
__global__ void __launch_bounds__(kIntThreads) k_int_kick2(double *__restrict__ p, const float *__restrict__ F,
                                                           int n, double *st, double *part) {
  const ff h = st_ff(st, kHff);
  ff x2 = {0.f, 0.f};
  double x2d = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bool ok = true;
    ff v[3], o[3];
    load_ff3(p, (size_t)i, v, ok);
    if (ok) {
      // p + (exp(-A h) - I) p + h F: the increments first, p added last
#pragma unroll
      for (int a = 0; a < 3; a++) {
        const ff d = ff_add(ff_add(ff_add(ff_mul(st_ff(st, kDhff + 3 * a), v[0]),
                                          ff_mul(st_ff(st, kDhff + 3 * a + 1), v[1])),
                                   ff_mul(st_ff(st, kDhff + 3 * a + 2), v[2])),
                            ff_mul_f(h, F[3 * (size_t)i + a]));
        o[a] = ff_add(v[a], d);
        p[3 * (size_t)i + a] = ff_to_double(o[a]);
      }
      x2 = ff_add(x2, ff_norm2(o));
    } else {
      const double hd = st[kH];
      double ox, oy, oz;
      mv3(st + kEh, p[3 * (size_t)i], p[3 * (size_t)i + 1], p[3 * (size_t)i + 2], ox, oy, oz);
      ox += hd * (double)F[3 * (size_t)i];
      oy += hd * (double)F[3 * (size_t)i + 1];
      oz += hd * (double)F[3 * (size_t)i + 2];
      p[3 * (size_t)i] = ox;
      p[3 * (size_t)i + 1] = oy;
      p[3 * (size_t)i + 2] = oz;
      x2d += (ox * ox + oy * oy) + oz * oz;
    }
  }
  block_p2(ff_to_double(x2) + x2d, part);
  last_block_scale<false>(st, part);
}

__global__ void __launch_bounds__(kIntThreads) k_int_final(double *__restrict__ p, int n,
                                                           const double *__restrict__ st) {
  const double sc = st[kScale];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x) p[i] *= sc;
}

int int_err(nemd_ctx *c, int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->msg, sizeof c->msg, fmt, ap);
  va_end(ap);
  return code;
}

bool on_device(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace nemd

namespace nemd {
namespace {

// The lattice at the context's device clock, as nemd_set_state does for a
// device array (no host query: callable while a stream is being captured).
int int_state_at_clock(nemd_ctx *c, double *q, int64_t n, double t_host) {
  c->n = n;
  c->t = t_host;
  c->q_dev = n > 0 ? q : nullptr;
  cudaError_t e = launch_lattice(c, 0, 0.0);
  if (e != cudaSuccess) return int_err(c, NEMD_ERR_CUDA, "integrate lattice: %s", cudaGetErrorString(e));
  c->have_state = true;
  c->have_cells = false;
  return NEMD_OK;
}

// The force evaluation of a step: the cell-list hot path, or (with a skin
// set by nemd_set_verlet) the Verlet list, rebuilt from a cell list when needed.
int int_forces(nemd_ctx *c, int variant, double rc, double t) {
  if (c->vl_skin > 0.0) {
    c->have_cells = true;  // the list's build makes its own cells
    return verlet_forces(c, c->f_int, variant, rc, t);
  }
  int r;
  if ((r = nemd_build_cells(c, variant, rc))) return r;
  return nemd_compute_forces(c, c->f_int, nullptr, nullptr);
}

// One step: first kick (which also advances the device clock), lattice at the
// new time, drift and wrap, the force evaluation, second kick.
int int_step(nemd_ctx *c, double *q, double *p, int64_t n, double t_host, int variant, double rc, int nb) {
  int r;
  k_int_kick1<<<nb, kIntThreads, 0, c->stream>>>(p, c->f_int, (int)n, c->int_state, c->int_part);
  if ((r = int_state_at_clock(c, q, n, t_host))) return r;
  k_int_drift<<<nb, kIntThreads, 0, c->stream>>>(q, p, (int)n, c->int_state, c->geo);
  if ((r = int_forces(c, variant, rc, t_host))) return r;
  k_int_kick2<<<nb, kIntThreads, 0, c->stream>>>(p, c->f_int, (int)n, c->int_state, c->int_part);
  c->launches += 3;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NEMD_OK : int_err(c, NEMD_ERR_CUDA, "integrate: %s", cudaGetErrorString(e));
}

}  // namespace
}  // namespace nemd

extern "C" {

int nemd_integrate(nemd_ctx *c, double *q, double *p, int64_t n, double t0, double dt, int64_t nsteps,
                   int variant, double rc, int thermostat) {
  if (!c) return NEMD_ERR_ARG;
  if (!c->have_flow) return nemd::int_err(c, NEMD_ERR_ORDER, "integrate before set_flow");
  if (n < 0 || n > (int64_t)0x7fffffff / 4 || nsteps < 0 || !(dt > 0.0) || !isfinite(dt) || !isfinite(t0))
    return nemd::int_err(c, NEMD_ERR_ARG, "integrate: bad n, dt or nsteps");
  if (n > 0 && (!q || !p || !nemd::on_device(q) || !nemd::on_device(p)))
    return nemd::int_err(c, NEMD_ERR_ARG, "integrate: q and p must be device arrays");
  if (cudaSetDevice(c->device) != cudaSuccess) return NEMD_ERR_CUDA;
  using namespace nemd;
  const int nb = (int)std::min<int64_t>(std::max<int64_t>((n + kIntThreads - 1) / kIntThreads, 1), 4 * (int64_t)c->sms);
  if (!c->int_state && cudaMalloc((void **)&c->int_state, sizeof(double) * kIntState) != cudaSuccess)
    return nemd::int_err(c, NEMD_ERR_NOMEM, "integrate: state");
  if (!c->int_part && cudaMalloc((void **)&c->int_part, sizeof(double) * 4 * (size_t)c->sms) != cudaSuccess)
    return nemd::int_err(c, NEMD_ERR_NOMEM, "integrate: partials");
  if (c->f_int_cap < n) {
    if (c->f_int) cudaFree(c->f_int);
    c->f_int = nullptr;
    c->f_int_cap = 0;
    if (cudaMalloc((void **)&c->f_int, sizeof(float) * 3 * (size_t)std::max<int64_t>(n, 1)) != cudaSuccess)
      return nemd::int_err(c, NEMD_ERR_NOMEM, "integrate: forces");
    c->f_int_cap = n;
  }
  int r = NEMD_OK;
  // the time of every step comes from the device clock (t0 + k dt, rounded the
  // same way whether the step is launched or replayed)
  Mat9 A;
  for (int k = 0; k < 9; k++) A.a[k] = c->A[k];
  k_int_setup<<<1, 32, 0, c->stream>>>(c->int_state, A, t0, dt, thermostat ? 1 : 0);
  c->launches += 1;
  c->t_dev = c->int_state + kTnow;
  do {
    if ((r = nemd_set_state(c, q, n, t0))) break;
    k_int_p2<<<nb, kIntThreads, 0, c->stream>>>(p, (int)n, c->int_part);
    k_int_k0<<<1, kIntThreads, 0, c->stream>>>(c->int_state, c->int_part, nb);
    c->launches += 2;
    if ((r = int_forces(c, variant, rc, t0))) break;
    int64_t k = 0;
    // the first step is launched (it sizes every buffer); then, unless the
    // options need per-step host work, one step is captured and replayed
    if (nsteps > 0) {
      if ((r = int_step(c, q, p, n, t0 + dt, variant, rc, nb))) break;
      k = 1;
    }
    // (the Verlet list decides its rebuilds on the host: its steps are launched)
    if (nsteps > 2 && c->int_graph && !c->async_host && !c->timing && c->vl_skin == 0.0) {
      // capture on a private stream (the context's may be the legacy default
      // stream, which cannot be captured); replay on the context's stream.  A
      // capture that fails leaves nothing executed: the steps are then launched.
      if (!c->cap_stream) cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      const int64_t l0 = c->launches;
      cudaStream_t home = c->stream;
      bool ok = c->cap_stream && cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
      if (ok) {
        c->stream = c->cap_stream;
        const int rs = int_step(c, q, p, n, t0 + 2.0 * dt, variant, rc, nb);
        c->stream = home;
        ok = cudaStreamEndCapture(c->cap_stream, &graph) == cudaSuccess && rs == NEMD_OK;
        ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
      }
      cudaGetLastError();
      const int64_t per_step = c->launches - l0;
      c->launches = l0;
      if (ok) {
        for (; k < nsteps; k++) {
          if (cudaGraphLaunch(exec, c->stream) != cudaSuccess) {
            r = int_err(c, NEMD_ERR_CUDA, "integrate: step graph launch failed");
            break;
          }
          c->launches += per_step;
        }
      }
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      if (r) break;
    }
    for (; k < nsteps; k++)
      if ((r = int_step(c, q, p, n, t0 + (double)(k + 1) * dt, variant, rc, nb))) break;
    if (r) break;
    k_int_final<<<nb, kIntThreads, 0, c->stream>>>(p, (int)n, c->int_state);
    c->launches += 1;
  } while (false);
  c->t_dev = nullptr;
  c->t = t0 + (double)nsteps * dt;
  if (r) return r;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NEMD_OK : nemd::int_err(c, NEMD_ERR_CUDA, "integrate: %s", cudaGetErrorString(e));
}

}  // extern "C"
