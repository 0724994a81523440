// verlet.cu -- Verlet neighbour list with a skin for nemd_integrate.
//
// The paper rebuilds its cell list at every step (Sec. 4.1).  With a skin the
// integrator keeps the pairs found within rl = rc + skin by one cell-list
// search (either variant) and evaluates only those at the following steps,
// rebuilding when a pair outside the list could have come within rc:
//
// * images: the integrator wraps positions into the unit cell of L(t) at every
//   step; fractional coordinates change only by a particle's peculiar
//   displacement, so the lattice vector m_i the wrap has moved particle i by
//   since the build is the integer nearest to s_i(build) - s_i(t), and a
//   listed pair (i, j, n) is the pair (i, j, n + m_j - m_i) at time t;
// * deformation: until the next remap L(t) = exp(A (t - t_b)) L(t_b), and
//   d|F x|^2/dt = 2 (F x)^T A (F x) >= 2 mu |F x|^2 (F = exp(A (t - t_b)), mu
//   the smallest eigenvalue of the symmetric part of A), so a pair at
//   distance |d_b| >= rl at the build is at least exp(mu (t - t_b)) rl - 2 delta
//   away at t, delta the largest peculiar displacement |L(t) u_i|.  The host
//   rebuilds when that falls below rc, and at every remap.
//
// Every listed pair carries the integer offset k between the cells of its two
// particles in a dynamic size grid of the build (cells at least rl wide),
// images included.  At each step a particle's position is taken relative to
// the centre of its build cell in the current lattice, p_i = G (c (s_i + m_i)
// - idx_i - 1/2) with G = L(t) / c, as an exact multiple of a quantum plus a
// float32 residual, so the displacement of a listed pair is
//     d = (p_j - p_i) + G k
// exactly in its quantised part -- the same precision scheme and guard bands
// as the cell-list kernels, with the candidates within float32 rounding of rc
// decided in float64 by the same fix-up pass (canonical images, Sec. 2).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "force_common.cuh"

namespace nemd {

namespace {

constexpr int kVlThreads = 128;
// Per-step position and residual of a particle in one 32-byte record
// (vl_pos[2k], vl_pos[2k + 1]): a gather of both touches one sector.
constexpr int kVlRec = 2;



// The list's grid at the build: c_a = floor(h_a / rl) cells along lattice
// direction a (at least 1).
__device__ __forceinline__ void list_counts(const Geo *g, double rl, int c[3]) {
  for (int a = 0; a < 3; a++) c[a] = max(1, (int)floor(g->h[a] / rl));
}

// Per sorted particle k at the build: fractional position s_b (the canonical
// wrap of Sec. 2), its cell of the list grid, the brick image of the dynamic
// offset frame (0 for dynamic size), and the particle's slot.
__global__ void k_vl_init(const Geo *__restrict__ g, const double *__restrict__ q, const float4 *__restrict__ pos4,
                          int n, double rl, double *__restrict__ sb, int4 *__restrict__ idx, int *__restrict__ slot,
                          VlGeo *vg) {
  int c[3];
  list_counts(g, rl, c);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    for (int a = 0; a < 3; a++) vg->c[a] = c[a];
    vg->rl = rl;
  }
  if (k >= n || (g->error & (ERRB_BOX | ERRB_CAPACITY))) return;
  const int oi = __float_as_int(pos4[k].w);
  double s[3];
  frac_wrap(g->Linv, q[3 * (size_t)oi], q[3 * (size_t)oi + 1], q[3 * (size_t)oi + 2], s);
  int m[3] = {0, 0, 0};
  if (g->variant == NEMD_DO) brick_image(g, q, oi, m);
  for (int a = 0; a < 3; a++) sb[3 * (size_t)k + a] = s[a];
  idx[k] = make_int4(min((int)floor(s[0] * c[0]), c[0] - 1), min((int)floor(s[1] * c[1]), c[1] - 1),
                     min((int)floor(s[2] * c[2]), c[2] - 1), vl_pack3(m[0], m[1], m[2]));
  slot[oi] = k;
}

// The list from the cell list of the build (built at the cut-off rl): every
// candidate whose quantised distance passes the coarse test at rl (a superset
// of the pairs within rl).  COUNT: entries per particle only.  Otherwise the
// entries (sorted j, cell offset k = idx_j - idx_i + c n, n the pair's lattice
// image) in ELL layout (entry e of particle k at ent[e n + k]), at most maxk
// per particle; both report the largest count in maxcnt (the host repeats
// the fill with more room if it exceeded maxk).
template <bool COUNT>
__global__ void __launch_bounds__(kVlThreads) k_vl_build(
    Geo *__restrict__ g, const float4 *__restrict__ pos, const int *__restrict__ cell_sorted,
    const int *__restrict__ start, const Row *__restrict__ rows, const int *__restrict__ rowcnt, int n,
    const int4 *__restrict__ idx, const VlGeo *__restrict__ vg, int *__restrict__ cnt, int2 *__restrict__ ent,
    int maxk, unsigned *__restrict__ maxcnt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  int e = 0;
  if (k < n && !(g->error & (ERRB_BOX | ERRB_CAPACITY))) {
    const float4 pi = pos[k];
    const int cell = cell_sorted[k];
    const int l1 = g->nc[0], l2 = g->nc[1];
    const int ix = cell % l1, rest = cell / l1, iy = rest % l2, iz = rest / l2;
    const int cls = iy + l2 * iz;
    const Row *rw = rows + (size_t)cls * g->maxrows;
    const int nr = rowcnt[cls];
    const float hi = g->rc2_hi;
    const float sx = g->step[0], sy = g->step[1], sz = g->step[2];
    const bool dyn_offset = g->variant == NEMD_DO;
    const int4 ii = idx[k];
    const int c0 = vg->c[0], c1 = vg->c[1], c2 = vg->c[2];
    for (int r = 0; r < nr; r++) {
      const Row R = rw[r];
      const int jxu = ix + R.dxlo;
      int kx = floordiv_dev(jxu, l1);
      int jx = jxu - kx * l1;
      for (int m = 0; m < R.cnt; m++) {
        const int nidx = R.dxlo + m + R.sxi;
        const float tx = sub_offset(pi.x, R.shx, nidx, sx), ty = sub_offset(pi.y, R.shy, nidx, sy),
                    tz = sub_offset(pi.z, R.shz, nidx, sz);
        const int cj = R.cbase + jx;
        for (int j = start[cj], je = start[cj + 1]; j < je; j++) {
          const float4 pj = pos[j];
          const float dx = pj.x - tx, dy = pj.y - ty, dz = pj.z - tz;
          if (!(fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < hi)) continue;
          if (j == k && kx == 0 && R.ky == 0 && R.kz == 0) continue;  // the particle itself
          if (!COUNT) {
            const int4 jj = idx[j];
            int n1 = kx, n2 = R.ky, n3 = R.kz;
            if (dyn_offset) {  // brick images: n = k + m_i - m_j
              n1 += vl_unpack3(ii.w, 0) - vl_unpack3(jj.w, 0);
              n2 += vl_unpack3(ii.w, 1) - vl_unpack3(jj.w, 1);
              n3 += vl_unpack3(ii.w, 2) - vl_unpack3(jj.w, 2);
            }
            if (e < maxk)
              ent[(size_t)e * n + k] =
                  make_int2(j, vl_pack_k(jj.x - ii.x + c0 * n1, jj.y - ii.y + c1 * n2, jj.z - ii.z + c2 * n3));
          }
          e++;
        }
        if (++jx == l1) {
          jx = 0;
          kx++;
        }
      }
    }
    atomicMax(maxcnt, (unsigned)e);
    if (!COUNT) cnt[k] = min(e, maxk);
  }
}

// The geometry of the list force at this step (one thread): G = L(t) / c;
// a quantum q (power of two) with every quantised value a kernel forms (cell
// positions, |k| <= 4 cells of offset, the displacement) below 2^23 q; G as an
// exact multiple of q plus a float32 residual; the coarse and fine float32
// bands of the cut-off rc as for the cell lists (the positions come from
// float64, so no wrap term).  The force of the list is Cartesian: the frame is
// the dynamic size one.
__global__ void k_vl_geo(Geo *g, VlGeo *vg, double rc) {
  if (threadIdx.x != 0) return;
  double gmax = 0.0;
  for (int a = 0; a < 3; a++) {
    double rs = 0.0;
    for (int b = 0; b < 3; b++) {
      const double v = g->L[3 * a + b] / (double)vg->c[b];
      vg->G[3 * a + b] = v;
      rs += fabs(v);
    }
    gmax = fmax(gmax, rs);
  }
  const double M = 8.0 * gmax + 2.0 * (rc + vg->rl);
  int e2;
  frexp(M, &e2);
  const double q = ldexp(1.0, e2 - 23);
  vg->quantum = q;
  vg->quantum_inv = ldexp(1.0, 23 - e2);
  vg->quantum_f = (float)q;
  vg->quantum_inv_f = (float)vg->quantum_inv;
  for (int k = 0; k < 9; k++) {
    const double sq = rint(vg->G[k] / q) * q;
    vg->Gq[k] = (float)sq;
    vg->Gr[k] = (float)(vg->G[k] - sq);
    const float hi = __double2float_rn(vg->G[k]);
    vg->Gff[k] = make_float2(hi, __double2float_rn(vg->G[k] - (double)hi));
    vg->Lf[k] = __double2float_rn(g->L[k]);
  }
  // coarse band: the omitted residuals (two positions, q / 2 each per
  // component, and G_r k, |k| <= 4: 6 q) and the rounding of r^2; fine band:
  // one rounding of each corrected component and of r^2
  const double u = 5.9604644775390625e-08;
  const double s3 = 1.7320508075688772;
  const double E = 8.0 * q, E2 = 2.0 * u * (rc + q);
  const double band = 2.0 * (2.0 * s3 * rc * E + 3.0 * E * E + 3.0 * u * rc * rc) + 1e-12 * rc * rc;
  const double band2 = 2.0 * (2.0 * s3 * rc * E2 + 3.0 * E2 * E2 + 3.0 * u * rc * rc) + 1e-12 * rc * rc;
  vg->rc2_lo = __double2float_rd(rc * rc - band);
  vg->rc2_hi = __double2float_ru(rc * rc + band);
  vg->rc2_lo2 = __double2float_rd(rc * rc - band2);
  vg->rc2_hi2 = __double2float_ru(rc * rc + band2);
  g->variant = NEMD_DS;  // pair images are plain lattice images; F and W Cartesian
  g->rc = rc;
  g->rc2 = rc * rc;
  for (int k = 0; k < 9; k++) g->Qf[k] = (k % 4 == 0) ? 1.0f : 0.0f;
}

// Per input particle at a step: its fractional position s (the canonical
// wrap, in float-float: frac_wrap_ff takes float64 wherever the float-float
// floor could differ), the image m = round(s_b - s) the wrap has moved it by
// since the build, its peculiar displacement |L u| (u = s + m - s_b, in float;
// the largest goes to disp as float bits), and its position relative to the
// centre of its build cell, p = G (c (s + m) - idx - 1/2), in float-float,
// split into an exact multiple of the quantum and a float32 residual, stored
// at its sorted slot (.w: input index; the residual's .w: m packed).  The
// float-float p is within ~2^-44 |p| of the float64 value: far below the
// float32 residual's rounding, which the guard bands already cover.
__global__ void __launch_bounds__(kVlThreads) k_vl_pos(const Geo *__restrict__ g, const VlGeo *__restrict__ vg,
                                                       const double *__restrict__ q, int n,
                                                       const int *__restrict__ slot, const double *__restrict__ sb,
                                                       const int4 *__restrict__ idx, float4 *__restrict__ pos,
                                                       float4 *__restrict__ res, unsigned *__restrict__ disp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float dmax = 0.0f;
  if (i < n) {
    const int k = slot[i];
    ff s[3];
    double s64[3];
    bool exact;
    float tol[3];
    frac_wrap_ff(g, q[3 * (size_t)i], q[3 * (size_t)i + 1], q[3 * (size_t)i + 2], s, s64, exact, tol);
    const int4 ii = idx[k];
    int m[3];
    ff t3[3];
    float u[3];
    const int ic[3] = {ii.x, ii.y, ii.z};
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const ff b = split_unit(sb[3 * (size_t)k + a]);
      m[a] = (int)rintf(__fsub_rn(b.hi, s[a].hi));  // |s_b - s - m| is a small displacement
      const ff hs = ff_add(s[a], ff{(float)m[a], 0.f});
      const ff du = ff_add(hs, ff_neg(b));
      u[a] = __fadd_rn(du.hi, du.lo);
      // c (s + m) - idx - 1/2 (c and idx + 1/2 exact in float)
      t3[a] = ff_add(ff_mul_f(hs, (float)vg->c[a]), ff{-((float)ic[a] + 0.5f), 0.f});
    }
    float du2 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const float v = fmaf(vg->Lf[3 * a + 2], u[2], fmaf(vg->Lf[3 * a + 1], u[1], vg->Lf[3 * a] * u[0]));
      du2 = fmaf(v, v, du2);
    }
    dmax = sqrtf(du2) * (1.0f + 1e-5f) + 1e-12f;
    float X[3], R[3];
    const float qf = vg->quantum_f, qi = vg->quantum_inv_f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const ff p = ff_add(ff_add(ff_mul(ff_of(vg->Gff[3 * a]), t3[0]), ff_mul(ff_of(vg->Gff[3 * a + 1]), t3[1])),
                          ff_mul(ff_of(vg->Gff[3 * a + 2]), t3[2]));
      // the multiple of the quantum nearest to p.hi + p.lo (scaling by powers of two is exact)
      const float tq = __fmul_rn(p.hi, qi);
      float r = rintf(tq);
      const float d = __fadd_rn(__fsub_rn(tq, r), __fmul_rn(p.lo, qi));
      r = d > 0.5f ? __fadd_rn(r, 1.f) : (d < -0.5f ? __fsub_rn(r, 1.f) : r);
      X[a] = __fmul_rn(r, qf);
      R[a] = __fadd_rn(__fsub_rn(p.hi, X[a]), p.lo);
    }
    pos[kVlRec * (size_t)k] = make_float4(X[0], X[1], X[2], __int_as_float(i));
    res[kVlRec * (size_t)k] = make_float4(R[0], R[1], R[2], __int_as_float(vl_pack3(m[0], m[1], m[2])));
  }
  // largest displacement of the block (positive floats order as their bits)
  for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if ((threadIdx.x & 31) == 0 && dmax > 0.0f) atomicMax(disp, __float_as_uint(dmax));
}

// Forces of the listed pairs (Sec. 5 potential, distance check first): one
// thread per sorted particle, its entries in order; the few candidates within
// float32 rounding of rc are deferred to the float64 fix-up pass with their
// canonical image n + m_j - m_i (RECORD: decided here and recorded).
// Six resident blocks per SM (80 registers): the kernel waits on its gathers,
// and more warps in flight beat the few spilled registers (measured per step
// of the N = 2^20 integrator: 1.26 ms at four blocks, 1.12 at six, 1.34 at
// eight).
#ifndef NEMD_VL_MINBLOCKS
#define NEMD_VL_MINBLOCKS 6
#endif
template <bool RECORD>
__global__ void __launch_bounds__(kVlThreads, NEMD_VL_MINBLOCKS) k_vl_force(
    const Geo *__restrict__ g, const VlGeo *__restrict__ vg, const float4 *__restrict__ pos,
    const float4 *__restrict__ res, const int *__restrict__ cnt, const int2 *__restrict__ ent,
    const int4 *__restrict__ idx, int n, const double *__restrict__ q, Pot pp, float *__restrict__ F,
    double *__restrict__ partials, int32_t *__restrict__ pair_buf, unsigned long long *__restrict__ pair_count,
    long long pair_cap, int4 *__restrict__ rlist, int *__restrict__ rcount, int *__restrict__ err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  Acc acc;
  acc.zero();
  int ncand = 0, nre = 0;
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  if (ok && k < n) {
    const float4 pi = pos[kVlRec * (size_t)k], ri = res[kVlRec * (size_t)k];
    const int oi = __float_as_int(pi.w);
    const float lo = vg->rc2_lo, hi = vg->rc2_hi, lo2 = vg->rc2_lo2, hi2 = vg->rc2_hi2;
    float Gq[9], Gr[9];
    for (int a = 0; a < 9; a++) {
      Gq[a] = vg->Gq[a];
      Gr[a] = vg->Gr[a];
    }
    const int ne = cnt[k];
    ncand = ne;
    constexpr int U = 4;  // entries loaded together (independent gathers in flight)
    for (int e0 = 0; e0 < ne; e0 += U) {
      int2 eu[U];
      float4 pu[U];
#pragma unroll
      for (int h = 0; h < U; h++)
        eu[h] = e0 + h < ne ? __ldcs(&ent[(size_t)(e0 + h) * n + k]) : make_int2(k, 0);
#pragma unroll
      for (int h = 0; h < U; h++) pu[h] = pos[kVlRec * (size_t)eu[h].x];
#pragma unroll
      for (int h = 0; h < U; h++) {
      if (e0 + h >= ne) break;
      const int2 en = eu[h];
      const int j = en.x;
      const float k0 = (float)vl_unpack_k(en.y, 0), k1 = (float)vl_unpack_k(en.y, 1), k2 = (float)vl_unpack_k(en.y, 2);
      const float4 pj = pu[h];
      // quantised part: exact (every term a multiple of the quantum, bounded)
      const float dx = (pj.x - pi.x) + ((Gq[0] * k0 + Gq[1] * k1) + Gq[2] * k2);
      const float dy = (pj.y - pi.y) + ((Gq[3] * k0 + Gq[4] * k1) + Gq[5] * k2);
      const float dz = (pj.z - pi.z) + ((Gq[6] * k0 + Gq[7] * k1) + Gq[8] * k2);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      if (!(r2 < hi)) continue;
      const float4 rj = res[kVlRec * (size_t)j];
      const float cx = dx + ((rj.x - ri.x) + fmaf(Gr[2], k2, fmaf(Gr[1], k1, Gr[0] * k0)));
      const float cy = dy + ((rj.y - ri.y) + fmaf(Gr[5], k2, fmaf(Gr[4], k1, Gr[3] * k0)));
      const float cz = dz + ((rj.z - ri.z) + fmaf(Gr[8], k2, fmaf(Gr[7], k1, Gr[6] * k0)));
      const float r2c = fmaf(cz, cz, fmaf(cy, cy, cx * cx));
      bool accept = r2c < lo2;
      if (!(r2 < lo)) nre++;
      int nn[3] = {0, 0, 0};
      const bool band = !accept && r2c < hi2;
      if (band || RECORD) {
        // the pair's canonical image: n = (k - idx_j + idx_i) / c, plus m_j - m_i
        const int4 ii = idx[k], jj = idx[j];
        nn[0] = (vl_unpack_k(en.y, 0) - jj.x + ii.x) / vg->c[0] + vl_unpack3(__float_as_int(rj.w), 0) -
                vl_unpack3(__float_as_int(ri.w), 0);
        nn[1] = (vl_unpack_k(en.y, 1) - jj.y + ii.y) / vg->c[1] + vl_unpack3(__float_as_int(rj.w), 1) -
                vl_unpack3(__float_as_int(ri.w), 1);
        nn[2] = (vl_unpack_k(en.y, 2) - jj.z + ii.z) / vg->c[2] + vl_unpack3(__float_as_int(rj.w), 2) -
                vl_unpack3(__float_as_int(ri.w), 2);
      }
      if (band) {
        if (RECORD)
          accept = guard_band_accept(g, q, oi, __float_as_int(pj.w), nn[0], nn[1], nn[2]);
        else
          defer_recheck(rlist, rcount, err, k, j, nn[0], nn[1], nn[2]);
      }
      if (!accept) continue;
      acc.add_r2(pp, cx, cy, cz, r2c);
      if (RECORD) record_pair(g, q, oi, __float_as_int(pj.w), nn[0], nn[1], nn[2], pair_buf, pair_count, pair_cap);
      }
    }
    if (F) {
      F[3 * (size_t)oi] = acc.fx;
      F[3 * (size_t)oi + 1] = acc.fy;
      F[3 * (size_t)oi + 2] = acc.fz;
    }
  }
  double v[kPartials] = {acc.u, acc.wxx, acc.wyy, acc.wzz, acc.wxy, acc.wxz, acc.wyz,
                         (double)acc.npair, (double)ncand, (double)nre};
  block_reduce_store<kVlThreads>(v, partials);
}

template <class T>
int vl_grow(nemd_ctx *c, T **p, int64_t count, int64_t *cap) {
  if (*p && *cap >= count) return NEMD_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (cudaMalloc((void **)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1)) != cudaSuccess) {
    cudaGetLastError();
    *cap = 0;
    snprintf(c->msg, sizeof c->msg, "verlet list: out of device memory");
    return NEMD_ERR_NOMEM;
  }
  *cap = count;
  return NEMD_OK;
}

int vl_cuda(nemd_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return NEMD_OK;
  cudaGetLastError();
  snprintf(c->msg, sizeof c->msg, "verlet list %s: %s", what, cudaGetErrorString(e));
  return NEMD_ERR_CUDA;
}

// Per-particle buffers for n particles (the entries are sized at each build).
int vl_reserve(nemd_ctx *c, int64_t n) {
  if (!c->vl_geo) {
    if (cudaMalloc((void **)&c->vl_geo, sizeof(VlGeo)) != cudaSuccess ||
        cudaMalloc((void **)&c->vl_disp, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_vl, 2 * sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      return NEMD_ERR_NOMEM;
    }
  }
  if (c->vl_capn >= n && c->vl_cnt) return NEMD_OK;
  int64_t cap = 0;
  int r;
  if ((r = vl_grow(c, &c->vl_cnt, n, &cap)) || (r = vl_grow(c, &c->vl_slot, n, &cap)) ||
      (r = vl_grow(c, &c->vl_sb, 3 * n, &cap)) || (r = vl_grow(c, &c->vl_idx, n, &cap)) ||
      (r = vl_grow(c, &c->vl_pos, kVlRec * n, &cap)))
    return r;
  c->vl_capn = n;
  return NEMD_OK;
}

}  // namespace

// Smallest eigenvalue of the symmetric 3x3 matrix (A + A^T)/2 (cyclic Jacobi
// rotations; float64, host), at most 0: the slowest contraction rate of the flow.
double flow_contraction_rate(const double *A) {
  double S[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) S[a][b] = 0.5 * (A[3 * a + b] + A[3 * b + a]);
  for (int sweep = 0; sweep < 50; sweep++) {
    const double off = S[0][1] * S[0][1] + S[0][2] * S[0][2] + S[1][2] * S[1][2];
    if (off < 1e-30 * (S[0][0] * S[0][0] + S[1][1] * S[1][1] + S[2][2] * S[2][2]) + 1e-300) break;
    for (int p = 0; p < 2; p++)
      for (int q = p + 1; q < 3; q++) {
        if (S[p][q] == 0.0) continue;
        const double th = 0.5 * (S[q][q] - S[p][p]) / S[p][q];
        const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; k++) {  // columns p, q
          const double kp = S[k][p], kq = S[k][q];
          S[k][p] = c * kp - s * kq;
          S[k][q] = s * kp + c * kq;
        }
        for (int k = 0; k < 3; k++) {  // rows p, q
          const double pk = S[p][k], qk = S[q][k];
          S[p][k] = c * pk - s * qk;
          S[q][k] = s * pk + c * qk;
        }
      }
  }
  return std::min(std::min(std::min(S[0][0], S[1][1]), S[2][2]), 0.0);
}

// Forces (into F) of the state the integrator has set (lattice at time t,
// positions c->q_dev) from the Verlet list, rebuilding it first when needed.
// Synchronises once per call (the displacement check).
int verlet_forces(nemd_ctx *c, float *F, int variant, double rc, double t) {
  const int64_t n = c->n;
  int r = vl_reserve(c, n);
  if (r) return r;
  const double rl = rc + c->vl_skin;
  const int nb = (int)std::max<int64_t>((n + kVlThreads - 1) / kVlThreads, 1);
  // the period the lattice is in: a remap between two calls invalidates the list
  long long period = 0;
  double anorm = 0.0;
  for (int k = 0; k < 9; k++) anorm += c->A[k] * c->A[k];
  anorm = sqrt(anorm);
  if (anorm > 0.0) period = (long long)floor(t / c->T + (c->remap_centered ? 0.5 : 0.0));
  bool rebuild = c->vl_n != n || c->vl_builds == 0 || period != c->vl_period;
  if (!rebuild) {
    k_vl_geo<<<1, 32, 0, c->stream>>>(c->geo, c->vl_geo, rc);
    if ((r = vl_cuda(c, cudaMemsetAsync(c->vl_disp, 0, sizeof(unsigned), c->stream), "memset"))) return r;
    k_vl_pos<<<nb, kVlThreads, 0, c->stream>>>(c->geo, c->vl_geo, c->q_dev, (int)n, c->vl_slot, c->vl_sb, c->vl_idx,
                                               c->vl_pos, c->vl_pos + 1, c->vl_disp);
    if ((r = vl_cuda(c, cudaMemcpyAsync(c->h_vl, c->vl_disp, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream),
                     "copy")))
      return r;
    if ((r = vl_cuda(c, cudaStreamSynchronize(c->stream), "sync"))) return r;
    c->launches += 2;
    float delta;
    memcpy(&delta, c->h_vl, sizeof delta);
    c->vl_delta = delta;
    // a pair outside the list is at least exp(mu (t - t_b)) rl - 2 delta away
    const double sigma = exp(flow_contraction_rate(c->A) * (t - c->vl_tb));
    rebuild = !(sigma * rl - 2.0 * (double)delta >= rc * (1.0 + 1e-9));
  }
  if (rebuild) {
    // the search of the build on cells half as wide (cell factor 2): fewer
    // candidates than at factor 1, same pairs
    const int kf = c->kfac;
    const bool tuned = c->autotuned;
    c->kfac = 2;
    c->autotuned = false;  // the tuned choice is for the force at rc
    r = nemd_build_cells(c, variant, rl);
    c->kfac = kf;
    c->autotuned = tuned;
    if (r) return r;
    k_vl_init<<<nb, kVlThreads, 0, c->stream>>>(c->geo, c->q_dev, c->pos4, (int)n, rl, c->vl_sb, c->vl_idx,
                                                c->vl_slot, c->vl_geo);
    c->launches += 1;
    // fill with the width of the previous list (plus room); if a particle has
    // more entries, fill again with the width the fill measured
    int maxk = c->vl_n == n && c->vl_maxk > 0 ? c->vl_maxk + 16 : 0;
    for (int pass = 0; pass < 2; pass++) {
      if ((r = vl_cuda(c, cudaMemsetAsync(c->vl_disp + 1, 0, sizeof(unsigned), c->stream), "memset"))) return r;
      if (maxk == 0) {
        k_vl_build<true><<<nb, kVlThreads, 0, c->stream>>>(c->geo, c->pos4, c->cell_sorted, c->start, c->rows,
                                                           c->rowcnt, (int)n, c->vl_idx, c->vl_geo, nullptr, nullptr,
                                                           0, c->vl_disp + 1);
      } else {
        if ((r = vl_grow(c, &c->vl_ent, (int64_t)maxk * n, &c->vl_capent))) return r;
        k_vl_build<false><<<nb, kVlThreads, 0, c->stream>>>(c->geo, c->pos4, c->cell_sorted, c->start, c->rows,
                                                            c->rowcnt, (int)n, c->vl_idx, c->vl_geo, c->vl_cnt,
                                                            c->vl_ent, maxk, c->vl_disp + 1);
      }
      c->launches += 1;
      if ((r = vl_cuda(c, cudaMemcpyAsync(c->h_vl + 1, c->vl_disp + 1, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                          c->stream),
                       "copy")))
        return r;
      if ((r = vl_cuda(c, cudaStreamSynchronize(c->stream), "sync"))) return r;
      const int need = (int)c->h_vl[1];
      c->vl_maxk = need;
      if (maxk > 0 && need <= maxk) break;
      maxk = need + 16;
      if (pass == 1) {
        // the count pass ran first: fill now with its width
        if ((r = vl_grow(c, &c->vl_ent, (int64_t)maxk * n, &c->vl_capent))) return r;
        k_vl_build<false><<<nb, kVlThreads, 0, c->stream>>>(c->geo, c->pos4, c->cell_sorted, c->start, c->rows,
                                                            c->rowcnt, (int)n, c->vl_idx, c->vl_geo, c->vl_cnt,
                                                            c->vl_ent, maxk, c->vl_disp + 1);
        c->launches += 1;
      }
    }
    k_vl_geo<<<1, 32, 0, c->stream>>>(c->geo, c->vl_geo, rc);
    if ((r = vl_cuda(c, cudaMemsetAsync(c->vl_disp, 0, sizeof(unsigned), c->stream), "memset"))) return r;
    k_vl_pos<<<nb, kVlThreads, 0, c->stream>>>(c->geo, c->vl_geo, c->q_dev, (int)n, c->vl_slot, c->vl_sb, c->vl_idx,
                                               c->vl_pos, c->vl_pos + 1, c->vl_disp);
    c->launches += 2;
    c->vl_n = n;
    c->vl_tb = t;
    c->vl_period = period;
    c->vl_builds++;
  }
  c->vl_steps++;
  // the force of the listed pairs, then the float64 fix-up and the totals
  if (c->record_cap > 0 &&
      (r = vl_cuda(c, cudaMemsetAsync(c->pair_count, 0, sizeof(unsigned long long), c->stream), "memset")))
    return r;
  if ((r = vl_cuda(c, cudaMemsetAsync(c->nrecheck, 0, sizeof(int), c->stream), "memset"))) return r;
  const Pot pp = make_pot(c);
  if (nb + kFixupBlocks > c->cap_partials) return NEMD_ERR_CAPACITY;
#define NEMD_VL_ARGS                                                                                         \
  c->geo, c->vl_geo, c->vl_pos, c->vl_pos + 1, c->vl_cnt, c->vl_ent, c->vl_idx, (int)n, c->q_dev, pp, F, c->partials, \
      c->pair_buf, c->pair_count, (long long)c->record_cap, c->recheck, c->nrecheck, &c->geo->error
  if (c->record_cap > 0)
    k_vl_force<true><<<nb, kVlThreads, 0, c->stream>>>(NEMD_VL_ARGS);
  else
    k_vl_force<false><<<nb, kVlThreads, 0, c->stream>>>(NEMD_VL_ARGS);
#undef NEMD_VL_ARGS
  c->launches += 1;
  cudaError_t e = launch_recheck_fixup(c, F, c->uw_out, nb, false, true);
  return vl_cuda(c, e, "force");
}

}  // namespace nemd

extern "C" {

int nemd_set_verlet(nemd_ctx *c, double skin) {
  if (!c) return NEMD_ERR_ARG;
  if (!(skin >= 0.0) || !isfinite(skin)) {
    snprintf(c->msg, sizeof c->msg, "verlet skin %g", skin);
    return NEMD_ERR_ARG;
  }
  c->vl_skin = skin;
  c->vl_n = 0;  // the next evaluation builds
  c->vl_builds = 0;
  c->vl_steps = 0;
  return NEMD_OK;
}

int nemd_get_verlet_stats(nemd_ctx *c, int64_t *builds, int64_t *steps, int64_t *width, double *delta) {
  if (!c) return NEMD_ERR_ARG;
  if (builds) *builds = c->vl_builds;
  if (steps) *steps = c->vl_steps;
  if (width) *width = c->vl_maxk;
  if (delta) *delta = c->vl_delta;
  return NEMD_OK;
}

}  // extern "C"
