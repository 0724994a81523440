// force_row.cu -- row kernel (Sec. 3 and 5: only neighbourhood cells are
// searched and the distance check comes before the force; the pair set and
// the pair arithmetic are those of the other kernels).
//
// Binning sorts every cell along kappa, the cell-units coordinate along its
// x-row, so each x-row of cells is one kappa-sorted run of particles.  A warp
// takes a chunk of at most 32 consecutive particles of one x-row, one per lane.
// For each neighbour row of the chunk's (iy, iz) class the warp stages the
// particles of the cells that can hold a partner of some lane in shared
// memory, already moved into the chunk's frame (exact quantised part, float32
// residual, kappa), and then each LANE searches the staged kappa values for
// its own window |kappa_j - kappa_i| <= rho1: two particles farther apart than
// rho1 cells along the row are farther apart than rc.  A lane tests about
// 2 rho1 cells of candidates per row instead of the union of the 32 windows of
// its warp.
//
// The per-lane test is coarse and in half precision: two staged candidates per
// instruction, read as half2 pairs of x, y and z (6 bytes per candidate from
// shared memory).  Its threshold rc2_hi + e_i bounds every rounding of the
// half-precision values for any candidate whose quantised distance is within
// the coarse band, so no partner is lost; a candidate accepted only through
// e_i fails the exact test of the flush.  The results of 32 candidates form one
// accept mask per lane (no dependence between the tests, one store per mask),
// and the accepted slots' forces are computed in flushes, run only when the
// next row would not fit in the stage (or the masks could overflow).  Rows are
// visited in opposite pairs (a lane with many partners in one row has few in
// the opposite one), so the lanes have about equally many accepted slots when
// they are flushed.  Each lane accumulates its particle's force in a fixed
// order: results are deterministic.
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include "batch_internal.cuh"

namespace nemd {

// Shape of the kernel (compile-time): resident blocks of four warps the
// register budget aims at, staged particles per warp, queue entries per lane.
#ifndef NEMD_ROW_MINBLOCKS
#define NEMD_ROW_MINBLOCKS 4
#endif
#ifndef NEMD_ROW_STAGE
#define NEMD_ROW_STAGE 240
#endif
#ifndef NEMD_ROW_WORDS
#define NEMD_ROW_WORDS 12
#endif
#ifndef NEMD_ROW_PASS
#define NEMD_ROW_PASS 2
#endif
constexpr int kRowThreads = 128;
constexpr int kRowMinBlocks = NEMD_ROW_MINBLOCKS;
constexpr int kRowStage = NEMD_ROW_STAGE;  // even
constexpr int kRowWords = NEMD_ROW_WORDS;  // accept masks per lane between two flushes
constexpr int kRowPass = NEMD_ROW_PASS;    // accepted slots a lane loads together in a flush pass
constexpr int kRowRowsStaged = 32;   // rows per class the kernel stages (cell factor <= 2)
constexpr int kRowABias = 64;        // SA[slot] = row | (A + kRowABias) << 5
constexpr int kRowPad = 32;          // half slots past the stage that a lane's last mask may read
static_assert(kRowStage % 2 == 0, "slots are tested in pairs");
static_assert(kRowStage <= 256, "mask bases are one byte");

// Shared memory of one warp.  The half arrays extend kRowPad slots past the
// stage: the tests of a mask read whole slot pairs, and every candidate outside
// the lane's window (stale or never written) is cleared from the mask.
struct RowStage {
  float4 X[kRowStage];   // chunk frame, exact quantised part; .w: kappa
  float4 R[kRowStage];   // residual part; .w: sorted index of j (bits)
  __half hx[kRowStage + kRowPad], hy[kRowStage + kRowPad], hz[kRowStage + kRowPad];
  unsigned short SA[kRowStage];  // row of the slot and its cell offset A from the chunk's first cell
  unsigned mq[kRowWords][32];       // accepted candidates of a lane: bit b is slot mb + b
  unsigned char mb[kRowWords][32];  // first slot of each mask
  float4 rows[kRowRowsStaged][3];
};

constexpr float kHalfSentinel = 65504.0f;  // largest finite half: its square overflows

// Bits k and 16 + k (the low and high candidate of slot pair k) to bits 2k and
// 2k + 1: the outer perfect shuffle of a 32-bit word, four swap steps
// (Warren, Hacker's Delight, Sec. 7-2).
__device__ __forceinline__ unsigned row_shuffle(unsigned x) {
  unsigned t;
  t = (x ^ (x >> 8)) & 0x0000FF00u;
  x ^= t ^ (t << 8);
  t = (x ^ (x >> 4)) & 0x00F000F0u;
  x ^= t ^ (t << 4);
  t = (x ^ (x >> 2)) & 0x0C0C0C0Cu;
  x ^= t ^ (t << 2);
  t = (x ^ (x >> 1)) & 0x22222222u;
  x ^= t ^ (t << 1);
  return x;
}

// Bits [a, e) of a 32-bit word, the bounds clamped to [0, 32].
__device__ __forceinline__ unsigned row_range_bits(int a, int e) {
  a = min(max(a, 0), 32);
  e = min(max(e, 0), 32);
  return (unsigned)(((1ull << e) - 1ull) & ~((1ull << a) - 1ull));
}

// Stencil image (kx, ky, kz) of a staged slot: its row gives (ky, kz) and the
// row's x-shift sxi; its unwrapped x-cell is ixlo + A - sxi.
__device__ __forceinline__ void row_slot_image(const RowStage &S, int slot, int ixlo, int l1, int &kx, int &ky,
                                               int &kz) {
  const int sa = S.SA[slot];
  const float4 s2 = S.rows[sa & 31][2];
  const int kyz = __float_as_int(s2.y);
  kx = floordiv_dev(ixlo + (sa >> 5) - kRowABias - __float_as_int(s2.z), l1);
  ky = (short)(kyz & 0xffff);
  kz = kyz >> 16;
}

// The lane's window [lo, hi) in the staged slots [sb, se): lo the first slot
// with X.w >= klo, hi the first with X.w > khi, found together by halving
// steps whose number depends only on se - sb (the same on every lane).
__device__ __forceinline__ void row_bounds(const RowStage &S, int sb, int se, float klo, float khi, int &lo,
                                           int &hi) {
  lo = sb;
  hi = sb;
  const int n = se - sb;
  for (int step = 1 << (31 - __clz(n)); step > 0; step >>= 1) {
    const bool okl = lo + step <= se, okh = hi + step <= se;
    const float vl = S.X[okl ? lo + step - 1 : sb].w, vh = S.X[okh ? hi + step - 1 : sb].w;
    if (okl && vl < klo) lo += step;
    if (okh && vh <= khi) hi += step;
  }
}

// Cells of one staged row that can hold a partner of a lane with kappa
// position (relative to the chunk's first cell) in [pmin, pmax]: window cells
// u in [ufirst, ulast] (ulast < ufirst: none), the wrapped x-cell jx of the
// first, and ulo = ixlo + dxlo.
struct RowCells {
  int ufirst, ulast, jx, ulo;
};

__device__ __forceinline__ RowCells row_cells(const float4 &s0, const float4 &s1, const float4 &s2, int ixlo,
                                              int ixhi, int l1, float kx0, float ky0, float kz0, float pmin,
                                              float pmax, float reach) {
  const int dxlo = __float_as_int(s1.w);
  const int rcnt = __float_as_int(s2.x), sxi = __float_as_int(s2.z);
  RowCells w;
  w.ulo = ixlo + dxlo;
  const int nu = ixhi - ixlo + rcnt;
  // the row's shift along the row, in cells
  const float sh1 = fmaf(kz0, s0.z + s1.z, fmaf(ky0, s0.y + s1.y, kx0 * (s0.x + s1.x)));
  const float a0 = (float)(dxlo + sxi) + sh1;
  w.ufirst = max(0, (int)ceilf(pmin - reach - a0));
  w.ulast = min(nu - 1, (int)floorf(pmax + reach - a0));
  const int ustart = w.ulo + w.ufirst;
  w.jx = ustart - floordiv_dev(ustart, l1) * l1;
  return w;
}

// Half-precision coarse threshold of a lane at chunk-frame position X_i:
// every candidate with quantised displacement d (|d_a| <= R, R^2 = rc2_hi)
// passes r2_h < thr.  With u = 2^-11 (half precision) each staged and lane
// coordinate rounds by at most u |x| (plus 2^-24 below the normal range), and
// |X_j,a| <= |X_i,a| + R, so the half difference of component a is within
//   e_a = u (2 |X_i,a| + 2 R) + u^2 (2 |X_i,a| + R) + 2^-23
// of d_a; the three half products and sums of r2_h round by at most
// 9 u (1 + u)^2 (R + e_max)^2 in all, and the squares move by at most
// 2 R sum e_a + sum e_a^2.  The bound is computed in float32 with a relative
// allowance of 2^-20 and rounded up to half precision.
__device__ __forceinline__ float row_half_threshold(float rc2_hi, float xi, float yi, float zi) {
  const float u = 4.8828125e-4f;  // 2^-11
  const float R = sqrtf(rc2_hi) * (1.0f + 1e-6f);
  const float ex = u * (2.0f * fabsf(xi) + 2.0f * R) + u * u * (2.0f * fabsf(xi) + R) + 1.2e-7f;
  const float ey = u * (2.0f * fabsf(yi) + 2.0f * R) + u * u * (2.0f * fabsf(yi) + R) + 1.2e-7f;
  const float ez = u * (2.0f * fabsf(zi) + 2.0f * R) + u * u * (2.0f * fabsf(zi) + R) + 1.2e-7f;
  const float em = fmaxf(ex, fmaxf(ey, ez));
  const float sq = (R + em) * (R + em);
  const float margin = 2.0f * R * (ex + ey + ez) + (ex * ex + ey * ey + ez * ez) + 9.0f * u * (1.0f + u) * (1.0f + u) * sq;
  return (rc2_hi + margin) * (1.0f + 9.5367431640625e-7f);
}

// ---- precise mode: energy and virial of accepted pairs in float-float ----
// The displacement of a pair is the exact quantised difference plus the
// difference of the float32 residuals; from it r^2, 1/r^2 (float reciprocal
// refined by one Newton step), (sigma^2/r^2)^3, the pair energy and the
// virial terms are formed in float-float (about 2^-45 relative per
// operation) and summed per particle in float-float; the blocks add the
// particles' sums in float64.  Forces stay float32.
struct PotFF {
  ff eps4, eps24, sig2, ushift;
};

__device__ __forceinline__ ff ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ PotFF make_pot_ff(const Pot &pp) {
  return {ff_from_double(pp.eps4d), ff_from_double(pp.eps24d), ff_from_double(pp.sig2d),
          ff_from_double(pp.ushiftd)};
}

struct AccFF {
  ff u, wxx, wyy, wzz, wxy, wxz, wyz;
  __device__ __forceinline__ void zero() {
    u = wxx = wyy = wzz = wxy = wxz = wyz = ff{0.f, 0.f};
  }
};

// d_a = h_a + l_a: h the exact quantised difference, l the residuals' difference.
// Returns the force on j (fr d, rounded once to float32); the force on i is its negative.
__device__ __forceinline__ float3 pair_ff(const PotFF &pf, float hx, float lx, float hy, float ly, float hz,
                                          float lz, AccFF &a) {
  const ff dx = ff_add(ff{hx, 0.f}, ff{lx, 0.f});
  const ff dy = ff_add(ff{hy, 0.f}, ff{ly, 0.f});
  const ff dz = ff_add(ff{hz, 0.f}, ff{lz, 0.f});
  const ff r2 = ff_add(ff_add(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz));
  const float x0 = __frcp_rn(r2.hi);
  const ff e = ff_add(ff{1.f, 0.f}, ff_neg(ff_mul_f(r2, x0)));
  const ff inv = ff_add(ff{x0, 0.f}, ff_mul_f(e, x0));
  const ff s2 = ff_mul(pf.sig2, inv);
  const ff s6 = ff_mul(ff_mul(s2, s2), s2);
  const ff u = ff_add(ff_mul(ff_mul(pf.eps4, s6), ff_add(s6, ff{-1.f, 0.f})), ff_neg(pf.ushift));
  const ff fr = ff_mul(ff_mul(ff_mul(pf.eps24, inv), s6), ff_add(ff_mul_f(s6, 2.f), ff{-1.f, 0.f}));
  const ff gx = ff_mul(fr, dx), gy = ff_mul(fr, dy), gz = ff_mul(fr, dz);
  a.u = ff_add(a.u, u);
  a.wxx = ff_add(a.wxx, ff_mul(gx, dx));
  a.wyy = ff_add(a.wyy, ff_mul(gy, dy));
  a.wzz = ff_add(a.wzz, ff_mul(gz, dz));
  a.wxy = ff_add(a.wxy, ff_mul(gx, dy));
  a.wxz = ff_add(a.wxz, ff_mul(gx, dz));
  a.wyz = ff_add(a.wyz, ff_mul(gy, dz));
  return make_float3(__fadd_rn(gx.hi, gx.lo), __fadd_rn(gy.hi, gy.lo), __fadd_rn(gz.hi, gz.lo));
}

// The next accepted slot of a lane: the highest set bit of its current mask,
// the next stored mask once that one is used up (qn counts what is left).
__device__ __forceinline__ int row_next_slot(const RowStage &S, int lane, unsigned &cur, int &base, int &wi) {
  if (cur == 0) {
    cur = S.mq[wi][lane];
    base = S.mb[wi][lane];
    wi++;
  }
  const int b = 31 - __clz(cur);
  cur ^= 1u << b;
  return base + b;
}

// Forces of the accepted slots of every lane (Sec. 5 potential): each is
// decided with the residuals added back; the few within float32 rounding of
// rc go to the float64 fix-up pass (RECORD: decided here in float64) and are
// counted in nre.  Fast mode sums the pair terms without the potential's
// constant factors (Acc::add_unscaled).
template <bool RECORD, bool PRECISE>
__device__ __forceinline__ void row_flush(RowStage &S, int &qn, int &nw, int &nre, int lane, int ki,
                                          const float4 &pi, const float3 &Xi, const float3 &Ri, int ixlo,
                                          const Geo *g, const float4 *__restrict__ pos, const Pot &pp,
                                          const PotFF &pf, Acc &acc, AccFF &accp, const double *q,
                                          int32_t *pair_buf, unsigned long long *pair_count, long long pair_cap,
                                          int4 *rlist, int *rcount, int *err) {
  const int m = __reduce_max_sync(0xffffffffu, qn);
  const float lo2 = g->rc2_lo2, hi2 = g->rc2_hi2;
  unsigned cur = 0;
  int base = 0, wi = 0;
  // kRowPass entries per pass, all loaded before any is used (independent
  // chains for the scheduler); each is decided and added on its own
  for (int s = 0; s < m; s += kRowPass) {
    bool vv[kRowPass];
    int sl[kRowPass];
    float4 XX[kRowPass], RR[kRowPass];
#pragma unroll
    for (int h = 0; h < kRowPass; h++) {
      vv[h] = s + h < qn;
      sl[h] = vv[h] ? row_next_slot(S, lane, cur, base, wi) : 0;
    }
#pragma unroll
    for (int h = 0; h < kRowPass; h++) {
      XX[h] = S.X[sl[h]];
      RR[h] = S.R[sl[h]];
    }
#pragma unroll
    for (int h = 0; h < kRowPass; h++) {
      if (!vv[h]) continue;
      const int slot = sl[h];
      const float4 X = XX[h], R = RR[h];
      const int j = __float_as_int(R.w);
      const float cx = (X.x - Xi.x) + (R.x - Ri.x);
      const float cy = (X.y - Xi.y) + (R.y - Ri.y);
      const float cz = (X.z - Xi.z) + (R.z - Ri.z);
      const float r2c = fmaf(cz, cz, fmaf(cy, cy, cx * cx));
      bool accept = r2c < lo2;
      if (!accept && r2c < hi2) {
        int kx, ky, kz;
        row_slot_image(S, slot, ixlo, g->nc[0], kx, ky, kz);
        nre++;
        if (RECORD)
          accept = guard_band_accept(g, q, __float_as_int(pi.w), __float_as_int(pos[j].w), kx, ky, kz);
        else
          defer_recheck(rlist, rcount, err, ki, j, kx, ky, kz);  // decided by the fix-up pass
      }
      // the particle itself: the same sorted index at exactly zero distance
      if (accept && !(j == ki && r2c == 0.f)) {
        if (PRECISE) {
          const float3 gj = pair_ff(pf, X.x - Xi.x, R.x - Ri.x, X.y - Xi.y, R.y - Ri.y, X.z - Xi.z, R.z - Ri.z, accp);
          acc.fx -= gj.x;
          acc.fy -= gj.y;
          acc.fz -= gj.z;
          acc.npair++;
        } else {
          acc.add_unscaled(pp.sig2, cx, cy, cz, r2c);
        }
        if (RECORD) {
          int kx, ky, kz;
          row_slot_image(S, slot, ixlo, g->nc[0], kx, ky, kz);
          record_pair(g, q, __float_as_int(pi.w), __float_as_int(pos[j].w), kx, ky, kz, pair_buf, pair_count,
                      pair_cap);
        }
      }
    }
  }
  qn = 0;
  nw = 0;
}

// Everything one warp does for one chunk cd (x: first sorted particle, y:
// count, z: class, w: ixlo | ixhi << 16): the rows of the chunk's class (crow,
// nr of them) are visited in opposite pairs (0, nr-1, 1, nr-2, ...); per row
// the cells within reach of some lane are staged, each lane tests its own
// kappa window, and the queues are flushed when the stage is full.  On return
// acc.fx, fy, fz hold the force on the lane's particle pi (sorted index ki;
// act is false for lanes past the chunk's count) in the variant's frame, and
// its pair sums have been added to acc.  cell_base is the system's first cell
// slot (0 for a single system).
template <bool RECORD, bool PRECISE>
__device__ __forceinline__ void row_chunk(const int4 cd, const Row *__restrict__ crow, int nr, int cell_base,
                                          const Geo *g, const float4 *__restrict__ pos,
                                          const float4 *__restrict__ posr, const int *__restrict__ cell_sorted,
                                          const int *__restrict__ start, RowStage &S, const Pot &pp,
                                          const PotFF &pf, const double *q, Acc &acc, AccFF &accp, int &ncand,
                                          int &nre, bool &act, float4 &pi,
                                          int &ki, int32_t *pair_buf, unsigned long long *pair_count,
                                          long long pair_cap, int4 *rlist, int *rcount, int *err) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int l1 = g->nc[0];
  const float sx = g->step[0], sy = g->step[1], sz = g->step[2];
  const float srx = g->step_r[0], sry = g->step_r[1], srz = g->step_r[2];
  const float kx0 = g->kap[0], ky0 = g->kap[1], kz0 = g->kap[2];
  act = lane < cd.y;
  ki = act ? cd.x + lane : cd.x;  // inactive lanes shadow a valid particle
  pi = pos[ki];
  const float4 pir = posr[ki];
  const int ixlo = cd.w & 0xffff, ixhi = cd.w >> 16;
  // positions are taken relative to the chunk's middle cell (smaller values for
  // the half-precision test); kappa and A relative to its first cell
  const int cofs = (ixhi - ixlo) >> 1;
  const int ixu = (cell_sorted[ki] - cell_base) % l1;
  const int ai = ixu - ixlo;
  const float ac = (float)(ai - cofs);
  const float3 Xi = make_float3(fmaf(ac, sx, pi.x), fmaf(ac, sy, pi.y), fmaf(ac, sz, pi.z));
  const float3 Ri = make_float3(fmaf(ac, srx, pir.x), fmaf(ac, sry, pir.y), fmaf(ac, srz, pir.z));
  const float kapi = pir.w + (float)ai;  // kappa of the lane's particle
  const __half2 xi2 = __float2half2_rn(Xi.x), yi2 = __float2half2_rn(Xi.y), zi2 = __float2half2_rn(Xi.z);
  const __half2 thr2 = __half2half2(act ? __float2half_ru(row_half_threshold(g->rc2_hi, Xi.x, Xi.y, Xi.z))
                                           : __float2half_rn(-kHalfSentinel));
  const float rho = g->rho1 + 1e-4f;
  if (nr > kRowRowsStaged) {
    // more rows than the stage holds (cell factor > 2): refused as a capacity error
    if (lane == 0) atomicOr(err, ERRB_CAPACITY);
    nr = kRowRowsStaged;
  }
  {
    const float4 *src = reinterpret_cast<const float4 *>(crow);
    __syncwarp();
    for (int e = lane; e < 3 * nr; e += 32) S.rows[e / 3][e % 3] = src[e];
    __syncwarp();
  }
  acc.fx = acc.fy = acc.fz = 0.f;
  int qn = 0, nw = 0, fill = 0;  // accepted slots and stored masks of the lane; staged slots
  // extent of the lanes along the row (cells from the chunk's first cell)
  float pmin = act ? kapi : 1e30f, pmax = act ? kapi : -1e30f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pmin = fminf(pmin, __shfl_xor_sync(FULL, pmin, o));
    pmax = fmaxf(pmax, __shfl_xor_sync(FULL, pmax, o));
  }
  const float reach = g->rho1 + 0.5f + 1e-4f;
  // lane r looks up the particle ranges of the first two runs of row r
  int rb0 = 0, re0 = 0, rb1 = 0, re1 = 0, rcnt = 0;
  if (lane < nr) {
    const float4 s0 = S.rows[lane][0], s1 = S.rows[lane][1], s2 = S.rows[lane][2];
    const RowCells w = row_cells(s0, s1, s2, ixlo, ixhi, l1, kx0, ky0, kz0, pmin, pmax, reach);
    const int cbase = __float_as_int(s0.w);
    if (w.ufirst <= w.ulast) {
      const int len0 = min(w.ulast + 1 - w.ufirst, l1 - w.jx);
      rb0 = start[cbase + w.jx];
      re0 = start[cbase + w.jx + len0];
      const int rest = w.ulast + 1 - w.ufirst - len0;
      if (rest > 0) {
        rb1 = start[cbase];
        re1 = start[cbase + min(rest, l1)];
      }
      // staged slots of the row; a row of more than two runs counts as the
      // whole stage
      rcnt = rest > l1 ? kRowStage : (re0 - rb0) + (re1 - rb1);
    }
  }

  // Per-lane window test of the staged slots [sb, se) of one row: binary
  // searches for the lane's kappa window [lo, hi), then slot pairs in half
  // precision from an even start m0, 32 candidates per accept mask.  Every lane
  // reads np pairs (the warp's longest window), from its own window or, where
  // that would run past the row, from the row's last np pairs: the reads stay
  // within the stage and its padding, and the mask keeps [lo, hi) only.
  auto test_range = [&](int sb, int se) {
    if (se <= sb) return;
    __syncwarp();
    int lo, hi;
    row_bounds(S, sb, se, kapi - rho, kapi + rho, lo, hi);
    if (!act || hi < lo) hi = lo;
    ncand += hi - lo;
    const int m0e = lo & ~1;
    const int np = (__reduce_max_sync(FULL, hi > lo ? hi - m0e : 0) + 1) >> 1;
    const int m0 = min(m0e, ((se + 1) & ~1) - 2 * np);
    const __half2 *hx2 = reinterpret_cast<const __half2 *>(S.hx + m0);
    const __half2 *hy2 = reinterpret_cast<const __half2 *>(S.hy + m0);
    const __half2 *hz2 = reinterpret_cast<const __half2 *>(S.hz + m0);
    for (int w0 = 0; w0 < np; w0 += 16) {
      if (__any_sync(FULL, nw == kRowWords))
        row_flush<RECORD, PRECISE>(S, qn, nw, nre, lane, ki, pi, Xi, Ri, ixlo, g, pos, pp, pf, acc, accp, q,
                                   pair_buf, pair_count, pair_cap, rlist, rcount, err);
      const int pend = min(16, np - w0);
      unsigned msk = 0;
      for (int k0 = 0; k0 < pend; k0 += 4) {
        unsigned m4 = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int p = w0 + k0 + k;
          const __half2 dx = __hsub2(hx2[p], xi2), dy = __hsub2(hy2[p], yi2), dz = __hsub2(hz2[p], zi2);
          const __half2 r2 = __hfma2(dx, dx, __hfma2(dy, dy, __hmul2(dz, dz)));
          // 0xffff in each half whose r2 is below the threshold (false for NaN)
          m4 |= __hlt2_mask(r2, thr2) & (0x00010001u << k);
        }
        msk |= m4 << k0;
      }
      const int base = m0 + 2 * w0;
      msk = row_shuffle(msk) & row_range_bits(lo - base, hi - base);
      if (msk) {
        S.mq[nw][lane] = msk;
        S.mb[nw][lane] = (unsigned char)base;
        nw++;
        qn += __popc(msk);
      }
    }
  };

  for (int t = 0; t < nr; t++) {
    const int r = (t & 1) ? nr - 1 - (t >> 1) : (t >> 1);
    const float4 s0 = S.rows[r][0], s1 = S.rows[r][1], s2 = S.rows[r][2];
    const int pb0 = __shfl_sync(FULL, rb0, r), pe0 = __shfl_sync(FULL, re0, r);
    const int pb1 = __shfl_sync(FULL, rb1, r), pe1 = __shfl_sync(FULL, re1, r);
    if (fill > 0 && fill + __shfl_sync(FULL, rcnt, r) > kRowStage) {
      // the row does not fit behind the rows staged so far: their queued pairs
      // first (flushes cover as many rows as the stage holds)
      row_flush<RECORD, PRECISE>(S, qn, nw, nre, lane, ki, pi, Xi, Ri, ixlo, g, pos, pp, pf, acc, accp, q,
                                 pair_buf, pair_count, pair_cap, rlist, rcount, err);
      fill = 0;
    }
    const int cbase = __float_as_int(s0.w), dxlo = __float_as_int(s1.w);
    const int sxi = __float_as_int(s2.z);
    const float kr = fmaf(kz0, s0.z, fmaf(ky0, s0.y, kx0 * s0.x));  // the row's shift along the row
    const RowCells w = row_cells(s0, s1, s2, ixlo, ixhi, l1, kx0, ky0, kz0, pmin, pmax, reach);
    int jx = w.jx;
    int sb = fill;
    // runs of consecutive cells without an x-wrap: contiguous particles
    for (int u = w.ufirst, run = 0; u <= w.ulast; run++) {
      const int len = min(w.ulast + 1 - u, l1 - jx);
      const int b = run == 0 ? pb0 : (run == 1 ? pb1 : start[cbase + jx]);
      const int e = run == 0 ? pe0 : (run == 1 ? pe1 : start[cbase + jx + len]);
      const int arun = dxlo + sxi + u - jx;  // A of a particle of cell jx' of this run: arun + jx'
      for (int p = b; p < e;) {
        if (fill == kRowStage) {
          // the stage is full: test what this row has in it, then start over
          test_range(sb, fill);
          row_flush<RECORD, PRECISE>(S, qn, nw, nre, lane, ki, pi, Xi, Ri, ixlo, g, pos, pp, pf, acc, accp, q,
                                     pair_buf, pair_count, pair_cap, rlist, rcount, err);
          fill = 0;
          sb = 0;
        }
        const int take = min(e - p, kRowStage - fill);
        __syncwarp();  // slots about to be overwritten are no longer read
        // two particles per lane per pass, both loaded before either is stored
        for (int t0 = lane; t0 < take; t0 += 64) {
          const bool two = t0 + 32 < take;
          const int j0 = p + t0, j1 = two ? j0 + 32 : j0;
          const float4 pj0 = pos[j0], pjr0 = posr[j0];
          const int c0 = cell_sorted[j0];
          const float4 pj1 = pos[j1], pjr1 = posr[j1];
          const int c1 = cell_sorted[j1];
#pragma unroll
          for (int h = 0; h < 2; h++) {
            if (h == 1 && !two) break;
            const int j = h ? j1 : j0;
            const float4 pj = h ? pj1 : pj0, pjr = h ? pjr1 : pjr0;
            const int A = arun + ((h ? c1 : c0) - cbase);
            const float Ac = (float)(A - cofs);
            const float xx = fmaf(Ac, sx, pj.x + s0.x), xy = fmaf(Ac, sy, pj.y + s0.y),
                        xz = fmaf(Ac, sz, pj.z + s0.z);
            const int slot = fill + t0 + 32 * h;
            S.X[slot] = make_float4(xx, xy, xz, (pjr.w + (float)A) + kr);
            S.R[slot] = make_float4(fmaf(Ac, srx, pjr.x + s1.x), fmaf(Ac, sry, pjr.y + s1.y),
                                    fmaf(Ac, srz, pjr.z + s1.z), __int_as_float(j));
            S.SA[slot] = (unsigned short)(r | ((A + kRowABias) << 5));
            S.hx[slot] = __float2half_rn(xx);
            S.hy[slot] = __float2half_rn(xy);
            S.hz[slot] = __float2half_rn(xz);
          }
        }
        fill += take;
        p += take;
      }
      u += len;
      jx += len;
      if (jx == l1) jx = 0;
    }
    test_range(sb, fill);
  }
  row_flush<RECORD, PRECISE>(S, qn, nw, nre, lane, ki, pi, Xi, Ri, ixlo, g, pos, pp, pf, acc, accp, q, pair_buf,
                             pair_count, pair_cap, rlist, rcount, err);
}

// F (Cartesian) of a lane's particle from its frame force: F = Q (fs F_frame),
// fs = 24 eps for the unscaled sums of fast mode, 1 in precise mode.
__device__ __forceinline__ void row_store_force(float *F, const Geo *g, const float4 &pi, const Acc &acc,
                                                float fs) {
  const float *Qm = g->Qf;
  const int oi = __float_as_int(pi.w);
  const float fx = fs * acc.fx, fy = fs * acc.fy, fz = fs * acc.fz;
  F[3 * (size_t)oi] = Qm[0] * fx + Qm[1] * fy + Qm[2] * fz;
  F[3 * (size_t)oi + 1] = Qm[3] * fx + Qm[4] * fy + Qm[5] * fz;
  F[3 * (size_t)oi + 2] = Qm[6] * fx + Qm[7] * fy + Qm[8] * fz;
}

template <bool RECORD, bool PRECISE>
__global__ void __launch_bounds__(kRowThreads, kRowMinBlocks) k_force_row(
    const Geo *__restrict__ g, const float4 *__restrict__ pos, const float4 *__restrict__ posr,
    const int *__restrict__ cell_sorted, const int *__restrict__ start, const Row *__restrict__ rows,
    const int *__restrict__ rowcnt, const int4 *__restrict__ chunks, const int *__restrict__ nchunks_p,
    const double *__restrict__ q, Pot pp, float *__restrict__ F, double *__restrict__ partials,
    int32_t *__restrict__ pair_buf, unsigned long long *__restrict__ pair_count, long long pair_cap,
    int4 *__restrict__ rlist, int *__restrict__ rcount, int *__restrict__ err) {
  constexpr int kWarps = kRowThreads / 32;
  __shared__ RowStage stage[kWarps];
  const int warp = threadIdx.x >> 5;
  Acc acc;  // U, W and the pair count accumulate over every particle this lane owns
  acc.zero();
  AccFF accp;  // precise mode: U and W in float-float
  accp.zero();
  const PotFF pf = make_pot_ff(pp);
  int ncand = 0, nre = 0;
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  const int nch = ok ? *nchunks_p : 0;
  const int maxrows = g->maxrows;
  for (int ch = blockIdx.x * kWarps + warp; ch < nch; ch += gridDim.x * kWarps) {
    const int4 cd = chunks[ch];
    bool act;
    float4 pi;
    int ki;
    row_chunk<RECORD, PRECISE>(cd, rows + (size_t)cd.z * maxrows, rowcnt[cd.z], 0, g, pos, posr, cell_sorted,
                               start, stage[warp], pp, pf, q, acc, accp, ncand, nre, act, pi, ki, pair_buf,
                               pair_count, pair_cap, rlist, rcount, err);
    if (act && F) row_store_force(F, g, pi, acc, PRECISE ? 1.0f : pp.eps24);
  }
  // fast mode: U = 4 eps sum s6 (s6 - 1) - (pairs) shift, W = 24 eps sum fr d d
  const double e4 = pp.eps4d, e24 = pp.eps24d;
  double v[kPartials] = {e4 * acc.u - pp.ushiftd * (double)acc.npair,
                         e24 * acc.wxx, e24 * acc.wyy, e24 * acc.wzz, e24 * acc.wxy, e24 * acc.wxz, e24 * acc.wyz,
                         (double)acc.npair, (double)ncand, (double)nre};
  if (PRECISE) {
    const ff *w[7] = {&accp.u, &accp.wxx, &accp.wyy, &accp.wzz, &accp.wxy, &accp.wxz, &accp.wyz};
    for (int k = 0; k < 7; k++) v[k] = (double)w[k]->hi + (double)w[k]->lo;
  }
  block_reduce_store<kRowThreads>(v, partials);
}

template <bool RECORD, bool PRECISE>
static int row_resident_blocks(int sms) {
  static int per_sm = 0;
  if (!per_sm) {
    cudaFuncSetAttribute(k_force_row<RECORD, PRECISE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_row<RECORD, PRECISE>, kRowThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  return per_sm * sms;
}

bool row_kernel_applies(const nemd_ctx *c) { return c->kfac <= 2; }

// The row kernel over the chunk list of the current step (32 particles per
// chunk); *nblocks receives the number of blocks whose partials it wrote.
cudaError_t launch_force_row(nemd_ctx *c, float *F, int *nblocks) {
  const Pot pp = make_pot(c);
  const bool rec = c->record_cap > 0, pre = c->precise != 0;
  int blocks = rec ? (pre ? row_resident_blocks<true, true>(c->sms) : row_resident_blocks<true, false>(c->sms))
                   : (pre ? row_resident_blocks<false, true>(c->sms) : row_resident_blocks<false, false>(c->sms));
  // a small system needs fewer blocks than the resident limit (one per 64
  // particles; the warps stride over the chunks either way), and the fix-up
  // then sums fewer partial rows
  const int64_t by_n = (c->n + 63) / 64;
  if ((int64_t)blocks > by_n) blocks = (int)std::max<int64_t>(by_n, 1);
  if (blocks > (int)(c->cap_partials - 1)) blocks = (int)(c->cap_partials - 1);
  *nblocks = blocks;
#define NEMD_ARGS                                                                                            \
  c->geo, c->pos4, c->posr, c->cell_sorted, c->start, c->rows, c->rowcnt, c->chunks, c->chunk_off + c->cap_cells, \
      c->q_dev, pp, F, c->partials, c->pair_buf, c->pair_count, (long long)c->record_cap, c->recheck, c->nrecheck, \
      &c->geo->error
  if (rec && pre)
    k_force_row<true, true><<<blocks, kRowThreads, 0, c->stream>>>(NEMD_ARGS);
  else if (rec)
    k_force_row<true, false><<<blocks, kRowThreads, 0, c->stream>>>(NEMD_ARGS);
  else if (pre)
    k_force_row<false, true><<<blocks, kRowThreads, 0, c->stream>>>(NEMD_ARGS);
  else
    k_force_row<false, false><<<blocks, kRowThreads, 0, c->stream>>>(NEMD_ARGS);
#undef NEMD_ARGS
  c->launches += 1;
  return cudaGetLastError();
}

// ---- batches: one persistent launch over every chunk of every system ----
// Warps take chunks from a shared counter (chunks of different systems differ
// widely in cost).  Each lane writes its particle's force and its particle's
// own pair sums (float32, per sorted particle); the per-system reduction adds
// those in float64 in a fixed order, so no result depends on which warp took
// which chunk.
__global__ void __launch_bounds__(kRowThreads, kRowMinBlocks) k_b_force_row(BatchView v) {
  constexpr int kWarps = kRowThreads / 32;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ RowStage stage[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nch = v.chunk_off[v.nclasses];
  // lane 0 claims the warp's next chunk while the current one is evaluated, so
  // the counter's round trip overlaps useful work
  int nxt = 0;
  if (lane == 0) nxt = atomicAdd(v.work, 1);
  for (;;) {
    const int ch = __shfl_sync(FULL, nxt, 0);
    if (ch >= nch) break;
    if (lane == 0) nxt = atomicAdd(v.work, 1);
    const int4 cd = v.chunks[ch];
    const int s = v.class_sys[cd.z];
    Geo *g = v.geo + s;
    const int coff = v.sys[s].coff;
    const Pot pp = v.pot[s];
    const PotFF pf = make_pot_ff(pp);
    Acc acc;
    acc.zero();
    AccFF accp;
    accp.zero();
    int ncand = 0, nre = 0;
    bool act;
    float4 pi;
    int ki;
    row_chunk<false, false>(cd, v.rows + (size_t)cd.z * kBatchRowStride, v.rowcnt[cd.z], coff, g, v.pos4, v.posr,
                            v.cell_sorted, v.start, stage[warp], pp, pf, v.q, acc, accp, ncand, nre, act, pi, ki,
                            nullptr, nullptr, 0, v.recheck, v.nrecheck, &g->error);
    if (act) {
      if (v.F) row_store_force(v.F, g, pi, acc, pp.eps24);
      // the particle's own sums with the potential's constant factors applied
      const float u = fmaf(pp.eps4, acc.u, -pp.ushift * (float)acc.npair);
      v.ppart[2 * (size_t)ki] = make_float4(u, pp.eps24 * acc.wxx, pp.eps24 * acc.wyy, pp.eps24 * acc.wzz);
      v.ppart[2 * (size_t)ki + 1] =
          make_float4(pp.eps24 * acc.wxy, pp.eps24 * acc.wxz, pp.eps24 * acc.wyz, __int_as_float(acc.npair));
    }
    const unsigned c = __reduce_add_sync(FULL, (unsigned)ncand), r = __reduce_add_sync(FULL, (unsigned)nre);
    if (lane == 0) {
      atomicAdd(&v.sys_counters[2 * s], (unsigned long long)c);
      if (r) atomicAdd(&v.sys_counters[2 * s + 1], (unsigned long long)r);
    }
  }
}

int batch_row_blocks(int sms) {
  static int per_sm = 0;
  if (!per_sm) {
    cudaFuncSetAttribute(k_b_force_row, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_force_row, kRowThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  return per_sm * sms;
}

cudaError_t launch_batch_force_row(cudaStream_t st, const BatchView &v, int blocks) {
  cudaError_t e = cudaMemsetAsync(v.work, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.nrecheck, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.sys_counters, 0, 2 * sizeof(unsigned long long) * (size_t)v.nsys, st);
  if (e != cudaSuccess) return e;
  k_b_force_row<<<blocks, kRowThreads, 0, st>>>(v);
  return cudaGetLastError();
}

}  // namespace nemd
