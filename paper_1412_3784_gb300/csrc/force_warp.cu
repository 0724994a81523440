// force_warp.cu -- warp force kernel (Sec. 3 and 5: neighbourhood cells only,
// distance check before force; same pair set and pair arithmetic as the other
// kernels).
//
// A warp takes a chunk of at most 32 consecutive particles of one x-row of
// cells, one particle per lane, and walks the neighbour rows of the chunk's
// (iy, iz) class.  For each row, the particles of the union of the lanes'
// x-windows are staged in shared memory already moved into the chunk's frame:
// a particle j of a cell A cells from the chunk's first cell is staged as
//     X_j = x_j + shift + A step        exact (multiples of the quantum)
//     R_j = r_j + shift_r + A step_r    float32 residual part
// and lane i holds X_i = x_i + a_i step, R_i = r_i + a_i step_r, a_i being its
// own cell's distance from the chunk's first cell.  Then X_j - X_i is exactly
// the quantised displacement the other kernels form, and (X_j - X_i) + (R_j - R_i)
// the displacement with the residuals added back.
//
// Test loop: every bound is uniform across the warp, staged X_j are read as
// shared-memory broadcasts, and a lane writes the slot of every tested
// candidate to its queue unconditionally, advancing only when the coarse test
// passes, so accepting costs no branch.  Flush: queued pairs are decided with
// the residuals added back (the float64 fix-up pass takes the few within float32
// rounding of rc) and their forces computed -- all from shared memory.  A flush
// runs when the stage is full, when a queue could overflow, and at the end of
// the chunk; each lane accumulates its particle's force in queue order, so
// results are deterministic.
#include <math.h>

#include <type_traits>

#include "batch_internal.cuh"

namespace nemd {

// Shape of the kernel (compile-time): threads per block, staged particles per
// warp, queue entries per lane, resident blocks the register allocation aims
// at.  Measured on GB300 (N = 2^20 general flow): five blocks of four warps per
// SM (96 registers, 45 KB of shared memory per block) beat 256 particles at
// four blocks by 16 %; within the same shared memory, 208 staged particles and
// an 80-entry queue beat 224 and 64 by 5.5 % (fewer, fuller flushes), while
// queues of 96-128 entries with 192-160 staged particles are slower again.
#ifndef NEMD_WARP_THREADS
#define NEMD_WARP_THREADS 128
#endif
#ifndef NEMD_WARP_STAGE
#define NEMD_WARP_STAGE 208
#endif
#ifndef NEMD_WARP_QUEUE
#define NEMD_WARP_QUEUE 80
#endif
#ifndef NEMD_WARP_MINBLOCKS
#define NEMD_WARP_MINBLOCKS 5
#endif
constexpr int kWarpThreads = NEMD_WARP_THREADS;
constexpr int kRowsStaged = 32;    // rows per class the kernel stages (cell factor <= 2)
constexpr int kWarpQueue = NEMD_WARP_QUEUE;  // queue entries per lane
constexpr int kTestBlock = 32;     // candidates tested between two queue checks
constexpr int kABias = 64;          // SA[slot] = row | (A + kABias) << 5, 0 <= A + kABias < 2^10
static_assert(kWarpQueue >= 2 * kTestBlock, "a queue check must leave room for a test block");

// Shared memory of one warp.  HALF (half neighbourhoods) also accumulates the
// force on every staged partner (Fj), and stages fewer particles so that four
// blocks still fit an SM.  A queue entry is a slot index: one byte for up to
// 256 slots, two beyond.
template <bool HALF>
struct WarpStageT {
  static constexpr int kSlots = HALF ? 192 : NEMD_WARP_STAGE;
  using Entry = typename std::conditional<(kSlots > 256), unsigned short, unsigned char>::type;
  float4 X[kSlots];  // .w: |X_j|^2
  float4 R[kSlots];  // .w: sorted index of j (bits)
  float Fj[HALF ? 3 : 1][HALF ? kSlots : 1];
  Entry q[kWarpQueue][32];
  float4 rows[kRowsStaged][3];
  unsigned short SA[kSlots];  // row of the slot and its cell offset A from the chunk's first cell
};
using WarpStage = WarpStageT<false>;

// Shared-memory reduction without a returned value.
__device__ __forceinline__ void red_shared_add(float *p, float v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// Stencil image (kx, ky, kz) of a staged slot: its row gives (ky, kz) and the
// row's x-shift sxi; its unwrapped x-cell is ixlo + A - sxi.
template <bool HALF>
__device__ __forceinline__ void slot_image(const WarpStageT<HALF> &S, int slot, int ixlo, int l1, int &kx, int &ky,
                                           int &kz) {
  const int sa = S.SA[slot];
  const float4 s2 = S.rows[sa & 31][2];
  const int kyz = __float_as_int(s2.y);
  kx = floordiv_dev(ixlo + (sa >> 5) - kABias - __float_as_int(s2.z), l1);
  ky = (short)(kyz & 0xffff);
  kz = kyz >> 16;
}

// Forces of the queued pairs of every lane.  HALF: entries of the home row
// (row rhome) count only towards partners ahead of the lane's particle --
// a larger unwrapped x-cell, or the same cell and a larger sorted index --
// and each accepted pair also adds its force to the partner's slot.
template <bool RECORD, bool HALF>
__device__ __forceinline__ void warp_flush(WarpStageT<HALF> &S, int &qn, int &nre, int lane, int ki,
                                           const float4 &pi, const float3 &Xi, const float3 &Ri, int ixu, int ixlo,
                                           int rhome,
                                           const Geo *g, const float4 *__restrict__ pos, const Pot &pp, Acc &acc,
                                           const double *q, int32_t *pair_buf, unsigned long long *pair_count,
                                           long long pair_cap, int4 *rlist, int *rcount, int *err) {
  const int m = __reduce_max_sync(0xffffffffu, qn);
  const float lo = g->rc2_lo, lo2 = g->rc2_lo2, hi2 = g->rc2_hi2;
  // HALF: lanes start at different points of their queues, so that one step of
  // the flush rarely adds to the same partner slot from several lanes
  int e = HALF && qn > 0 ? (7 * lane) % qn : 0;
  for (int s = 0; s < m; s++) {
    if (s < qn) {
      const int slot = S.q[HALF ? e : s][lane];
      if (HALF && ++e == qn) e = 0;
      const float4 X = S.X[slot], R = S.R[slot];
      const int j = __float_as_int(R.w);
      if (HALF) {
        const int sa = S.SA[slot];
        if ((sa & 31) == rhome) {
          // the home row has no x-shift: unwrapped x-cell = ixlo + A
          const int jxu = ixlo + (sa >> 5) - kABias;
          if (!(jxu > ixu || (jxu == ixu && j > ki))) continue;
        }
      }
      const float cx = (X.x - Xi.x) + (R.x - Ri.x);
      const float cy = (X.y - Xi.y) + (R.y - Ri.y);
      const float cz = (X.z - Xi.z) + (R.z - Ri.z);
      const float r2c = fmaf(cz, cz, fmaf(cy, cy, cx * cx));
      bool accept = r2c < lo2;
      if (!(r2c < lo)) nre++;
      if (!accept && r2c < hi2) {
        int kx, ky, kz;
        slot_image(S, slot, ixlo, g->nc[0], kx, ky, kz);
        if (RECORD)
          accept = guard_band_accept(g, q, __float_as_int(pi.w), __float_as_int(pos[j].w), kx, ky, kz);
        else
          defer_recheck(rlist, rcount, err, ki, j, kx, ky, kz);  // decided by the fix-up pass
      }
      // the particle itself: the same sorted index at exactly zero distance
      if (accept && !(j == ki && r2c == 0.f)) {
        if (HALF) {
          float gx, gy, gz;
          acc.add_pair(pp, cx, cy, cz, r2c, gx, gy, gz);
          red_shared_add(&S.Fj[0][slot], gx);
          red_shared_add(&S.Fj[HALF ? 1 : 0][slot], gy);
          red_shared_add(&S.Fj[HALF ? 2 : 0][slot], gz);
        } else {
          acc.add_r2(pp, cx, cy, cz, r2c);
        }
        if (RECORD) {
          int kx, ky, kz;
          slot_image(S, slot, ixlo, g->nc[0], kx, ky, kz);
          record_pair(g, q, __float_as_int(pi.w), __float_as_int(pos[j].w), kx, ky, kz, pair_buf, pair_count,
                      pair_cap);
        }
      }
    }
  }
  qn = 0;
}

// HALF: add the forces accumulated on staged partners [0, fill) to F
// (Cartesian, F = Q F_frame), then the slots may be reused.
template <bool HALF>
__device__ __forceinline__ void flush_partners(WarpStageT<HALF> &S, int fill, int lane, const Geo *g,
                                               const float4 *__restrict__ pos, float *F) {
  if (!HALF) return;
  __syncwarp();
  if (F) {
    const float *Qm = g->Qf;
    for (int t = lane; t < fill; t += 32) {
      const float fx = S.Fj[0][t], fy = S.Fj[HALF ? 1 : 0][t], fz = S.Fj[HALF ? 2 : 0][t];
      if (fx != 0.f || fy != 0.f || fz != 0.f) {
        const int oj = __float_as_int(pos[__float_as_int(S.R[t].w)].w);
        atomicAdd(&F[3 * (size_t)oj], Qm[0] * fx + Qm[1] * fy + Qm[2] * fz);
        atomicAdd(&F[3 * (size_t)oj + 1], Qm[3] * fx + Qm[4] * fy + Qm[5] * fz);
        atomicAdd(&F[3 * (size_t)oj + 2], Qm[6] * fx + Qm[7] * fy + Qm[8] * fz);
      }
    }
  }
  __syncwarp();
}

// Window of one staged row for the chunk: the window cells u in [ufirst, ulast]
// (ulast < ufirst: none) whose A = dxlo + sxi + u can hold a partner of a lane
// with kappa position in [pmin, pmax], and the wrapped x-cell jx of the first.
struct RowWindow {
  int ufirst, ulast, jx, ulo;
};

__device__ __forceinline__ RowWindow row_window(const float4 &s0, const float4 &s1, const float4 &s2, int ixlo,
                                                int ixhi, int l1, float kx0, float ky0, float kz0, float pmin,
                                                float pmax, float reach1) {
  const int dxlo = __float_as_int(s1.w);
  const int rcnt = __float_as_int(s2.x), sxi = __float_as_int(s2.z);
  RowWindow w;
  w.ulo = ixlo + dxlo;
  const int nu = ixhi - ixlo + rcnt;
  // the row shift along the row
  const float sh1 = fmaf(kz0, s0.z + s1.z, fmaf(ky0, s0.y + s1.y, kx0 * (s0.x + s1.x)));
  const float a0 = (float)(dxlo + sxi) + sh1;
  w.ufirst = max(0, (int)ceilf(pmin - reach1 - a0));
  w.ulast = min(nu - 1, (int)floorf(pmax + reach1 - a0));
  const int ustart = w.ulo + w.ufirst;
  w.jx = ustart - floordiv_dev(ustart, l1) * l1;
  return w;
}

// Everything one warp does for one chunk cd: stage the rows of the chunk's
// class (crow, nr of them), then per row stage, test and queue, flushing as
// needed.  On return acc.fx, fy, fz hold the force on the lane's particle pi
// (sorted index ki; act is false for lanes past the chunk's count) in the
// variant's frame, and its pair sums have been added to acc.  cell_base is the
// system's first cell slot (0 for a single system).  HALF visits only the rows
// ahead of the home row and the forward half of the home row, and adds the
// partners' forces to F (which must start at zero) as it goes.
template <bool RECORD, bool HALF>
__device__ __forceinline__ void warp_chunk(const int4 cd, const Row *__restrict__ crow, int nr, int cell_base,
                                           const Geo *g, const float4 *__restrict__ pos,
                                           const float4 *__restrict__ posr, const int *__restrict__ cell_sorted,
                                           const int *__restrict__ start, WarpStageT<HALF> &S, const Pot &pp,
                                           const double *q, float *F, Acc &acc, int &ncand, int &nre, bool &act,
                                           float4 &pi, int &ki, int32_t *pair_buf, unsigned long long *pair_count,
                                           long long pair_cap, int4 *rlist, int *rcount, int *err) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int kStage = WarpStageT<HALF>::kSlots;
  const int lane = threadIdx.x & 31;
  const int l1 = g->nc[0];
  const float sx = g->step[0], sy = g->step[1], sz = g->step[2];
  const float srx = g->step_r[0], sry = g->step_r[1], srz = g->step_r[2];
  act = lane < cd.y;
  ki = act ? cd.x + lane : cd.x;  // inactive lanes shadow a valid particle
  pi = pos[ki];
  const float4 pir = posr[ki];
  const int ixlo = cd.w & 0xffff, ixhi = cd.w >> 16;
  const int ixu = (cell_sorted[ki] - cell_base) % l1;
  const float ai = (float)(ixu - ixlo);
  const float3 Xi = make_float3(fmaf(ai, sx, pi.x), fmaf(ai, sy, pi.y), fmaf(ai, sz, pi.z));
  const float3 Ri = make_float3(fmaf(ai, srx, pir.x), fmaf(ai, sry, pir.y), fmaf(ai, srz, pir.z));
  if (nr > kRowsStaged) {
    // more rows than the stage holds (cell factor > 2): refused as a capacity error
    if (lane == 0) atomicOr(err, ERRB_CAPACITY);
    nr = kRowsStaged;
  }
  {
    const float4 *src = reinterpret_cast<const float4 *>(crow);
    __syncwarp();
    for (int e = lane; e < 3 * nr; e += 32) S.rows[e / 3][e % 3] = src[e];
    __syncwarp();
  }
  int rhome = -1;
  if (HALF)
    for (int r = 0; r < nr; r++)
      if (__float_as_int(S.rows[r][2].w) == 0) rhome = r;
  // Coarse test in dot-product form: r^2 = |X_i|^2 + |X_j|^2 - 2 X_i . X_j, so a
  // test is three fused multiply-adds on the staged (X_j, |X_j|^2) against
  // thr = rc2_hi - |X_i|^2 + margin.  Every candidate with exact quantised r^2
  // below rc2_hi has |X_j| <= |X_i| + rc + 1, and for such candidates the
  // roundings (of |X_j|^2, the three products, |X_i|^2 and thr) stay below
  // 10 u (2 |X_i| + rc + 1)^2, u = 2^-24: the margin, so no partner is lost.
  // Candidates accepted only through the margin are rejected by the flush's
  // corrected distance, so the pair set is unchanged.
  const float n2i = fmaf(Xi.z, Xi.z, fmaf(Xi.y, Xi.y, Xi.x * Xi.x));
  const float mxi = -2.0f * Xi.x, myi = -2.0f * Xi.y, mzi = -2.0f * Xi.z;
  const float ebound = 2.0f * (fabsf(Xi.x) + fabsf(Xi.y) + fabsf(Xi.z)) + sqrtf(g->rc2_hi) + 1.0f;
  const float thr = act ? (g->rc2_hi - n2i) + 5.9604645e-7f * ebound * ebound : -1e30f;  // inactive: accepts nothing
  acc.fx = acc.fy = acc.fz = 0.f;
  int qn = 0, fill = 0;
  // extent of the lanes along the row (cell units from the chunk's first cell):
  // a staged cell whose kappa range lies farther than rho1 from every lane
  // holds no partner of any lane and is skipped
  const float kx0 = g->kap[0], ky0 = g->kap[1], kz0 = g->kap[2];
  const float P = ai + fmaf(kz0, pi.z, fmaf(ky0, pi.y, kx0 * pi.x));
  float pmin = act ? P : 1e30f, pmax = act ? P : -1e30f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pmin = fminf(pmin, __shfl_xor_sync(FULL, pmin, o));
    pmax = fmaxf(pmax, __shfl_xor_sync(FULL, pmax, o));
  }
  const float reach1 = g->rho1 + 0.5f + 1e-4f;
  // lane r looks up the particle ranges of the first two runs of row r, so that
  // the row loop finds them without a dependent global load
  int rb0 = 0, re0 = 0, rb1 = 0, re1 = 0;
  if (lane < nr) {
    const float4 s0 = S.rows[lane][0], s1 = S.rows[lane][1], s2 = S.rows[lane][2];
    const RowWindow w = row_window(s0, s1, s2, ixlo, ixhi, l1, kx0, ky0, kz0, pmin, pmax, reach1);
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
    }
  }

  for (int r = 0; r < nr; r++) {
    const float4 s0 = S.rows[r][0], s1 = S.rows[r][1], s2 = S.rows[r][2];
    const int pb0 = __shfl_sync(FULL, rb0, r), pe0 = __shfl_sync(FULL, re0, r);
    const int pb1 = __shfl_sync(FULL, rb1, r), pe1 = __shfl_sync(FULL, re1, r);
    if (HALF && __float_as_int(s2.w) < 0) continue;  // met from the partner's side
    const int cbase = __float_as_int(s0.w), dxlo = __float_as_int(s1.w);
    const int sxi = __float_as_int(s2.z);
    const RowWindow w = row_window(s0, s1, s2, ixlo, ixhi, l1, kx0, ky0, kz0, pmin, pmax, reach1);
    const int ufirst = w.ufirst, ulast = w.ulast;
    int jx = w.jx;
    // runs of consecutive cells without an x-wrap: contiguous particles
    for (int u = ufirst, run = 0; u <= ulast; run++) {
      const int len = min(ulast + 1 - u, l1 - jx);
      const int b = run == 0 ? pb0 : (run == 1 ? pb1 : start[cbase + jx]);
      const int e = run == 0 ? pe0 : (run == 1 ? pe1 : start[cbase + jx + len]);
      const int arun = dxlo + sxi + u - jx;  // A of a particle of cell jx' of this run: arun + jx'
      if (act) ncand += e - b;
      for (int p = b; p < e;) {
        if (fill == kStage) {
          warp_flush<RECORD, HALF>(S, qn, nre, lane, ki, pi, Xi, Ri, ixu, ixlo, rhome, g, pos, pp, acc, q, pair_buf,
                                   pair_count, pair_cap, rlist, rcount, err);
          flush_partners<HALF>(S, fill, lane, g, pos, F);
          fill = 0;
        }
        const int take = min(e - p, kStage - fill);
        __syncwarp();  // slots about to be overwritten are no longer read
        // two particles per lane per pass, both loaded before either is stored
        for (int t0 = lane; t0 < take; t0 += 64) {
          const int t1 = t0 + 32;
          const bool two = t1 < take;
          const int j0 = p + t0, j1 = two ? p + t1 : j0;
          const float4 pj0 = pos[j0], pjr0 = posr[j0];
          const int c0 = cell_sorted[j0];
          const float4 pj1 = pos[j1], pjr1 = posr[j1];
          const int c1 = cell_sorted[j1];
#pragma unroll
          for (int h = 0; h < 2; h++) {
            if (h == 1 && !two) break;
            const int t = h ? t1 : t0, j = h ? j1 : j0;
            const float4 pj = h ? pj1 : pj0, pjr = h ? pjr1 : pjr0;
            const int cjx = (h ? c1 : c0) - cbase;
            const float A = (float)(arun + cjx);
            const float xx = fmaf(A, sx, pj.x + s0.x), xy = fmaf(A, sy, pj.y + s0.y), xz = fmaf(A, sz, pj.z + s0.z);
            S.X[fill + t] = make_float4(xx, xy, xz, fmaf(xz, xz, fmaf(xy, xy, xx * xx)));
            S.R[fill + t] = make_float4(fmaf(A, srx, pjr.x + s1.x), fmaf(A, sry, pjr.y + s1.y),
                                        fmaf(A, srz, pjr.z + s1.z), __int_as_float(j));
            S.SA[fill + t] = (unsigned short)(r | ((arun + cjx + kABias) << 5));
            if (HALF) {
              S.Fj[0][fill + t] = 0.f;
              S.Fj[HALF ? 1 : 0][fill + t] = 0.f;
              S.Fj[HALF ? 2 : 0][fill + t] = 0.f;
            }
          }
        }
        __syncwarp();
        for (int k0 = fill; k0 < fill + take; k0 += kTestBlock) {
          const int k1 = min(fill + take, k0 + kTestBlock);
          if (__any_sync(FULL, qn > kWarpQueue - kTestBlock))
            warp_flush<RECORD, HALF>(S, qn, nre, lane, ki, pi, Xi, Ri, ixu, ixlo, rhome, g, pos, pp, acc, q, pair_buf,
                                     pair_count, pair_cap, rlist, rcount, err);
#define NEMD_TEST(P, K)                                                       \
  {                                                                           \
    const float t = fmaf(mxi, (P).x, fmaf(myi, (P).y, fmaf(mzi, (P).z, (P).w))); \
    S.q[qn][lane] = (typename WarpStageT<HALF>::Entry)(K);                    \
    qn += (t < thr) ? 1 : 0;                                                  \
  }
          int k = k0;
          for (; k + 4 <= k1; k += 4) {
            const float4 p0 = S.X[k], p1 = S.X[k + 1], p2 = S.X[k + 2], p3 = S.X[k + 3];
            NEMD_TEST(p0, k);
            NEMD_TEST(p1, k + 1);
            NEMD_TEST(p2, k + 2);
            NEMD_TEST(p3, k + 3);
          }
          for (; k < k1; k++) {
            const float4 p0 = S.X[k];
            NEMD_TEST(p0, k);
          }
#undef NEMD_TEST
        }
        fill += take;
        p += take;
      }
      u += len;
      jx += len;
      if (jx == l1) jx = 0;
    }
  }
  warp_flush<RECORD, HALF>(S, qn, nre, lane, ki, pi, Xi, Ri, ixu, ixlo, rhome, g, pos, pp, acc, q, pair_buf, pair_count,
                           pair_cap, rlist, rcount, err);
  flush_partners<HALF>(S, fill, lane, g, pos, F);
}

// F (Cartesian) of a lane's particle from its frame force: F = Q F_frame.
__device__ __forceinline__ void store_force(float *F, const Geo *g, const float4 &pi, const Acc &acc) {
  const float *Qm = g->Qf;
  const int oi = __float_as_int(pi.w);
  F[3 * (size_t)oi] = Qm[0] * acc.fx + Qm[1] * acc.fy + Qm[2] * acc.fz;
  F[3 * (size_t)oi + 1] = Qm[3] * acc.fx + Qm[4] * acc.fy + Qm[5] * acc.fz;
  F[3 * (size_t)oi + 2] = Qm[6] * acc.fx + Qm[7] * acc.fy + Qm[8] * acc.fz;
}

// HALF: other warps add partner forces to the same particles, so the lane's own
// force is added too.
__device__ __forceinline__ void add_force(float *F, const Geo *g, const float4 &pi, const Acc &acc) {
  const float *Qm = g->Qf;
  const int oi = __float_as_int(pi.w);
  atomicAdd(&F[3 * (size_t)oi], Qm[0] * acc.fx + Qm[1] * acc.fy + Qm[2] * acc.fz);
  atomicAdd(&F[3 * (size_t)oi + 1], Qm[3] * acc.fx + Qm[4] * acc.fy + Qm[5] * acc.fz);
  atomicAdd(&F[3 * (size_t)oi + 2], Qm[6] * acc.fx + Qm[7] * acc.fy + Qm[8] * acc.fz);
}

template <bool RECORD, bool HALF>
__global__ void __launch_bounds__(kWarpThreads, NEMD_WARP_MINBLOCKS) k_force_warp(
    const Geo *__restrict__ g, const float4 *__restrict__ pos, const float4 *__restrict__ posr,
    const int *__restrict__ cell_sorted, const int *__restrict__ start, const Row *__restrict__ rows,
    const int *__restrict__ rowcnt, const int4 *__restrict__ chunks, const int *__restrict__ nchunks_p,
    const double *__restrict__ q, Pot pp, float *__restrict__ F, double *__restrict__ partials,
    int32_t *__restrict__ pair_buf, unsigned long long *__restrict__ pair_count, long long pair_cap,
    int4 *__restrict__ rlist, int *__restrict__ rcount, int *__restrict__ err) {
  constexpr int kWarps = kWarpThreads / 32;
  __shared__ WarpStageT<HALF> stage[kWarps];
  const int warp = threadIdx.x >> 5;

  Acc acc;  // U, W and the pair count accumulate over every particle this lane owns
  acc.zero();
  int ncand = 0, nre = 0;
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  const int nch = ok ? *nchunks_p : 0;
  const int maxrows = g->maxrows;

  for (int ch = blockIdx.x * kWarps + warp; ch < nch; ch += gridDim.x * kWarps) {
    const int4 cd = chunks[ch];
    bool act;
    float4 pi;
    int ki;
    warp_chunk<RECORD, HALF>(cd, rows + (size_t)cd.z * maxrows, rowcnt[cd.z], 0, g, pos, posr, cell_sorted, start,
                             stage[warp], pp, q, F, acc, ncand, nre, act, pi, ki, pair_buf, pair_count, pair_cap,
                             rlist, rcount, err);
    if (act && F) {
      if (HALF)
        add_force(F, g, pi, acc);
      else
        store_force(F, g, pi, acc);
    }
  }
  double v[kPartials] = {acc.u, acc.wxx, acc.wyy, acc.wzz, acc.wxy, acc.wxz, acc.wyz,
                         (double)acc.npair, (double)ncand, (double)nre};
  block_reduce_store<kWarpThreads>(v, partials);
}

template <bool RECORD, bool HALF>
static int warp_resident_blocks(int sms) {
  static int per_sm = 0;
  if (!per_sm) {
    cudaFuncSetAttribute(k_force_warp<RECORD, HALF>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_warp<RECORD, HALF>, kWarpThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  return per_sm * sms;
}

bool warp_kernel_applies(const nemd_ctx *c) { return c->kfac <= 2; }

// half: half neighbourhoods (F must have been zeroed; not with pair records).
cudaError_t launch_force_warp(nemd_ctx *c, float *F, int *nblocks, bool half) {
  const Pot pp = make_pot(c);
  const bool rec = c->record_cap > 0;
  half = half && !rec;
  int blocks = rec ? warp_resident_blocks<true, false>(c->sms)
                   : (half ? warp_resident_blocks<false, true>(c->sms) : warp_resident_blocks<false, false>(c->sms));
  if (blocks > (int)(c->cap_partials - 1)) blocks = (int)(c->cap_partials - 1);
  *nblocks = blocks;
#define NEMD_ARGS                                                                                            \
  c->geo, c->pos4, c->posr, c->cell_sorted, c->start, c->rows, c->rowcnt, c->chunks, c->chunk_off + c->cap_cells, \
      c->q_dev, pp, F, c->partials, c->pair_buf, c->pair_count, (long long)c->record_cap, c->recheck, c->nrecheck, \
      &c->geo->error
  if (rec)
    k_force_warp<true, false><<<blocks, kWarpThreads, 0, c->stream>>>(NEMD_ARGS);
  else if (half)
    k_force_warp<false, true><<<blocks, kWarpThreads, 0, c->stream>>>(NEMD_ARGS);
  else
    k_force_warp<false, false><<<blocks, kWarpThreads, 0, c->stream>>>(NEMD_ARGS);
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
__global__ void __launch_bounds__(kWarpThreads, NEMD_WARP_MINBLOCKS) k_b_force_warp(BatchView v) {
  constexpr int kWarps = kWarpThreads / 32;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ WarpStage stage[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nch = v.chunk_off[v.nclasses];
  for (;;) {
    int ch = 0;
    if (lane == 0) ch = atomicAdd(v.work, 1);
    ch = __shfl_sync(FULL, ch, 0);
    if (ch >= nch) break;
    const int4 cd = v.chunks[ch];
    const int s = v.class_sys[cd.z];
    Geo *g = v.geo + s;
    const int coff = v.sys[s].coff;
    const Pot pp = v.pot[s];
    Acc acc;
    acc.zero();
    int ncand = 0, nre = 0;
    bool act;
    float4 pi;
    int ki;
    warp_chunk<false, false>(cd, v.rows + (size_t)cd.z * kBatchRowStride, v.rowcnt[cd.z], coff, g, v.pos4, v.posr,
                             v.cell_sorted, v.start, stage[warp], pp, v.q, v.F, acc, ncand, nre, act, pi, ki, nullptr,
                             nullptr, 0, v.recheck, v.nrecheck, &g->error);
    if (act) {
      if (v.F) store_force(v.F, g, pi, acc);
      v.ppart[2 * (size_t)ki] = make_float4(acc.u, acc.wxx, acc.wyy, acc.wzz);
      v.ppart[2 * (size_t)ki + 1] = make_float4(acc.wxy, acc.wxz, acc.wyz, __int_as_float(acc.npair));
    }
    const unsigned c = __reduce_add_sync(FULL, (unsigned)ncand), r = __reduce_add_sync(FULL, (unsigned)nre);
    if (lane == 0) {
      atomicAdd(&v.sys_counters[2 * s], (unsigned long long)c);
      if (r) atomicAdd(&v.sys_counters[2 * s + 1], (unsigned long long)r);
    }
  }
}

int batch_force_blocks(int sms) {
  static int per_sm = 0;
  if (!per_sm) {
    cudaFuncSetAttribute(k_b_force_warp, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_force_warp, kWarpThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  return per_sm * sms;
}

cudaError_t launch_batch_force(cudaStream_t st, const BatchView &v, int blocks) {
  cudaError_t e = cudaMemsetAsync(v.work, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.nrecheck, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.sys_counters, 0, 2 * sizeof(unsigned long long) * (size_t)v.nsys, st);
  if (e != cudaSuccess) return e;
  k_b_force_warp<<<blocks, kWarpThreads, 0, st>>>(v);
  return cudaGetLastError();
}

}  // namespace nemd
