// force_warp.cu -- warp force kernel: the grouped kernel's algorithm with one
// chunk per warp (Sec. 3 and 5: neighbourhood cells only, distance check
// before force; same pair set and pair arithmetic as the other kernels).
//
// A warp takes a chunk of at most 32 consecutive particles of one x-row of
// cells, one particle per lane.  Every loop bound is uniform across the warp
// (one chunk, one cell at a time), so the test loop carries no per-candidate
// bookkeeping: it is unrolled four-fold, inactive lanes are switched off by a
// threshold that no r^2 can pass, and every tested candidate is written to the
// lane's queue slot unconditionally -- the slot only advances when the test
// passes -- so accepting costs no branch.  The chunk's rows are staged in
// shared memory for the force phase (flush), which reads them per queued pair.
#include <math.h>

#include "batch_internal.cuh"

namespace nemd {

#ifndef NEMD_WARP_QUEUE
#define NEMD_WARP_QUEUE 64
#endif
#ifndef NEMD_FLUSH_UNROLL
#define NEMD_FLUSH_UNROLL 1
#endif
constexpr int kWarpQueue = NEMD_WARP_QUEUE;   // queue entries per lane
constexpr int kFlushUnroll = NEMD_FLUSH_UNROLL;  // queued pairs gathered at once in a flush
constexpr int kWarpThreads = 128;  // 4 warps per block
constexpr int kRowsStaged = 32;    // rows per class the kernel stages (cell factor <= 2)
constexpr int kWJBits = 21;
constexpr unsigned kWJMask = (1u << kWJBits) - 1u;
constexpr unsigned kWBandFlag = 1u << kWJBits;

// One queued pair: displacement with the residuals added back, coarse-band
// decision, force.
template <bool RECORD>
__device__ __forceinline__ void warp_pair(unsigned int ent, const float4 &pj, const float4 &pjr, int &nre, const float4 &pi,
                                          const float4 &pir, int ki, int ix, int jbase, const float4 (*rs)[3], const Geo *g,
                                          const Pot &pp, Acc &acc, const double *q, int32_t *pair_buf,
                                          unsigned long long *pair_count, long long pair_cap, int4 *rlist,
                                          int *rcount, int *err) {
  const int j = jbase + (int)(ent & kWJMask), r = (ent >> 22) & 31, nidx = (int)(ent >> 27) - 16;
  const float4 sh = rs[r][0], sr = rs[r][1];
  const float cx = (pj.x - sub_offset(pi.x, sh.x, nidx, g->step[0])) + (pjr.x - sub_residual(pir.x, sr.x, nidx, g->step_r[0]));
  const float cy = (pj.y - sub_offset(pi.y, sh.y, nidx, g->step[1])) + (pjr.y - sub_residual(pir.y, sr.y, nidx, g->step_r[1]));
  const float cz = (pj.z - sub_offset(pi.z, sh.z, nidx, g->step[2])) + (pjr.z - sub_residual(pir.z, sr.z, nidx, g->step_r[2]));
  bool accept = true;
  if (ent & kWBandFlag) {
    nre++;
    const float r2c = fmaf(cz, cz, fmaf(cy, cy, cx * cx));
    accept = r2c < g->rc2_lo2;
    if (!accept && r2c < g->rc2_hi2) {
      const float4 r2w = rs[r][2];
      const int sxi = __float_as_int(r2w.z), kyz = __float_as_int(r2w.y);
      const int kx = floordiv_dev(ix + nidx - sxi, g->nc[0]);
      const int ky = (short)(kyz & 0xffff), kz = kyz >> 16;
      if (RECORD)
        accept = guard_band_accept(g, q, __float_as_int(pi.w), __float_as_int(pj.w), kx, ky, kz);
      else
        defer_recheck(rlist, rcount, err, ki, j, kx, ky, kz);  // decided by the fix-up pass
    }
  }
  // the particle itself: offset 0 and identical coordinates give exactly 0
  if (accept && !(j == ki && cx == 0.f && cy == 0.f && cz == 0.f)) {
    acc.add(pp, cx, cy, cz);
    if (RECORD) {
      const float4 r2w = rs[r][2];
      const int sxi = __float_as_int(r2w.z), kyz = __float_as_int(r2w.y);
      record_pair(g, q, __float_as_int(pi.w), __float_as_int(pj.w), floordiv_dev(ix + nidx - sxi, g->nc[0]),
                  (short)(kyz & 0xffff), kyz >> 16, pair_buf, pair_count, pair_cap);
    }
  }
}

// Forces of the queued pairs of every lane; the warp takes kFlushUnroll
// entries per lane at a time so that their gathers overlap.
template <bool RECORD>
__device__ __forceinline__ void warp_flush(unsigned int (*myq)[32], int &qn, int &nre, int lane, const float4 &pi,
                                           int ki, int ix, int jbase, const float4 (*rs)[3], const Geo *g, const float4 *pos,
                                           const float4 *posr, const Pot &pp, Acc &acc, const double *q,
                                           int32_t *pair_buf, unsigned long long *pair_count, long long pair_cap,
                                           int4 *rlist, int *rcount, int *err) {
  const int m = __reduce_max_sync(0xffffffffu, qn);
  if (m == 0) return;
  const float4 pir = posr[ki];
  for (int s = 0; s < m; s += kFlushUnroll) {
    unsigned int ent[kFlushUnroll];
    float4 pj[kFlushUnroll], pjr[kFlushUnroll];
#pragma unroll
    for (int u = 0; u < kFlushUnroll; u++) {
      // past the lane's own entries: a harmless stand-in (entry 0, or the lane's own particle)
      ent[u] = myq[min(s + u, kWarpQueue - 1)][lane];
      const int j = (s + u < qn) ? jbase + (int)(ent[u] & kWJMask) : ki;
      pj[u] = pos[j];
      pjr[u] = posr[j];
    }
#pragma unroll
    for (int u = 0; u < kFlushUnroll; u++)
      if (s + u < qn)
        warp_pair<RECORD>(ent[u], pj[u], pjr[u], nre, pi, pir, ki, ix, jbase, rs, g, pp, acc, q, pair_buf, pair_count,
                          pair_cap, rlist, rcount, err);
  }
  qn = 0;
}

// Everything one warp does for one chunk cd (Sec. 3 and 5): stage the rows of
// the chunk's class, test every particle of the union of the lanes' windows,
// queue and flush.  On return acc.fx, fy, fz hold the force on the lane's
// particle pi (index ki; act is false for lanes past the chunk's count) in the
// variant's frame, and its pair sums have been added to acc.  cell_base and
// jbase are the system's first cell slot and first sorted particle (0 for a
// single system): queue entries hold partner indices relative to jbase.
template <bool RECORD>
__device__ __forceinline__ void warp_chunk(const int4 cd, const Row *__restrict__ crow, int nr, int cell_base,
                                           int jbase, const Geo *g, const float4 *__restrict__ pos,
                                           const float4 *__restrict__ posr, const int *__restrict__ cell_sorted,
                                           const int *__restrict__ start, unsigned int (*myq)[32],
                                           float4 (*rs)[3], const Pot &pp, const double *q, Acc &acc, int &ncand,
                                           int &nre, bool &act, float4 &pi, int &ki, int32_t *pair_buf,
                                           unsigned long long *pair_count, long long pair_cap, int4 *rlist,
                                           int *rcount, int *err) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int l1 = g->nc[0];
  const float lo = g->rc2_lo, hi = g->rc2_hi;
  const float sx = g->step[0], sy = g->step[1], sz = g->step[2];
  act = lane < cd.y;
  ki = act ? cd.x + lane : cd.x;  // inactive lanes shadow a valid particle
  pi = pos[ki];
  const int ix = (cell_sorted[ki] - cell_base) % l1;
  const int ixlo = cd.w & 0xffff, ixhi = cd.w >> 16;
  {
    const float4 *src = reinterpret_cast<const float4 *>(crow);
    __syncwarp();
    for (int e = lane; e < 3 * nr; e += 32) rs[e / 3][e % 3] = src[e];
    __syncwarp();
  }
  const float hil = act ? hi : -1.0f;  // an inactive lane accepts nothing
  acc.fx = acc.fy = acc.fz = 0.f;
  int qn = 0;

  for (int r = 0; r < nr; r++) {
    const float4 s0 = rs[r][0];
    const int cbase = __float_as_int(s0.w), dxlo = __float_as_int(rs[r][1].w);
    const int rcnt = __float_as_int(rs[r][2].x), sxi = __float_as_int(rs[r][2].z);
    const int ulo = ixlo + dxlo, nu = ixhi - ixlo + rcnt;
    int jx = ulo - floordiv_dev(ulo, l1) * l1;
    for (int u = 0; u < nu; u++) {
      const int b = start[cbase + jx], e = start[cbase + jx + 1];
      const int nidx = ulo + u - ix + sxi;
      const float tx = sub_offset(pi.x, s0.x, nidx, sx), ty = sub_offset(pi.y, s0.y, nidx, sy),
                  tz = sub_offset(pi.z, s0.z, nidx, sz);
      const unsigned int tag = ((unsigned)r << 22) | ((unsigned)(nidx + 16) << 27);
      if (act) ncand += e - b;
      // segments of at most kWarpQueue - 1 candidates: the unconditional store
      // of a test must always land inside the queue
      for (int seg = b; seg < e; seg += kWarpQueue - 1) {
        const int send = min(e, seg + kWarpQueue - 1);
        if (__any_sync(FULL, qn + (send - seg) > kWarpQueue - 1))
          warp_flush<RECORD>(myq, qn, nre, lane, pi, ki, ix, jbase, rs, g, pos, posr, pp, acc, q, pair_buf,
                             pair_count, pair_cap, rlist, rcount, err);
#define NEMD_TEST(P, J)                                                                   \
  {                                                                                       \
    const float ddx = (P).x - tx, ddy = (P).y - ty, ddz = (P).z - tz;                     \
    const float r2 = fmaf(ddz, ddz, fmaf(ddy, ddy, ddx * ddx));                           \
    myq[qn][lane] = (unsigned)(J) | tag | (r2 < lo ? 0u : kWBandFlag);                    \
    qn += (r2 < hil) ? 1 : 0;                                                             \
  }
        int j = seg;
        for (; j + 4 <= send; j += 4) {
          const float4 p0 = pos[j], p1 = pos[j + 1], p2 = pos[j + 2], p3 = pos[j + 3];
          const int jr = j - jbase;
          NEMD_TEST(p0, jr);
          NEMD_TEST(p1, jr + 1);
          NEMD_TEST(p2, jr + 2);
          NEMD_TEST(p3, jr + 3);
        }
        for (; j < send; j++) {
          const float4 p0 = pos[j];
          NEMD_TEST(p0, j - jbase);
        }
#undef NEMD_TEST
      }
      if (++jx == l1) jx = 0;
    }
  }
  warp_flush<RECORD>(myq, qn, nre, lane, pi, ki, ix, jbase, rs, g, pos, posr, pp, acc, q, pair_buf, pair_count,
                     pair_cap, rlist, rcount, err);
}

// F (Cartesian) of a lane's particle from its frame force: F = Q F_frame.
__device__ __forceinline__ void store_force(float *F, const Geo *g, const float4 &pi, const Acc &acc) {
  const float *Qm = g->Qf;
  const int oi = __float_as_int(pi.w);
  F[3 * (size_t)oi] = Qm[0] * acc.fx + Qm[1] * acc.fy + Qm[2] * acc.fz;
  F[3 * (size_t)oi + 1] = Qm[3] * acc.fx + Qm[4] * acc.fy + Qm[5] * acc.fz;
  F[3 * (size_t)oi + 2] = Qm[6] * acc.fx + Qm[7] * acc.fy + Qm[8] * acc.fz;
}

template <bool RECORD>
__global__ void __launch_bounds__(kWarpThreads) k_force_warp(
    const Geo *__restrict__ g, const float4 *__restrict__ pos, const float4 *__restrict__ posr,
    const int *__restrict__ cell_sorted, const int *__restrict__ start, const Row *__restrict__ rows,
    const int *__restrict__ rowcnt, const int4 *__restrict__ chunks, const int *__restrict__ nchunks_p,
    const double *__restrict__ q, Pot pp, float *__restrict__ F, double *__restrict__ partials,
    int32_t *__restrict__ pair_buf, unsigned long long *__restrict__ pair_count, long long pair_cap,
    int4 *__restrict__ rlist, int *__restrict__ rcount, int *__restrict__ err) {
  constexpr int kWarps = kWarpThreads / 32;
  __shared__ unsigned int qbuf[kWarps][kWarpQueue][32];
  __shared__ float4 rstage[kWarps][kRowsStaged][3];
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
    warp_chunk<RECORD>(cd, rows + (size_t)cd.z * maxrows, rowcnt[cd.z], 0, 0, g, pos, posr, cell_sorted, start,
                       qbuf[warp], rstage[warp], pp, q, acc, ncand, nre, act, pi, ki, pair_buf, pair_count, pair_cap,
                       rlist, rcount, err);
    if (act && F) store_force(F, g, pi, acc);
  }
  double v[kPartials] = {acc.u, acc.wxx, acc.wyy, acc.wzz, acc.wxy, acc.wxz, acc.wyz,
                         (double)acc.npair, (double)ncand, (double)nre};
  block_reduce_store<kWarpThreads>(v, partials);
}

template <bool RECORD>
static int warp_resident_blocks(int sms) {
  static int per_sm = 0;
  if (!per_sm) {
    cudaFuncSetAttribute(k_force_warp<RECORD>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_warp<RECORD>, kWarpThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  return per_sm * sms;
}

bool warp_kernel_applies(const nemd_ctx *c) { return c->n <= (1 << kWJBits) && c->kfac <= 2; }

cudaError_t launch_force_warp(nemd_ctx *c, float *F, int *nblocks) {
  const Pot pp = make_pot(c);
  const bool rec = c->record_cap > 0;
  int blocks = rec ? warp_resident_blocks<true>(c->sms) : warp_resident_blocks<false>(c->sms);
  if (blocks > (int)(c->cap_partials - 1)) blocks = (int)(c->cap_partials - 1);
  *nblocks = blocks;
#define NEMD_ARGS                                                                                                \
  c->geo, c->pos4, c->posr, c->cell_sorted, c->start, c->rows, c->rowcnt, c->chunks, c->nchunks, c->q_dev, pp, \
      F, c->partials, c->pair_buf, c->pair_count, (long long)c->record_cap, c->recheck, c->nrecheck, &c->geo->error
  if (rec)
    k_force_warp<true><<<blocks, kWarpThreads, 0, c->stream>>>(NEMD_ARGS);
  else
    k_force_warp<false><<<blocks, kWarpThreads, 0, c->stream>>>(NEMD_ARGS);
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
__global__ void __launch_bounds__(kWarpThreads) k_b_force_warp(BatchView v) {
  constexpr int kWarps = kWarpThreads / 32;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ unsigned int qbuf[kWarps][kWarpQueue][32];
  __shared__ float4 rstage[kWarps][kRowsStaged][3];
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
    const int jbase = v.start[coff];
    const Pot pp = v.pot[s];
    Acc acc;
    acc.zero();
    int ncand = 0, nre = 0;
    bool act;
    float4 pi;
    int ki;
    warp_chunk<false>(cd, v.rows + (size_t)cd.z * kBatchRowStride, v.rowcnt[cd.z], coff, jbase, g, v.pos4, v.posr,
                      v.cell_sorted, v.start, qbuf[warp], rstage[warp], pp, v.q, acc, ncand, nre, act, pi, ki,
                      nullptr, nullptr, 0, v.recheck, v.nrecheck, &g->error);
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
