// force_chunk.cu -- grouped force kernel (same pair set and pair arithmetic as
// the plain kernel; Sec. 3 and 5: neighbourhood cells only, distance check
// before force).
//
// Work unit: a chunk of at most GS consecutive particles (in cell order) of one
// x-row of cells, spanning at most kMaxSpan cells.  A group of GS lanes takes
// one chunk, one particle per lane.  All its lanes share the row table of the
// chunk's (iy, iz) class, so for every neighbour row the group walks the union
// of its lanes' x-windows cell by cell, every lane testing every particle of
// the cell (broadcast loads, one trip count per group); a particle outside a
// lane's own window is simply farther than rc and fails the test.
//
// The test loop does not compute forces: a lane that accepts a candidate
// appends a 4-byte entry (partner index, row, offset index, and a flag when the
// candidate lies in the coarse guard band) to its own queue in shared memory,
// and the forces of the queued pairs are computed in flushes in which every
// lane works (the accept branch of a test is almost always taken by some lane
// of a warp, so forces computed inside the test loop would be paid per
// candidate).  Flagged entries are decided in the flush (residuals added back,
// then float64 if still undecided).  Each particle's force is accumulated by
// its own lane in a fixed order, so results are deterministic.
#include <math.h>

#include "batch_internal.cuh"

namespace nemd {

constexpr int kQueue = 64;  // queue entries per lane
constexpr int kChunkThreads = 128;

// Walk one x-row of cells (cells c0 .. c0 + l1 - 1) in order, cutting its
// particles into chunks of at most gs particles spanning at most span cells
// (Geo::span); emit(first, count, ixlo, ixhi) for each chunk, in order.
template <class Emit>
__device__ __forceinline__ void chunk_walk(const int *__restrict__ start, int c0, int l1, int gs, int span,
                                           Emit &&emit) {
  int first = 0, count = 0, ixlo = 0, ixhi = 0;
  for (int ix = 0; ix < l1; ix++) {
    const int b = start[c0 + ix], nc = start[c0 + ix + 1] - b;
    int off = 0;
    while (off < nc) {
      if (count > 0 && ix - ixlo >= span) {
        emit(first, count, ixlo, ixhi);
        count = 0;
      }
      if (count == 0) {
        first = b + off;
        ixlo = ix;
      }
      const int take = min(gs - count, nc - off);
      count += take;
      off += take;
      ixhi = ix;
      if (count == gs) {
        emit(first, count, ixlo, ixhi);
        count = 0;
      }
    }
  }
  if (count > 0) emit(first, count, ixlo, ixhi);
}

// Chunk descriptor: x = first sorted particle, y = count, z = class (iy + l2 iz),
// w = ixlo | ixhi << 16.  Built in a fixed order: chunks per class, their
// exclusive scan, and the descriptors at the scanned offsets -- so the chunk
// list, and every sum of the force kernels that walk it, are the same from run
// to run.  One warp per class: the lanes stage the row's cell starts in shared
// memory and one lane walks them.
constexpr int kWalkCells = 512;  // row lengths staged in shared memory (longer rows walk global memory)
constexpr int kWalkWarps = 4;

template <class Emit>
__device__ __forceinline__ void chunk_walk_warp(const int *__restrict__ start, int c0, int l1, int gs, int span,
                                                int *sm, int lane, Emit &&emit) {
  const bool staged = l1 < kWalkCells;
  __syncwarp();
  if (staged)
    for (int k = lane; k <= l1; k += 32) sm[k] = start[c0 + k];
  __syncwarp();
  if (lane == 0) {
    if (staged)
      chunk_walk(sm, 0, l1, gs, span, emit);
    else
      chunk_walk(start, c0, l1, gs, span, emit);
  }
}

__global__ void __launch_bounds__(32 * kWalkWarps) k_chunk_count(const Geo *__restrict__ g,
                                                                 const int *__restrict__ start,
                                                                 int *__restrict__ cnt, int gs, int wide) {
  __shared__ int sm[kWalkWarps][kWalkCells + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  const int l1 = g->nc[0], ncls = ok ? g->nc[1] * g->nc[2] : 0;
  const int nw = gridDim.x * kWalkWarps;
  for (int cls = blockIdx.x * kWalkWarps + warp; cls < ncls; cls += nw) {
    int n = 0;
    chunk_walk_warp(start, cls * l1, l1, gs, wide ? g->span : kMaxSpan, sm[warp], lane,
                    [&](int, int, int, int) { n++; });
    if (lane == 0) cnt[cls] = n;
  }
}

__global__ void __launch_bounds__(32 * kWalkWarps) k_chunk_write(const Geo *__restrict__ g,
                                                                 const int *__restrict__ start,
                                                                 const int *__restrict__ off,
                                                                 int4 *__restrict__ chunks, int gs, int wide) {
  __shared__ int sm[kWalkWarps][kWalkCells + 1];
  if (g->error & (ERRB_BOX | ERRB_CAPACITY)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l1 = g->nc[0], ncls = g->nc[1] * g->nc[2];
  const int nw = gridDim.x * kWalkWarps;
  for (int cls = blockIdx.x * kWalkWarps + warp; cls < ncls; cls += nw) {
    int k = off[cls];
    chunk_walk_warp(start, cls * l1, l1, gs, wide ? g->span : kMaxSpan, sm[warp], lane,
                    [&](int first, int count, int ixlo, int ixhi) {
      chunks[k++] = make_int4(first, count, cls, ixlo | (ixhi << 16));
    });
  }
}

// Queue entry: partner index (21 bits), coarse-band flag (1), row (5),
// offset index + 16 (5).
constexpr int kJBits = 21;
constexpr unsigned kJMask = (1u << kJBits) - 1u;
constexpr unsigned kBandFlag = 1u << kJBits;

// Forces of the queued pairs of one lane; every lane of the warp takes part.
template <bool RECORD>
__device__ __forceinline__ void flush_queue(unsigned int (*myq)[32], int &qn, int &nre, int lane, const float4 &pi,
                                            int ki, int ix, const Row *rw, const Geo *g, const float4 *pos,
                                            const float4 *posr, const Pot &pp, Acc &acc, const double *q,
                                            int32_t *pair_buf, unsigned long long *pair_count, long long pair_cap,
                                            int4 *rlist, int *rcount, int *err) {
  const int m = __reduce_max_sync(0xffffffffu, qn);
  if (m == 0) return;
  const float4 pir = posr[ki];
  const float sx = g->step[0], sy = g->step[1], sz = g->step[2];
  const float srx = g->step_r[0], sry = g->step_r[1], srz = g->step_r[2];
  for (int s = 0; s < m; s++) {
    if (s < qn) {
      const unsigned int ent = myq[s][lane];
      const int j = ent & kJMask, r = (ent >> 22) & 31, nidx = (int)(ent >> 27) - 16;
      const float4 sh = *reinterpret_cast<const float4 *>(&rw[r].shx);
      const float4 sr = *reinterpret_cast<const float4 *>(&rw[r].srx);
      const float4 pj = pos[j], pjr = posr[j];
      const float cx = (pj.x - sub_offset(pi.x, sh.x, nidx, sx)) + (pjr.x - sub_residual(pir.x, sr.x, nidx, srx));
      const float cy = (pj.y - sub_offset(pi.y, sh.y, nidx, sy)) + (pjr.y - sub_residual(pir.y, sr.y, nidx, sry));
      const float cz = (pj.z - sub_offset(pi.z, sh.z, nidx, sz)) + (pjr.z - sub_residual(pir.z, sr.z, nidx, srz));
      bool accept = true;
      if (ent & kBandFlag) {
        // coarse band: d now carries the residuals; float64 only within rounding of rc
        nre++;
        const float r2c = fmaf(cz, cz, fmaf(cy, cy, cx * cx));
        accept = r2c < g->rc2_lo2;
        if (!accept && r2c < g->rc2_hi2) {
          const int kx = floordiv_dev(ix + nidx - rw[r].sxi, g->nc[0]);
          if (RECORD)
            accept = guard_band_accept(g, q, __float_as_int(pi.w), __float_as_int(pj.w), kx, rw[r].ky, rw[r].kz);
          else
            defer_recheck(rlist, rcount, err, ki, j, kx, rw[r].ky, rw[r].kz);  // decided by the fix-up pass
        }
      }
      // the particle itself: offset 0 and identical coordinates give exactly 0
      if (accept && !(j == ki && cx == 0.f && cy == 0.f && cz == 0.f)) {
        acc.add(pp, cx, cy, cz);
        if (RECORD)
          record_pair(g, q, __float_as_int(pi.w), __float_as_int(pj.w),
                      floordiv_dev(ix + nidx - rw[r].sxi, g->nc[0]), rw[r].ky, rw[r].kz, pair_buf, pair_count,
                      pair_cap);
      }
    }
  }
  qn = 0;
}

template <int GS, bool RECORD>
__global__ void __launch_bounds__(kChunkThreads, 4) k_force_chunk(
    const Geo *__restrict__ g, const float4 *__restrict__ pos, const float4 *__restrict__ posr,
    const int *__restrict__ cell_sorted, const int *__restrict__ start, const Row *__restrict__ rows,
    const int *__restrict__ rowcnt, const int4 *__restrict__ chunks, const int *__restrict__ nchunks_p,
    const double *__restrict__ q, Pot pp, float *__restrict__ F, double *__restrict__ partials,
    int32_t *__restrict__ pair_buf, unsigned long long *__restrict__ pair_count, long long pair_cap,
    int4 *__restrict__ rlist, int *__restrict__ rcount, int *__restrict__ err) {
  constexpr int kWarps = kChunkThreads / 32;
  constexpr int GPW = 32 / GS;  // groups per warp
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ unsigned int qbuf[kWarps][kQueue][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane % GS, grp = lane / GS;
  unsigned int(*myq)[32] = qbuf[warp];

  Acc acc;  // U, W and the pair count accumulate over every particle this lane owns
  acc.zero();
  int ncand = 0, nre = 0;
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  const int nch = ok ? *nchunks_p : 0;
  const int l1 = g->nc[0], maxrows = g->maxrows;
  const float lo = g->rc2_lo, hi = g->rc2_hi;
  const float sx = g->step[0], sy = g->step[1], sz = g->step[2];

  for (int base = (blockIdx.x * kWarps + warp) * GPW; base < nch; base += gridDim.x * kWarps * GPW) {
    const int ch = base + grp;
    const bool have = ch < nch;
    const int4 cd = have ? chunks[ch] : make_int4(0, 0, 0, 0);
    const bool act = have && gl < cd.y;
    const int ki = act ? cd.x + gl : cd.x;  // inactive lanes shadow a valid particle
    const float4 pi = pos[ki];
    const int ix = cell_sorted[ki] % l1;
    const int ixlo = cd.w & 0xffff, ixhi = cd.w >> 16;
    const Row *rw = rows + (size_t)cd.z * maxrows;
    const int nr = have ? rowcnt[cd.z] : 0;
    const int nrmax = __reduce_max_sync(FULL, nr);
    acc.fx = acc.fy = acc.fz = 0.f;
    int qn = 0;

    for (int r = 0; r < nrmax; r++) {
      int cbase = 0, dxlo = 0, rcnt = 0, sxi = 0;
      float4 sh = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < nr) {
        sh = *reinterpret_cast<const float4 *>(&rw[r].shx);
        cbase = __float_as_int(sh.w);
        dxlo = rw[r].dxlo;
        rcnt = rw[r].cnt;
        sxi = rw[r].sxi;
      }
      const int ulo = ixlo + dxlo;
      const int nu = r < nr ? ixhi - ixlo + rcnt : 0;
      const int numax = __reduce_max_sync(FULL, nu);
      int jx = ulo - floordiv_dev(ulo, l1) * l1;
      for (int u = 0; u < numax; u++) {
        int b = 0, cnt = 0;
        if (u < nu) {
          b = start[cbase + jx];
          cnt = start[cbase + jx + 1] - b;
        }
        const int nidx = ulo + u - ix + sxi;
        const float tx = sub_offset(pi.x, sh.x, nidx, sx), ty = sub_offset(pi.y, sh.y, nidx, sy),
                    tz = sub_offset(pi.z, sh.z, nidx, sz);
        const unsigned int tag = ((unsigned)r << 22) | ((unsigned)(nidx + 16) << 27);
        if (act) ncand += cnt;
        const int cmax = __reduce_max_sync(FULL, cnt);
        // a lane pushes at most one entry per candidate: segments of at most
        // kQueue candidates, flushing first whenever a lane could overflow
        for (int seg = 0; seg < cmax; seg += kQueue) {
          if (__any_sync(FULL, act && qn + min(cnt - seg, kQueue) > kQueue))
            flush_queue<RECORD>(myq, qn, nre, lane, pi, ki, ix, rw, g, pos, posr, pp, acc, q, pair_buf, pair_count,
                                pair_cap, rlist, rcount, err);
          const int send = min(cmax, seg + kQueue);
          for (int jj = seg; jj < send; jj++) {
            const int j = jj < cnt ? b + jj : ki;
            const float4 pj = pos[j];
            const float ddx = pj.x - tx, ddy = pj.y - ty, ddz = pj.z - tz;
            const float r2 = fmaf(ddz, ddz, fmaf(ddy, ddy, ddx * ddx));
            if (act && jj < cnt && r2 < hi) {
              myq[qn][lane] = (unsigned)j | tag | (r2 < lo ? 0u : kBandFlag);
              qn++;
            }
          }
        }
        if (++jx == l1) jx = 0;
      }
    }
    flush_queue<RECORD>(myq, qn, nre, lane, pi, ki, ix, rw, g, pos, posr, pp, acc, q, pair_buf, pair_count, pair_cap,
                        rlist, rcount, err);
    if (act && F) {
      const float *Qm = g->Qf;
      const int oi = __float_as_int(pi.w);
      F[3 * (size_t)oi] = Qm[0] * acc.fx + Qm[1] * acc.fy + Qm[2] * acc.fz;
      F[3 * (size_t)oi + 1] = Qm[3] * acc.fx + Qm[4] * acc.fy + Qm[5] * acc.fz;
      F[3 * (size_t)oi + 2] = Qm[6] * acc.fx + Qm[7] * acc.fy + Qm[8] * acc.fz;
    }
  }
  double v[kPartials] = {acc.u, acc.wxx, acc.wyy, acc.wzz, acc.wxy, acc.wxz, acc.wyz,
                         (double)acc.npair, (double)ncand, (double)nre};
  block_reduce_store<kChunkThreads>(v, partials);
}

// wide: chunks span up to Geo::span cells (the row kernel), else kMaxSpan (the
// grouped and warp kernels, whose queue entries hold the cell offset in 5 bits).
cudaError_t launch_chunk_build(nemd_ctx *c, int gs, bool wide) {
  const int cap = (int)c->cap_cells;
  int64_t blocks = (c->cap_cells + kWalkWarps - 1) / kWalkWarps;
  if (blocks > 16 * (int64_t)c->sms) blocks = 16 * (int64_t)c->sms;
  if (blocks < 1) blocks = 1;
  k_chunk_count<<<(int)blocks, 32 * kWalkWarps, 0, c->stream>>>(c->geo, c->start, c->chunk_cnt, gs, wide);
  cudaError_t e = launch_class_scan(c, c->chunk_cnt, c->chunk_off, cap);
  if (e != cudaSuccess) return e;
  k_chunk_write<<<(int)blocks, 32 * kWalkWarps, 0, c->stream>>>(c->geo, c->start, c->chunk_off, c->chunks, gs,
                                                                 wide);
  c->launches += 2;
  return cudaGetLastError();
}

// Entries hold the partner index in 21 bits, the row in 5 and the offset index
// + 16 in 5: the grouped kernel needs N <= 2^21 and at most 32 rows per class
// (cell factor k <= 2); the caller falls back to the plain kernel otherwise.
bool chunk_kernel_applies(const nemd_ctx *c) { return c->n <= (1 << kJBits) && c->kfac <= 2; }

// Persistent grid: as many blocks as fit on the device at once.
template <int GS, bool RECORD>
static int resident_blocks(int sms) {
  static int per_sm = 0;
  if (!per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_chunk<GS, RECORD>, kChunkThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  return per_sm * sms;
}

cudaError_t launch_force_chunk(nemd_ctx *c, float *F, int *nblocks) {
  const Pot pp = make_pot(c);
  const bool rec = c->record_cap > 0;
  int blocks;
  switch (c->group) {
    case 4: blocks = rec ? resident_blocks<4, true>(c->sms) : resident_blocks<4, false>(c->sms); break;
    case 8: blocks = rec ? resident_blocks<8, true>(c->sms) : resident_blocks<8, false>(c->sms); break;
    case 16: blocks = rec ? resident_blocks<16, true>(c->sms) : resident_blocks<16, false>(c->sms); break;
    default: blocks = rec ? resident_blocks<32, true>(c->sms) : resident_blocks<32, false>(c->sms); break;
  }
  if (blocks > (int)(c->cap_partials - 1)) blocks = (int)(c->cap_partials - 1);
  *nblocks = blocks;
#define NEMD_ARGS                                                                                                \
  c->geo, c->pos4, c->posr, c->cell_sorted, c->start, c->rows, c->rowcnt, c->chunks, c->chunk_off + c->cap_cells, c->q_dev, pp, \
      F, c->partials, c->pair_buf, c->pair_count, (long long)c->record_cap, c->recheck, c->nrecheck, &c->geo->error
#define NEMD_LAUNCH(GS)                                                                              \
  do {                                                                                               \
    if (rec)                                                                                         \
      k_force_chunk<GS, true><<<blocks, kChunkThreads, 0, c->stream>>>(NEMD_ARGS);                   \
    else                                                                                             \
      k_force_chunk<GS, false><<<blocks, kChunkThreads, 0, c->stream>>>(NEMD_ARGS);                  \
  } while (0)
  switch (c->group) {
    case 4: NEMD_LAUNCH(4); break;
    case 8: NEMD_LAUNCH(8); break;
    case 16: NEMD_LAUNCH(16); break;
    default: NEMD_LAUNCH(32); break;
  }
#undef NEMD_LAUNCH
#undef NEMD_ARGS
  c->launches += 1;
  return cudaGetLastError();
}


// ---- batches: chunk lists in a fixed order (count per class slot, scan, write),
// so that the chunk of a particle and every sum are the same from run to run ----

__device__ __forceinline__ bool batch_class(const BatchView &v, int slot, const Geo *&g, int &c0, int &l1) {
  const int s = v.class_sys[slot];
  g = v.geo + s;
  if (g->error & (ERRB_BOX | ERRB_CAPACITY)) return false;
  const SysInfo si = v.sys[s];
  const int cls = slot - si.clo;
  if (cls >= g->nc[1] * g->nc[2]) return false;
  l1 = g->nc[0];
  c0 = si.coff + cls * l1;
  return true;
}

// One thread per class slot: the rows of batched systems are short (a few
// dozen cells) and there are many of them, so each thread walks its own row
// in global memory.  The batched force kernels take chunks from a shared
// counter and write every particle's sums to its own slot, so no result
// depends on where a chunk sits in the list: one kernel builds it, each thread
// walking its row once and keeping the first kChunkBuf chunks in shared
// memory, each warp claiming a contiguous range of the list for its rows'
// chunks with one atomic addition, then writing them (a row with more chunks
// is walked again for the rest).  The list's length ends at
// chunk_off[nclasses], which the force kernels read.
constexpr int kBatchWalkThreads = 128;
constexpr int kChunkBuf = 8;

__global__ void __launch_bounds__(kBatchWalkThreads) k_b_chunk_list(BatchView v) {
  __shared__ int4 cbuf[kChunkBuf][kBatchWalkThreads];
  const int lane = threadIdx.x & 31;
  int *total = v.chunk_off + v.nclasses;
  for (int b0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); b0 < v.nclasses; b0 += gridDim.x * blockDim.x) {
    const int slot = b0 + lane;
    const Geo *g = nullptr;
    int c0 = 0, l1 = 0, n = 0;
    const bool has = slot < v.nclasses && batch_class(v, slot, g, c0, l1);
    const int span = has ? (v.wide ? g->span : kMaxSpan) : 0;
    if (has)
      chunk_walk(v.start, c0, l1, v.gs, span, [&](int first, int count, int ixlo, int ixhi) {
        if (n < kChunkBuf) cbuf[n][threadIdx.x] = make_int4(first, count, slot, ixlo | (ixhi << 16));
        n++;
      });
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int wsum = __shfl_sync(0xffffffffu, incl, 31);
    int wbase = 0;
    if (lane == 0 && wsum > 0) wbase = atomicAdd(total, wsum);
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    const int k = wbase + incl - n;
    for (int j = 0; j < min(n, kChunkBuf); j++) v.chunks[k + j] = cbuf[j][threadIdx.x];
    if (n > kChunkBuf) {
      int j = 0;
      chunk_walk(v.start, c0, l1, v.gs, span, [&](int first, int count, int ixlo, int ixhi) {
        if (j >= kChunkBuf) v.chunks[k + j] = make_int4(first, count, slot, ixlo | (ixhi << 16));
        j++;
      });
    }
  }
}

cudaError_t launch_batch_chunks(cudaStream_t st, const BatchView &v, int sms) {
  int blocks = (v.nclasses + kBatchWalkThreads - 1) / kBatchWalkThreads;
  if (blocks > 16 * sms) blocks = 16 * sms;
  if (blocks < 1) blocks = 1;
  cudaError_t e = cudaMemsetAsync(v.chunk_off + v.nclasses, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_b_chunk_list<<<blocks, kBatchWalkThreads, 0, st>>>(v);
  return cudaGetLastError();
}

}  // namespace nemd
