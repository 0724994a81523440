// bin.cu -- fractional wrap into the unit cell (Sec. 2: the box is the unit cell
// Omega of the lattice) and counting-sort binning of particles in cell order
// (Sec. 3: "each particle is assigned to a cell based off of its position";
// Sec. 4.1: "convert particle positions to the underlying lattice basis";
// Sec. 4.2: rectangular rearrangement of the rotated box).
//
// Pipeline (all O(N), HBM-bound):
//   k_wrap      s = frac(L^-1 q) (FP64), cell index, position relative to the
//               cell centre in the variant's frame as a float32 multiple of the
//               step's quantum plus a float32 residual, rank = atomicAdd(count[cell])
//   k_scan_*    exclusive scan of the per-cell counts -> start[]
//   k_scatter   perm[start[cell] + rank] = i (cells contiguous, arrival order within)
//   k_rankpack  per slot, the particle's place in its cell in increasing kappa
//               (the coordinate along the x-row of cells), ties by input index
//               -- its rank among the cell's particles -- and the sorted
//               float4 {rel position, input index}, {residual, kappa} and cell
//               id written there: the order depends only on the positions, so
//               sums are reproducible from run to run, and every x-row of
//               cells is one kappa-sorted run
#include <math.h>

#include "batch_internal.cuh"
#include "nemd_device.cuh"

namespace nemd {

// One particle: cell_base is the system's first cell slot (0 for a single
// system); the cell index stored in relc.w and counted is cell_base + local.
__device__ __forceinline__ void wrap_body(Geo *g, const double *__restrict__ q, int i, int cell_base,
                                          float4 *__restrict__ relc, float4 *__restrict__ relr,
                                          int *__restrict__ rank, int *__restrict__ count) {
  double x = q[3 * (size_t)i], y = q[3 * (size_t)i + 1], z = q[3 * (size_t)i + 2];
  // NaN or infinity: every exponent bit set (integer test, no float64 work)
  const unsigned long long ex = 0x7ff0000000000000ull;
  if ((__double_as_longlong(x) & ex) == ex || (__double_as_longlong(y) & ex) == ex ||
      (__double_as_longlong(z) & ex) == ex) {
    atomicOr(&g->error, ERRB_NONFINITE);
    x = y = z = 0.0;
  }
  // fractional coordinates in float-float (float64 only for the rare particle
  // within rounding of an integer), the wrapped image exactly the definition's
  double s64[3];
  ff sf[3];
  bool exact;
  float tol[3];
  frac_wrap_ff(g, x, y, z, sf, s64, exact, tol);
  const int l1 = g->nc[0], l2 = g->nc[1], l3 = g->nc[2];
  // Everything after the fractional coordinates runs in float-float (float64
  // throughput is a small fraction of float32 throughput here); the position
  // error stays below g->wrap_tol, which the guard bands and the dynamic offset
  // windows include.
  // position relative to the centre of its cell, in the variant's frame:
  // dynamic size: Cartesian, G (u - 1/2) with u = c s - idx the cell-fractional part
  // (the cell index that of the float64 product c s: taken from float-float
  // unless c s lies within its error bound of a cell face);
  // dynamic offset: the rotated frame, b - (idx + 1/2) w for the brick point b
  int idx[3];
  ff rel[3];
  if (g->variant == NEMD_DS) {
    ff u[3];
    for (int a = 0; a < 3; a++) {
      const float c = (float)g->nc[a];
      const ff t = ff_mul_f(sf[a], c);
      int k;
      const float r = rintf(t.hi);
      const float d = __fadd_rn(__fsub_rn(t.hi, r), t.lo);
      if (!exact && fabsf(d) > 4.0f * c * tol[a]) {
        k = (int)(d < 0.f ? __fsub_rn(r, 1.f) : r);
      } else {
        if (!exact) {
          frac_wrap(g->Linv, x, y, z, s64);
          exact = true;
        }
        k = __double2int_rd(__dmul_rn(s64[a], g->Ginv_scale[a]));
      }
      k = min(max(k, 0), g->nc[a] - 1);
      idx[a] = k;
      u[a] = ff_add(t, ff{-((float)k + 0.5f), 0.f});
    }
    for (int a = 0; a < 3; a++)
      rel[a] = ff_add(ff_add(ff_mul(ff_of(g->Gff[3 * a]), u[0]), ff_mul(ff_of(g->Gff[3 * a + 1]), u[1])),
                      ff_mul(ff_of(g->Gff[3 * a + 2]), u[2]));
  } else {
    ff b[3];
    int m[3];
    brick_wrap_ff(g, sf, b, m);
    for (int a = 0; a < 3; a++) {
      int k = (int)ff_floor(ff_mul(b[a], ff_of(g->Ginvff[a])));
      k = min(max(k, 0), g->nc[a] - 1);
      idx[a] = k;
      rel[a] = ff_add(b[a], ff_neg(ff_mul_f(ff_of(g->wff[a]), (float)k + 0.5f)));
    }
  }
  // split into an exact multiple of the quantum q and a float32 residual:
  // t = rel / q (exact power-of-two scaling), r = nearest integer to t,
  // stored r q (exact) and (t - r) q (t.hi - r exact, one rounding)
  const float qf = g->quantum_f, qif = g->quantum_inv_f;
  float rq[3], rr[3];
  for (int a = 0; a < 3; a++) {
    const float th = __fmul_rn(rel[a].hi, qif), tl = __fmul_rn(rel[a].lo, qif);
    float r = rintf(th);
    const float d = __fadd_rn(__fsub_rn(th, r), tl);
    if (d > 0.5f) r = __fadd_rn(r, 1.f);
    else if (d < -0.5f) r = __fsub_rn(r, 1.f);
    rq[a] = __fmul_rn(r, qf);
    rr[a] = __fmaf_rn(tl, qf, __fmul_rn(__fsub_rn(th, r), qf));
  }
  const int cell = cell_base + idx[0] + l1 * (idx[1] + l2 * idx[2]);
  (void)l3;
  // kappa of the quantised position: the cell-units coordinate along the
  // x-row, in [-1/2, 1/2] inside the cell (the within-cell sort key)
  const float kap = fmaf(g->kap[2], rq[2], fmaf(g->kap[1], rq[1], g->kap[0] * rq[0]));
  relc[i] = make_float4(rq[0], rq[1], rq[2], __int_as_float(cell));
  relr[i] = make_float4(rr[0], rr[1], rr[2], kap);
  rank[i] = atomicAdd(&count[cell], 1);
}

__global__ void k_wrap(Geo *g, const double *__restrict__ q, int n, float4 *__restrict__ relc,
                       float4 *__restrict__ relr, int *__restrict__ rank, int *__restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (g->error & (ERRB_BOX | ERRB_CAPACITY)) return;
  wrap_body(g, q, i, 0, relc, relr, rank, count);
}

// ---- exclusive scan of count[0..ncells) into start[0..ncells], start[ncells] = n ----
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int *sh, int &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  int incl = x + (warp > 0 ? sh[warp - 1] : 0);
  total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return incl - v;
}

// Per tile of kScanTile counts: exclusive scan within the tile, tile total.
__device__ __forceinline__ void scan_tiles_body(const int *__restrict__ count, int *__restrict__ start,
                                                int *__restrict__ tile_sums, int ncells) {
  __shared__ int sh[32];
  const int base = blockIdx.x * kScanTile;
  if (base >= ncells) return;  // whole block uniform
  int v[kScanItems];
  int sum = 0;
  for (int k = 0; k < kScanItems; k++) {
    int idx = base + threadIdx.x * kScanItems + k;
    v[k] = (idx < ncells) ? count[idx] : 0;
    sum += v[k];
  }
  int total;
  int ex = block_exclusive_scan(sum, sh, total);
  for (int k = 0; k < kScanItems; k++) {
    int idx = base + threadIdx.x * kScanItems + k;
    if (idx < ncells) start[idx] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const Geo *g, const int *__restrict__ count,
                                                             int *__restrict__ start, int *__restrict__ tile_sums) {
  if (g->error & (ERRB_BOX | ERRB_CAPACITY)) return;
  scan_tiles_body(count, start, tile_sums, g->ncells);
}

// One block: exclusive scan of the tile totals; returns the grand total.
__device__ __forceinline__ int scan_top_body(int *__restrict__ tile_sums, int ntiles) {
  __shared__ int sh[32];
  int carry = 0;
  for (int base = 0; base < ntiles; base += kScanThreads) {
    int idx = base + threadIdx.x;
    int v = (idx < ntiles) ? tile_sums[idx] : 0;
    int total;
    int ex = block_exclusive_scan(v, sh, total);
    if (idx < ntiles) tile_sums[idx] = ex + carry;
    carry += total;
  }
  return carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(const Geo *g, int *__restrict__ tile_sums) {
  if (g->error & (ERRB_BOX | ERRB_CAPACITY)) return;
  scan_top_body(tile_sums, (g->ncells + kScanTile - 1) / kScanTile);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(const Geo *g, int *__restrict__ start,
                                                           const int *__restrict__ tile_sums, int n) {
  if (g->error & (ERRB_BOX | ERRB_CAPACITY)) return;
  const int ncells = g->ncells;
  const int base = blockIdx.x * kScanTile;
  if (base > ncells) return;
  const int add = tile_sums[blockIdx.x];
  for (int k = 0; k < kScanItems; k++) {
    int idx = base + threadIdx.x * kScanItems + k;
    if (idx < ncells) start[idx] += add;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) start[ncells] = n;
}

// perm[start[cell] + rank] = i.
__device__ __forceinline__ void scatter_body(const float4 *__restrict__ relc, const int *__restrict__ rank,
                                             const int *__restrict__ start, int *__restrict__ perm, int i) {
  const int cell = __float_as_int(relc[i].w);
  perm[start[cell] + rank[i]] = i;
}

__global__ void k_scatter(const Geo *g, const float4 *__restrict__ relc, const int *__restrict__ rank,
                          const int *__restrict__ start, int *__restrict__ perm, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (g->error & (ERRB_BOX | ERRB_CAPACITY)) return;
  scatter_body(relc, rank, start, perm, i);
}

// (kappa, input index) of particle i: the within-cell order, a strict total
// order (input indices are distinct).
__device__ __forceinline__ bool sort_before(float ka, int ia, float kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// Scattered slot u (cells contiguous, arrival order within a cell): particle
// i = perm[u] goes to slot start[c] + (number of the cell's particles that sort
// before it), which over the cell is a permutation of its slots -- the order
// of a sort of the cell by (kappa, input index).  There it is packed: float4
// {rel position, input index}, {residual, kappa} and its cell id.  A block of
// kRankThreads threads takes kRankThreads consecutive slots and first puts its
// slots' keys (input index and kappa, the latter relr[perm[v]].w) in shared
// memory: each thread then reads the keys of its cell's slots there, and only
// a cell that crosses the block's range reads the rest of its keys from
// global memory.
constexpr int kRankThreads = 256;

// valid: the block's slot u = blockIdx.x * kRankThreads + threadIdx.x holds a
// binned particle.
__device__ __forceinline__ void rankpack_block(const float4 *__restrict__ relc, const float4 *__restrict__ relr,
                                               const int *__restrict__ perm, const int *__restrict__ start,
                                               float4 *__restrict__ pos4, float4 *__restrict__ posr,
                                               int *__restrict__ cell_sorted, bool valid) {
  __shared__ int sidx[kRankThreads];
  __shared__ float skap[kRankThreads];
  const int u0 = blockIdx.x * kRankThreads;
  const int u = u0 + threadIdx.x;
  const int i = valid ? perm[u] : 0;
  const float4 rr = valid ? relr[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  sidx[threadIdx.x] = i;
  skap[threadIdx.x] = rr.w;
  __syncthreads();
  if (!valid) return;
  const float4 r = relc[i];
  const int c = __float_as_int(r.w);
  const int b = start[c], e = start[c + 1];
  const float *kap = reinterpret_cast<const float *>(relr) + 3;  // kappa of particle j: kap[4 j]
  // the cell's slots in this block: [lo, hi), which holds slot u
  const int lo = max(b, u0), hi = min(e, u0 + kRankThreads);
  int k = b;
  for (int v = b; v < lo; v++) {
    const int iv = perm[v];
    k += sort_before(__ldg(kap + 4 * (size_t)iv), iv, rr.w, i);
  }
  int v = lo;
  for (; v + 4 <= hi; v += 4) {
#pragma unroll
    for (int h = 0; h < 4; h++) k += sort_before(skap[v + h - u0], sidx[v + h - u0], rr.w, i);
  }
  for (; v < hi; v++) k += sort_before(skap[v - u0], sidx[v - u0], rr.w, i);
  for (v = hi; v < e; v++) {
    const int iv = perm[v];
    k += sort_before(__ldg(kap + 4 * (size_t)iv), iv, rr.w, i);
  }
  pos4[k] = make_float4(r.x, r.y, r.z, __int_as_float(i));
  posr[k] = rr;
  cell_sorted[k] = c;
}

__global__ void __launch_bounds__(kRankThreads) k_rankpack(const Geo *g, const float4 *__restrict__ relc,
                                                           const float4 *__restrict__ relr,
                                                           const int *__restrict__ perm, const int *__restrict__ start,
                                                           float4 *__restrict__ pos4, float4 *__restrict__ posr,
                                                           int *__restrict__ cell_sorted, int n) {
  if (g->error & (ERRB_BOX | ERRB_CAPACITY)) return;
  rankpack_block(relc, relr, perm, start, pos4, posr, cell_sorted, blockIdx.x * kRankThreads + threadIdx.x < n);
}

cudaError_t launch_bin(nemd_ctx *c) {
  const int n = (int)c->n;
  cudaError_t e = cudaMemsetAsync(c->count, 0, sizeof(int) * (size_t)(c->cap_cells + 1), c->stream);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    const int tb = 256;
    const int nb = (n + tb - 1) / tb;
    k_wrap<<<nb, tb, 0, c->stream>>>(c->geo, c->q_dev, n, c->relc, c->relr, c->rank, c->count);
    c->launches += 1;
  }
  const int64_t tiles = (c->cap_cells + 1 + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<(int)tiles, kScanThreads, 0, c->stream>>>(c->geo, c->count, c->start, c->block_sums);
  k_scan_top<<<1, kScanThreads, 0, c->stream>>>(c->geo, c->block_sums);
  k_scan_add<<<(int)tiles, kScanThreads, 0, c->stream>>>(c->geo, c->start, c->block_sums, n);
  c->launches += 3;
  if (n > 0) {
    const int tb = 256;
    const int nb = (n + tb - 1) / tb;
    k_scatter<<<nb, tb, 0, c->stream>>>(c->geo, c->relc, c->rank, c->start, c->perm, n);
    k_rankpack<<<(n + kRankThreads - 1) / kRankThreads, kRankThreads, 0, c->stream>>>(
        c->geo, c->relc, c->relr, c->perm, c->start, c->pos4, c->posr, c->cell_sorted, n);
    c->launches += 2;
  }
  return cudaGetLastError();
}


// ---- one-block scan of the per-class chunk counts ----
// out[0..ncls) exclusive prefix sums of in[0..ncls), ncls = c2 c3 classes read
// from the grid (0 after a box or capacity error), and the total at out[cap],
// where the force kernels read the number of chunks.
__global__ void __launch_bounds__(kScanThreads) k_fscan_classes(const Geo *g, const int *__restrict__ in,
                                                                int *__restrict__ out, int cap) {
  __shared__ int sh[32];
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  const int len = ok ? g->nc[1] * g->nc[2] : 0;
  int carry = 0;
  for (int base = 0; base < len; base += kScanTile) {
    int v[kScanItems];
    int sum = 0;
    for (int k = 0; k < kScanItems; k++) {
      const int idx = base + threadIdx.x * kScanItems + k;
      v[k] = (idx < len) ? in[idx] : 0;
      sum += v[k];
    }
    int total;
    int ex = block_exclusive_scan(sum, sh, total) + carry;
    for (int k = 0; k < kScanItems; k++) {
      const int idx = base + threadIdx.x * kScanItems + k;
      if (idx < len) out[idx] = ex;
      ex += v[k];
    }
    carry += total;
  }
  if (threadIdx.x == 0) out[cap] = carry;
}

cudaError_t launch_class_scan(nemd_ctx *c, const int *in, int *out, int cap) {
  k_fscan_classes<<<1, kScanThreads, 0, c->stream>>>(c->geo, in, out, cap);
  c->launches += 1;
  return cudaGetLastError();
}

// ---- batches: every system's particles in one launch per stage ----

__global__ void k_b_wrap(BatchView v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.ntot) return;
  const int s = v.sys_of[i];
  Geo *g = v.geo + s;
  if (g->error & (ERRB_BOX | ERRB_CAPACITY)) return;
  wrap_body(g, v.q, i, v.sys[s].coff, v.relc, v.relr, v.rank, v.count);
}

__global__ void k_b_scatter(BatchView v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.ntot) return;
  if (v.geo[v.sys_of[i]].error & (ERRB_BOX | ERRB_CAPACITY)) return;
  scatter_body(v.relc, v.rank, v.start, v.perm, i);
}

// One block per system: the exclusive scan of the counts of its cells
// j < ncells into start[coff + j], from the base poff (system s's particles
// take the sorted slots [poff, poff + n), as in the input), and
// start[coff + ncells] = poff + n.  Only the cells of the step's grid are read
// (a system's cell slots are sized for the largest cell factor); a system that
// failed this step binned nothing, and no kernel reads its cells.
__global__ void __launch_bounds__(kScanThreads) k_b_scan_cells(BatchView v) {
  __shared__ int sh[32];
  const Geo *g = v.geo + blockIdx.x;
  if (g->error & (ERRB_BOX | ERRB_CAPACITY)) return;
  const SysInfo si = v.sys[blockIdx.x];
  const int len = g->ncells;
  const int *in = v.count + si.coff;
  int *out = v.start + si.coff;
  int carry = si.poff;
  for (int base = 0; base < len; base += kScanTile) {
    int c[kScanItems];
    int sum = 0;
    for (int k = 0; k < kScanItems; k++) {
      const int idx = base + threadIdx.x * kScanItems + k;
      c[k] = (idx < len) ? in[idx] : 0;
      sum += c[k];
    }
    int total;
    int ex = block_exclusive_scan(sum, sh, total) + carry;
    for (int k = 0; k < kScanItems; k++) {
      const int idx = base + threadIdx.x * kScanItems + k;
      if (idx < len) out[idx] = ex;
      ex += c[k];
    }
    carry += total;
  }
  if (threadIdx.x == 0) out[len] = carry;
}

// Sorted slots of every system that binned (the slots of a system that failed
// this step hold nothing).
__global__ void __launch_bounds__(kRankThreads) k_b_rankpack(BatchView v) {
  const int u = blockIdx.x * kRankThreads + threadIdx.x;
  const bool valid = u < v.ntot && !(v.geo[v.sys_of[u]].error & (ERRB_BOX | ERRB_CAPACITY));
  rankpack_block(v.relc, v.relr, v.perm, v.start, v.pos4, v.posr, v.cell_sorted, valid);
}

cudaError_t launch_batch_bin(cudaStream_t st, const BatchView &v, int sms) {
  cudaError_t e = cudaMemsetAsync(v.count, 0, sizeof(int) * ((size_t)v.ncells + 1), st);
  if (e != cudaSuccess) return e;
  const int tb = 256;
  const int nb = v.ntot > 0 ? (v.ntot + tb - 1) / tb : 1;
  k_b_wrap<<<nb, tb, 0, st>>>(v);
  k_b_scan_cells<<<v.nsys > 0 ? v.nsys : 1, kScanThreads, 0, st>>>(v);
  k_b_scatter<<<nb, tb, 0, st>>>(v);
  k_b_rankpack<<<v.ntot > 0 ? (v.ntot + kRankThreads - 1) / kRankThreads : 1, kRankThreads, 0, st>>>(v);
  (void)sms;
  return cudaGetLastError();
}

}  // namespace nemd
