// force.cu -- cell-pair force, energy and virial (Sec. 3: only the 27 cells of a
// neighbourhood are searched; Sec. 5: every force evaluation is preceded by a
// distance check), the plain force kernel, and the deterministic float64
// reductions shared by every force kernel.
//
// Plain kernel: one thread per particle in cell order.  The thread walks the
// rows of its home cell's stencil (Sec. 4.1: 27 cells; Sec. 4.2: 27-36 cells),
// each row a run of consecutive x-cells, and tests every particle of every
// cell with a float32 distance check on quantised cell-centred coordinates
// (exact in float32).  Candidates near the cut-off are re-tested with the
// residuals added back, and the few still within rounding of rc are decided
// by the canonical float64 displacement, so the pair set is exactly the
// definition's.  Full neighbourhoods: each unordered pair is met from both
// sides, every particle's force is accumulated by its own thread, and U, W are
// halved.
#include <math.h>

#include "batch_internal.cuh"

namespace nemd {

template <int NT, bool RECORD, bool PRECISE>
__global__ void __launch_bounds__(NT) k_force_plain(const Geo *__restrict__ g, const float4 *__restrict__ pos,
                                                    const float4 *__restrict__ posr,
                                                    const int *__restrict__ cell_sorted,
                                                    const int *__restrict__ start, const Row *__restrict__ rows,
                                                    const int *__restrict__ rowcnt, const double *__restrict__ q,
                                                    int n, Pot pp, float *__restrict__ F,
                                                    double *__restrict__ partials, int32_t *__restrict__ pair_buf,
                                                    unsigned long long *__restrict__ pair_count, long long pair_cap,
                                                    int4 *__restrict__ rlist, int *__restrict__ rcount,
                                                    int *__restrict__ err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  Acc acc;
  acc.zero();
  double du = 0, dfx = 0, dfy = 0, dfz = 0, dwxx = 0, dwyy = 0, dwzz = 0, dwxy = 0, dwxz = 0, dwyz = 0;
  int ncand = 0, nre = 0;
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  if (ok && k < n) {
    const float4 pi = pos[k];
    const float4 pir = posr[k];
    const int oi = __float_as_int(pi.w);
    const int cell = cell_sorted[k];
    const int l1 = g->nc[0], l2 = g->nc[1];
    const int ix = cell % l1, rest = cell / l1, iy = rest % l2, iz = rest / l2;
    const int cls = iy + l2 * iz;
    const Row *rw = rows + (size_t)cls * g->maxrows;
    const int nr = rowcnt[cls];
    const float lo = g->rc2_lo, hi = g->rc2_hi, lo2 = g->rc2_lo2, hi2 = g->rc2_hi2;
    const float sx = g->step[0], sy = g->step[1], sz = g->step[2];
    const float srx = g->step_r[0], sry = g->step_r[1], srz = g->step_r[2];
    for (int r = 0; r < nr; r++) {
      const Row R = rw[r];
      const int jxu = ix + R.dxlo;
      int kx = floordiv_dev(jxu, l1);
      int jx = jxu - kx * l1;
      for (int m = 0; m < R.cnt; m++) {
        const int nidx = R.dxlo + m + R.sxi;
        // t = x_i - o exactly (quantised); T = residual of x_i - o
        const float tx = sub_offset(pi.x, R.shx, nidx, sx), ty = sub_offset(pi.y, R.shy, nidx, sy),
                    tz = sub_offset(pi.z, R.shz, nidx, sz);
        const float Tx = sub_residual(pir.x, R.srx, nidx, srx), Ty = sub_residual(pir.y, R.sry, nidx, sry),
                    Tz = sub_residual(pir.z, R.srz, nidx, srz);
        const int c = R.cbase + jx;
        const int b = start[c], e = start[c + 1];
        ncand += e - b;
        for (int j = b; j < e; j++) {
          const float4 pj = pos[j];
          const float dx = pj.x - tx, dy = pj.y - ty, dz = pj.z - tz;
          const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          if (r2 < hi) {
            if (j == k && kx == 0 && R.ky == 0 && R.kz == 0) continue;
            const int oj = __float_as_int(pj.w);
            // residuals added back: d to one rounding of d itself
            const float4 pjr = posr[j];
            const float cx = dx + (pjr.x - Tx), cy = dy + (pjr.y - Ty), cz = dz + (pjr.z - Tz);
            bool accept = r2 < lo;
            if (!accept) {
              nre++;
              const float r2c = fmaf(cz, cz, fmaf(cy, cy, cx * cx));
              accept = r2c < lo2;
              if (!accept && r2c < hi2) {
                if (RECORD || PRECISE)
                  accept = guard_band_accept(g, q, oi, oj, kx, R.ky, R.kz);
                else
                  defer_recheck(rlist, rcount, err, k, j, kx, R.ky, R.kz);  // decided by the fix-up pass
              }
            }
            if (!accept) continue;
            if (PRECISE) {
              int nn[3];
              pair_image(g, q, oi, oj, kx, R.ky, R.kz, nn);
              double dd[3];
              const double cr2 = canon_r2(g, q, oi, oj, nn[0], nn[1], nn[2], dd);
              const double inv = 1.0 / cr2;
              const double s2 = pp.sig2d * inv;
              const double s6 = s2 * s2 * s2;
              const double fr = pp.eps24d * inv * s6 * (2.0 * s6 - 1.0);
              du += pp.eps4d * s6 * (s6 - 1.0) - pp.ushiftd;
              dfx -= fr * dd[0];
              dfy -= fr * dd[1];
              dfz -= fr * dd[2];
              dwxx += fr * dd[0] * dd[0];
              dwyy += fr * dd[1] * dd[1];
              dwzz += fr * dd[2] * dd[2];
              dwxy += fr * dd[0] * dd[1];
              dwxz += fr * dd[0] * dd[2];
              dwyz += fr * dd[1] * dd[2];
              acc.npair++;
            } else {
              acc.add(pp, cx, cy, cz);
            }
            if (RECORD) record_pair(g, q, oi, oj, kx, R.ky, R.kz, pair_buf, pair_count, pair_cap);
          }
        }
        if (++jx == l1) {
          jx = 0;
          kx++;
        }
      }
    }
    if (F) {
      float ox, oy, oz;
      if (PRECISE) {
        ox = (float)dfx;
        oy = (float)dfy;
        oz = (float)dfz;
      } else {
        const float *Qm = g->Qf;
        ox = Qm[0] * acc.fx + Qm[1] * acc.fy + Qm[2] * acc.fz;
        oy = Qm[3] * acc.fx + Qm[4] * acc.fy + Qm[5] * acc.fz;
        oz = Qm[6] * acc.fx + Qm[7] * acc.fy + Qm[8] * acc.fz;
      }
      F[3 * (size_t)oi] = ox;
      F[3 * (size_t)oi + 1] = oy;
      F[3 * (size_t)oi + 2] = oz;
    }
  }
  double v[kPartials];
  if (PRECISE) {
    v[0] = du;
    v[1] = dwxx;
    v[2] = dwyy;
    v[3] = dwzz;
    v[4] = dwxy;
    v[5] = dwxz;
    v[6] = dwyz;
  } else {
    v[0] = acc.u;
    v[1] = acc.wxx;
    v[2] = acc.wyy;
    v[3] = acc.wzz;
    v[4] = acc.wxy;
    v[5] = acc.wxz;
    v[6] = acc.wyz;
  }
  v[7] = acc.npair;
  v[8] = ncand;
  v[9] = nre;
  block_reduce_store<NT>(v, partials);
}

// Publishes the totals sh0 (the fixed-order sums of every block's partials):
// halves the full-neighbourhood double count, rotates the virial of the
// dynamic offset frame back to Cartesian (W = Q W_R Q^T), writes U, W and the
// counters.  One thread.
__device__ __forceinline__ void publish_uw(Geo *__restrict__ g, const double (&sh0)[kPartials],
                                          int frame_is_cartesian, double *__restrict__ uw,
                                          unsigned long long *__restrict__ counters, double hf) {
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  // hf: 1/2 for full neighbourhoods (every pair met from both sides), 1 for half
  double U = hf * sh0[0];
  double Wr[9];
  Wr[0] = hf * sh0[1];
  Wr[4] = hf * sh0[2];
  Wr[8] = hf * sh0[3];
  Wr[1] = Wr[3] = hf * sh0[4];
  Wr[2] = Wr[6] = hf * sh0[5];
  Wr[5] = Wr[7] = hf * sh0[6];
  double W[9];
  if (!frame_is_cartesian && g->variant == NEMD_DO) {
    double T9[9];
    const double *Q = g->Q;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) T9[3 * a + b] = Q[3 * a] * Wr[b] + Q[3 * a + 1] * Wr[3 + b] + Q[3 * a + 2] * Wr[6 + b];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++)
        W[3 * a + b] = T9[3 * a] * Q[3 * b] + T9[3 * a + 1] * Q[3 * b + 1] + T9[3 * a + 2] * Q[3 * b + 2];
  } else {
    for (int k = 0; k < 9; k++) W[k] = Wr[k];
  }
  uw[0] = ok ? U : 0.0;
  for (int k = 0; k < 9; k++) uw[1 + k] = ok ? W[k] : 0.0;
  counters[0] = (unsigned long long)(hf * sh0[7] + 0.25);
  counters[1] = (unsigned long long)(sh0[8] + 0.5);
  counters[2] = (unsigned long long)(sh0[9] + 0.5);
  g->sticky |= g->error;
}

// Fixed-point scales of the fix-up's sums (per unit of eps): every deferred
// pair lies within float32 rounding of rc, where |u| / eps and |r f| / eps are
// O(1) for any rc >= 0.3 sigma, far inside 2^23 (energy, virial) and 2^31
// (force) at these scales; the roundings (2^-41, 2^-33 per pair) are far
// below float32.  Integer sums do not depend on the order of the additions.
constexpr double kFixUW = 1099511627776.0;   // 2^40
constexpr double kFixF = 4294967296.0;       // 2^32

__device__ __forceinline__ unsigned long long to_fix(double x, double scale) {
  return (unsigned long long)__double2ll_rn(x * scale);
}
__device__ __forceinline__ double from_fix(unsigned long long x, double iscale) {
  return (double)(long long)x * iscale;
}

// Float64 fix-up of the candidates the force kernels left within float32
// rounding of rc: the canonical decision (Sec. 2 images, strict r < rc), and for
// each accepted pair the force on i (Cartesian), half of u and of r (x) f (the
// other half comes from the pair's other orientation, which the full
// neighbourhood also defers), in the variant's frame.  The force kernels append
// the candidates in no fixed order, so their sums are formed in 64-bit fixed
// point (exact, order-free): U, W and the pair count summed over all blocks in
// fix_uw, forces per particle in fix_f; the last block converts each total
// once (adding U and W to the force kernel's partials, summed in block order,
// and each particle's force to F), taking it by an atomic exchange that also
// returns the scratch to zero.  Runs after the force kernel.
__global__ void __launch_bounds__(256) k_recheck_fixup(Geo *__restrict__ g, const int4 *__restrict__ list,
                                                       const int *__restrict__ count, const float4 *__restrict__ pos,
                                                       const double *__restrict__ q, Pot pp, float *__restrict__ F,
                                                       unsigned long long *__restrict__ fix_f,
                                                       unsigned long long *__restrict__ fix_uw,
                                                       double *__restrict__ partials, int nforce, int half,
                                                       int frame_is_cartesian, double *__restrict__ uw,
                                                       unsigned long long *__restrict__ counters) {
  double *partial_slot = partials + (size_t)nforce * kPartials;
  double v[kPartials];
  for (int k = 0; k < kPartials; k++) v[k] = 0.0;
  unsigned long long vf[8] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};  // U, W (6), pairs
  const double ie = 1.0 / pp.eps4d * 4.0;  // 1 / eps
  const int n = min(*count, kRecheckCap);
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  // entries dealt round robin over the blocks, so that their float64 work
  // (a small fraction of the float32 rate here) spreads over as many SMs
  bool has = false;
  for (int e = blockIdx.x + gridDim.x * threadIdx.x; ok && e < n; e += gridDim.x * blockDim.x) {
    has = true;
    const int4 it = list[e];
    const int oi = __float_as_int(pos[it.x].w), oj = __float_as_int(pos[it.y].w);
    const int ky = (short)(it.w & 0xffff), kz = it.w >> 16;
    int nn[3];
    pair_image(g, q, oi, oj, it.z, ky, kz, nn);
    double d[3];
    const double r2 = canon_r2(g, q, oi, oj, nn[0], nn[1], nn[2], d);
    if (!(r2 < g->rc2)) continue;
    const double inv = 1.0 / r2, s2 = pp.sig2d * inv, s6 = s2 * s2 * s2;
    const double fr = pp.eps24d * inv * s6 * (2.0 * s6 - 1.0);
    if (F && fix_f)
      for (int a = 0; a < 3; a++) {
        atomicAdd(&fix_f[3 * (size_t)oi + a], to_fix(-fr * d[a] * ie, kFixF));
        // half neighbourhoods defer only one orientation of the pair
        if (half) atomicAdd(&fix_f[3 * (size_t)oj + a], to_fix(fr * d[a] * ie, kFixF));
      }
    // frame components: W_frame = Q^T (d d^T) Q fr, d_frame = Q^T d
    double df[3];
    for (int a = 0; a < 3; a++) df[a] = g->Q[a] * d[0] + g->Q[3 + a] * d[1] + g->Q[6 + a] * d[2];
    if (g->variant != NEMD_DO)
      for (int a = 0; a < 3; a++) df[a] = d[a];
    vf[0] += to_fix((pp.eps4d * s6 * (s6 - 1.0) - pp.ushiftd) * ie, kFixUW);
    vf[1] += to_fix(fr * df[0] * df[0] * ie, kFixUW);
    vf[2] += to_fix(fr * df[1] * df[1] * ie, kFixUW);
    vf[3] += to_fix(fr * df[2] * df[2] * ie, kFixUW);
    vf[4] += to_fix(fr * df[0] * df[1] * ie, kFixUW);
    vf[5] += to_fix(fr * df[0] * df[2] * ie, kFixUW);
    vf[6] += to_fix(fr * df[1] * df[2] * ie, kFixUW);
    vf[7] += 1ull;
  }
  // Block sum, in a fixed order: the warps' entry sums, then this block's slice
  // of the force kernel's partials (rows b, b + G, b + 2G, ..., G = gridDim.x;
  // thread t < 10 P sums value t % 10 of slice rows p, p + P, ... with p = t / 10).
  constexpr int P = 24;
  __shared__ double shw[256 / 32][kPartials];
  __shared__ double shp[P][kPartials];
  __shared__ unsigned long long shf[256 / 32][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool any = __any_sync(0xffffffffu, has);
#pragma unroll
  for (int k = 0; k < kPartials; k++) {
    if (lane == 0) shw[warp][k] = 0.0;
  }
#pragma unroll
  for (int k = 0; k < 8; k++) {
    unsigned long long x = vf[k];
    if (any) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    }
    if (lane == 0) shf[warp][k] = any ? x : 0ull;
  }
  if (threadIdx.x < P * kPartials) {
    const int k = threadIdx.x % kPartials, pp0 = threadIdx.x / kPartials;
    const int G = gridDim.x;
    double x = 0.0;
    for (int r = blockIdx.x + G * pp0; r < nforce; r += G * P) x += __ldcg(&partials[(size_t)r * kPartials + k]);
    shp[pp0][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    // the deferred pairs' fixed-point sums, added exactly to the totals of all blocks
    unsigned long long f = 0ull;
    for (int w = 0; w < 256 / 32; w++) f += shf[w][threadIdx.x];
    if (f) atomicAdd(&fix_uw[threadIdx.x], f);
  }
  if (threadIdx.x < kPartials) {
    // this block's slice of the force partials in a fixed order
    double x = 0.0;
    for (int w = 0; w < 256 / 32; w++) x += shw[w][threadIdx.x];
    for (int p = 0; p < P; p++) x += shp[p][threadIdx.x];
    partial_slot[(size_t)blockIdx.x * kPartials + threadIdx.x] = x;
  }
  // The last block to finish (ticket in counters[3], returned to zero) adds the
  // blocks' sums in block order and publishes U, W and the counters.
  __shared__ bool last;
  __shared__ double tot[kPartials];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&counters[3], 1ull) == (unsigned long long)(gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // each deferred particle's fixed-point force total, taken once and added to F
  if (F && fix_f && ok) {
    const double eps = pp.eps4d * 0.25;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int4 it = list[e];
      const int ps[2] = {__float_as_int(pos[it.x].w), __float_as_int(pos[it.y].w)};
      for (int h = 0; h < (half ? 2 : 1); h++)
        for (int a = 0; a < 3; a++) {
          const unsigned long long x = atomicExch(&fix_f[3 * (size_t)ps[h] + a], 0ull);
          if (x) F[3 * (size_t)ps[h] + a] += (float)(from_fix(x, 1.0 / kFixF) * eps);
        }
    }
  }
  if (threadIdx.x < kPartials) {
    double x = 0.0;
    for (int b = 0; b < (int)gridDim.x; b++) x += __ldcg(&partial_slot[(size_t)b * kPartials + threadIdx.x]);
    // then the deferred pairs' exact totals, each converted once
    if (threadIdx.x < 8) {
      const unsigned long long f = atomicExch(&fix_uw[threadIdx.x], 0ull);
      x += threadIdx.x < 7 ? from_fix(f, 1.0 / kFixUW) * (pp.eps4d * 0.25) : (double)(long long)f;
    }
    tot[threadIdx.x] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sh0[kPartials];
    for (int k = 0; k < kPartials; k++) sh0[k] = tot[k];
    publish_uw(g, sh0, frame_is_cartesian, uw, counters, half ? 1.0 : 0.5);
    counters[3] = 0ull;
  }
}

Pot make_pot(const nemd_ctx *c) {
  Pot p;
  double eps = c->eps, sig = c->sigma, rc = c->rc;
  double ush = 0.0;
  if (c->shift) {
    double sr2 = (sig * sig) / (rc * rc);
    double sr6 = sr2 * sr2 * sr2;
    ush = 4.0 * eps * (sr6 * sr6 - sr6);
  }
  p.eps4d = 4.0 * eps;
  p.eps24d = 24.0 * eps;
  p.sig2d = sig * sig;
  p.ushiftd = ush;
  p.eps4 = (float)p.eps4d;
  p.eps24 = (float)p.eps24d;
  p.sig2 = (float)p.sig2d;
  p.ushift = (float)ush;
  return p;
}


template <int NT>
static void launch_plain(nemd_ctx *c, int nblocks, Pot pp, float *F) {
  const bool rec = c->record_cap > 0;
  const bool pre = c->precise != 0;
  const int n = (int)c->n;
#define NEMD_ARGS                                                                                               \
  c->geo, c->pos4, c->posr, c->cell_sorted, c->start, c->rows, c->rowcnt, c->q_dev, n, pp, F, c->partials, \
      c->pair_buf, c->pair_count, (long long)c->record_cap, c->recheck, c->nrecheck, &c->geo->error
  if (rec && pre)
    k_force_plain<NT, true, true><<<nblocks, NT, 0, c->stream>>>(NEMD_ARGS);
  else if (rec)
    k_force_plain<NT, true, false><<<nblocks, NT, 0, c->stream>>>(NEMD_ARGS);
  else if (pre)
    k_force_plain<NT, false, true><<<nblocks, NT, 0, c->stream>>>(NEMD_ARGS);
  else
    k_force_plain<NT, false, false><<<nblocks, NT, 0, c->stream>>>(NEMD_ARGS);
#undef NEMD_ARGS
  c->launches += 1;
}

cudaError_t launch_forces(nemd_ctx *c, float *F_dev, double *UW_dev) {
  if (c->record_cap > 0) {
    cudaError_t e = cudaMemsetAsync(c->pair_count, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
  }
  {
    cudaError_t e = cudaMemsetAsync(c->nrecheck, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
  }
  // the grouped and warp kernels have no precise pair path: precise mode runs the
  // plain kernel for them (the row kernel has its own float-float path); pair
  // records take the full-neighbourhood warp kernel
  const bool grouped = c->kernel == 1 && !c->precise && chunk_kernel_applies(c);
  const bool warped = (c->kernel == 2 || c->kernel == 3) && !c->precise && warp_kernel_applies(c);
  const bool rowk = c->kernel == 4 && row_kernel_applies(c);
  const bool half = warped && c->kernel == 3 && c->record_cap == 0;
  if (half && F_dev && c->n > 0) {
    // half neighbourhoods add the partners' forces with atomics: start from zero
    cudaError_t e = cudaMemsetAsync(F_dev, 0, sizeof(float) * 3 * (size_t)c->n, c->stream);
    if (e != cudaSuccess) return e;
  }
  if (grouped || warped || rowk) {
    cudaError_t e = launch_chunk_build(c, (warped || rowk) ? 32 : c->group, rowk);
    if (e != cudaSuccess) return e;
  }
  const bool timed = c->timing && c->ev && c->ev_n < c->ev_cap;
  if (timed) cudaEventRecord(c->ev[2 * c->ev_n], c->stream);
  int nblocks;
  if (rowk) {
    cudaError_t e = launch_force_row(c, F_dev, &nblocks);
    if (e != cudaSuccess) return e;
  } else if (warped) {
    cudaError_t e = launch_force_warp(c, F_dev, &nblocks, half);
    if (e != cudaSuccess) return e;
  } else if (grouped) {
    cudaError_t e = launch_force_chunk(c, F_dev, &nblocks);
    if (e != cudaSuccess) return e;
  } else {
    const int NT = 128;
    nblocks = (int)((c->n + NT - 1) / NT);
    if (nblocks < 1) nblocks = 1;
    launch_plain<NT>(c, nblocks, make_pot(c), F_dev);
  }
  if (timed) {
    cudaEventRecord(c->ev[2 * c->ev_n + 1], c->stream);
    c->ev_n++;
  }
  return launch_recheck_fixup(c, F_dev, UW_dev, nblocks, half, c->precise && !rowk);
}

// The deferred float64 decisions, as a few more blocks of partials after the
// force kernel's nblocks (at least one slot is always left), and the totals.
cudaError_t launch_recheck_fixup(nemd_ctx *c, float *F_dev, double *UW_dev, int nblocks, bool half,
                                 bool frame_is_cartesian) {
  int nfix = kFixupBlocks;
  if (nblocks + nfix > c->cap_partials) nfix = (int)(c->cap_partials - nblocks);
  if (!c->fix_uw) {
    cudaError_t e = cudaMalloc((void **)&c->fix_uw, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->fix_uw, 0, 8 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
  }
  if (F_dev && c->fix_cap < c->n) {
    // the fixed-point force scratch, zero from the start (the fix-up returns
    // every slot it touches to zero)
    if (c->fix_f) cudaFree(c->fix_f);
    c->fix_f = nullptr;
    c->fix_cap = 0;
    const size_t bytes = sizeof(unsigned long long) * 3 * (size_t)std::max<int64_t>(c->n, 1);
    cudaError_t e = cudaMalloc((void **)&c->fix_f, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->fix_f, 0, bytes, c->stream);
    if (e != cudaSuccess) return e;
    c->fix_cap = c->n;
  }
  k_recheck_fixup<<<nfix, 256, 0, c->stream>>>(c->geo, c->recheck, c->nrecheck, c->pos4, c->q_dev, make_pot(c),
                                               F_dev, F_dev ? c->fix_f : nullptr, c->fix_uw, c->partials, nblocks,
                                               half ? 1 : 0,
                                               frame_is_cartesian ? 1 : 0, UW_dev, c->counters);
  c->launches += 1;
  return cudaGetLastError();
}


// ---- batches ----

// Float64 fix-up of the deferred candidates of every system (as
// k_recheck_fixup); the accepted pair terms go to the particle's own sums.
__global__ void k_b_fixup(BatchView v) {
  const int n = min(*v.nrecheck, kRecheckCap);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int4 it = v.recheck[e];
    const int oi = __float_as_int(v.pos4[it.x].w), oj = __float_as_int(v.pos4[it.y].w);
    const int s = v.sys_of[oi];
    const Geo *g = v.geo + s;
    const int ky = (short)(it.w & 0xffff), kz = it.w >> 16;
    int nn[3];
    pair_image(g, v.q, oi, oj, it.z, ky, kz, nn);
    double d[3];
    const double r2 = canon_r2(g, v.q, oi, oj, nn[0], nn[1], nn[2], d);
    if (!(r2 < g->rc2)) continue;
    const Pot pp = v.pot[s];
    const double inv = 1.0 / r2, s2 = pp.sig2d * inv, s6 = s2 * s2 * s2;
    const double fr = pp.eps24d * inv * s6 * (2.0 * s6 - 1.0);
    if (v.F)
      for (int a = 0; a < 3; a++) atomicAdd(&v.F[3 * (size_t)oi + a], (float)(-fr * d[a]));
    double df[3];
    for (int a = 0; a < 3; a++) df[a] = g->Q[a] * d[0] + g->Q[3 + a] * d[1] + g->Q[6 + a] * d[2];
    if (g->variant != NEMD_DO)
      for (int a = 0; a < 3; a++) df[a] = d[a];
    float *p0 = &v.ppart[2 * (size_t)it.x].x, *p1 = &v.ppart[2 * (size_t)it.x + 1].x;
    atomicAdd(p0, (float)(pp.eps4d * s6 * (s6 - 1.0) - pp.ushiftd));
    atomicAdd(p0 + 1, (float)(fr * df[0] * df[0]));
    atomicAdd(p0 + 2, (float)(fr * df[1] * df[1]));
    atomicAdd(p0 + 3, (float)(fr * df[2] * df[2]));
    atomicAdd(p1, (float)(fr * df[0] * df[1]));
    atomicAdd(p1 + 1, (float)(fr * df[0] * df[2]));
    atomicAdd(p1 + 2, (float)(fr * df[1] * df[2]));
    atomicAdd(reinterpret_cast<int *>(p1 + 3), 1);
  }
}

// kReduceSplit blocks per system: block r sums the r-th contiguous quarter of
// the system's sorted particles' pair sums; the last of them to finish (a
// ticket per system, returned to zero) adds the blocks' sums in block order,
// halves them for the full neighbourhoods, rotates the virial back to
// Cartesian for the dynamic offset frame (W = Q W_R Q^T) and publishes.  The
// order of every addition is fixed.

__global__ void __launch_bounds__(256) k_b_reduce(BatchView v) {
  // float32 pair sums accumulated in float-float (the float64 pipe runs at
  // 1/64 of the float32 rate here), pair counts in 64-bit integers; a fixed
  // order throughout (threads over particles, shuffle tree, warps in order)
  constexpr int K = 7;
  constexpr int kW = 256 / 32;
  __shared__ float shh[kW][K], shl[kW][K];
  __shared__ long long shn[kW];
  __shared__ bool last;
  const int s = blockIdx.x / kReduceSplit, r = blockIdx.x % kReduceSplit;
  Geo *g = v.geo + s;
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  int b = 0, e = 0;
  if (ok) {
    const int coff = v.sys[s].coff;
    const int b0 = v.start[coff], e0 = v.start[coff + g->ncells];
    const long long len = e0 - b0;
    b = b0 + (int)(len * r / kReduceSplit);
    e = b0 + (int)(len * (r + 1) / kReduceSplit);
  }
  ff a[K];
#pragma unroll
  for (int k = 0; k < K; k++) a[k] = {0.f, 0.f};
  long long np = 0;
  // four particles' loads in flight before their sums (the same order of
  // additions as one particle at a time)
  constexpr int kAhead = 4;
  for (int k0 = b + threadIdx.x; k0 < e; k0 += kAhead * blockDim.x) {
    float4 p0[kAhead], p1[kAhead];
#pragma unroll
    for (int h = 0; h < kAhead; h++) {
      const int k = k0 + h * blockDim.x;
      if (k < e) {
        p0[h] = v.ppart[2 * (size_t)k];
        p1[h] = v.ppart[2 * (size_t)k + 1];
      }
    }
#pragma unroll
    for (int h = 0; h < kAhead; h++) {
      if (k0 + h * (int)blockDim.x >= e) break;
      a[0] = ff_add(a[0], ff{p0[h].x, 0.f});
      a[1] = ff_add(a[1], ff{p0[h].y, 0.f});
      a[2] = ff_add(a[2], ff{p0[h].z, 0.f});
      a[3] = ff_add(a[3], ff{p0[h].w, 0.f});
      a[4] = ff_add(a[4], ff{p1[h].x, 0.f});
      a[5] = ff_add(a[5], ff{p1[h].y, 0.f});
      a[6] = ff_add(a[6], ff{p1[h].z, 0.f});
      np += __float_as_int(p1[h].w);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; k++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      a[k] = ff_add(a[k], ff{__shfl_down_sync(0xffffffffu, a[k].hi, o), __shfl_down_sync(0xffffffffu, a[k].lo, o)});
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) np += __shfl_down_sync(0xffffffffu, np, o);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) {
      shh[warp][k] = a[k].hi;
      shl[warp][k] = a[k].lo;
    }
    shn[warp] = np;
  }
  __syncthreads();
  // this block's sums in float64 (thread k: value k, warps in order)
  static_assert(K + 1 == kReduceSums, "reduction sums");
  double *mine = v.red_part + (size_t)blockIdx.x * kReduceSums;
  if (threadIdx.x < K) {
    double x = 0.0;
    for (int w = 0; w < kW; w++) x += (double)shh[w][threadIdx.x] + (double)shl[w][threadIdx.x];
    mine[threadIdx.x] = x;
  } else if (threadIdx.x == K) {
    long long n2 = 0;
    for (int w = 0; w < kW; w++) n2 += shn[w];
    mine[K] = (double)n2;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    last = atomicAdd(&v.red_ticket[s], 1u) == (unsigned)(kReduceSplit - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double sh0[K + 1];
  if (threadIdx.x <= K) {
    const double *part = v.red_part + (size_t)s * kReduceSplit * kReduceSums;
    double x = 0.0;
    for (int q = 0; q < kReduceSplit; q++) x += __ldcg(part + q * kReduceSums + threadIdx.x);
    sh0[threadIdx.x] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    v.red_ticket[s] = 0u;
    double Wr[9];
    Wr[0] = 0.5 * sh0[1];
    Wr[4] = 0.5 * sh0[2];
    Wr[8] = 0.5 * sh0[3];
    Wr[1] = Wr[3] = 0.5 * sh0[4];
    Wr[2] = Wr[6] = 0.5 * sh0[5];
    Wr[5] = Wr[7] = 0.5 * sh0[6];
    double W[9];
    if (g->variant == NEMD_DO) {
      double T9[9];
      const double *Q = g->Q;
      for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T9[3 * i + j] = Q[3 * i] * Wr[j] + Q[3 * i + 1] * Wr[3 + j] + Q[3 * i + 2] * Wr[6 + j];
      for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
          W[3 * i + j] = T9[3 * i] * Q[3 * j] + T9[3 * i + 1] * Q[3 * j + 1] + T9[3 * i + 2] * Q[3 * j + 2];
    } else {
      for (int k = 0; k < 9; k++) W[k] = Wr[k];
    }
    if (v.UW) {
      v.UW[10 * (size_t)s] = ok ? 0.5 * sh0[0] : 0.0;
      for (int k = 0; k < 9; k++) v.UW[10 * (size_t)s + 1 + k] = ok ? W[k] : 0.0;
    }
    v.sys_pairs[s] = (unsigned long long)(0.5 * sh0[7] + 0.25);
    g->sticky |= g->error;
  }
}

cudaError_t launch_batch_finish(cudaStream_t st, const BatchView &v) {
  k_b_fixup<<<4, 256, 0, st>>>(v);
  k_b_reduce<<<v.nsys * kReduceSplit, 256, 0, st>>>(v);
  return cudaGetLastError();
}

}  // namespace nemd
