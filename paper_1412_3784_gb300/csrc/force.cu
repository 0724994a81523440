// force.cu -- cell-pair force, energy and virial (Sec. 3: only the 27 cells of a
// neighbourhood are searched; Sec. 5: every force evaluation is preceded by a
// distance check) and the deterministic float64 reductions.
//
// Plain kernel: one thread per particle in cell order.  The thread walks the
// rows of its home cell's stencil (Sec. 4.1: 27 cells; Sec. 4.2: 27-36 cells),
// each row a run of consecutive x-cells, and tests every particle of every
// cell with a float32 distance check in cell-relative coordinates.  Candidates
// whose float32 r^2 lies within the guard band of rc^2 are decided by the
// canonical float64 displacement, so the pair set is exactly the definition's.
// Full neighbourhoods: each unordered pair is met from both sides, every
// particle's force is accumulated by its own thread, and U, W are halved.
#include <math.h>

#include "nemd_device.cuh"
#include "nemd_internal.cuh"

namespace nemd {

struct Pot {
  float eps4, eps24, sig2, ushift;
  double eps4d, eps24d, sig2d, ushiftd;
};

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

template <int NT, bool RECORD, bool PRECISE>
__global__ void __launch_bounds__(NT) k_force_plain(const Geo *__restrict__ g, const float4 *__restrict__ pos,
                                                    const float4 *__restrict__ posr,
                                                    const int *__restrict__ cell_sorted,
                                                    const int *__restrict__ start, const Row *__restrict__ rows,
                                                    const int *__restrict__ rowcnt, const double *__restrict__ q,
                                                    int n, Pot pp, float *__restrict__ F,
                                                    double *__restrict__ partials, int32_t *__restrict__ pair_buf,
                                                    unsigned long long *__restrict__ pair_count, long long pair_cap) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  float fx = 0.f, fy = 0.f, fz = 0.f, uu = 0.f;
  float wxx = 0.f, wyy = 0.f, wzz = 0.f, wxy = 0.f, wxz = 0.f, wyz = 0.f;
  double dfx = 0, dfy = 0, dfz = 0, du = 0, dwxx = 0, dwyy = 0, dwzz = 0, dwxy = 0, dwxz = 0, dwyz = 0;
  int npair = 0, ncand = 0, nre = 0;
  const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
  if (ok && k < n) {
    const float4 pi = pos[k];
    const int oi = __float_as_int(pi.w);
    const int cell = cell_sorted[k];
    const int l1 = g->nc[0], l2 = g->nc[1];
    const int ix = cell % l1, rest = cell / l1, iy = rest % l2, iz = rest / l2;
    const int cls = iy + l2 * iz;
    const Row *rw = rows + (size_t)cls * g->maxrows;
    const int nr = rowcnt[cls];
    const float lo = g->rc2_lo, hi = g->rc2_hi;
    const float sx = g->step[0], sy = g->step[1], sz = g->step[2];
    const float srx = g->step_r[0], sry = g->step_r[1], srz = g->step_r[2];
    const bool is_do = (g->variant == NEMD_DO);
    const float4 pir = posr[k];
    int mi[3] = {0, 0, 0};
    bool have_mi = false;
    for (int r = 0; r < nr; r++) {
      const Row R = rw[r];
      // t = x_i - o exactly (multiples of the quantum); T = residual of x_i - o
      float tx = pi.x - R.ox, ty = pi.y - R.oy, tz = pi.z - R.oz;
      float Tx = pir.x - R.rx, Ty = pir.y - R.ry, Tz = pir.z - R.rz;
      const int jxu = ix + R.dxlo;
      int kx = floordiv_dev(jxu, l1);
      int jx = jxu - kx * l1;
      for (int m = 0; m < R.cnt; m++) {
        const int c = R.cbase + jx;
        const int b = start[c], e = start[c + 1];
        ncand += e - b;
        for (int j = b; j < e; j++) {
          const float4 pj = pos[j];
          float dx = pj.x - tx, dy = pj.y - ty, dz = pj.z - tz;
          const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          if (r2 < hi) {
            const int oj = __float_as_int(pj.w);
            if (j == k && kx == 0 && R.ky == 0 && R.kz == 0) continue;
            int n1 = kx, n2 = R.ky, n3 = R.kz;
            if ((RECORD || PRECISE || r2 >= lo) && is_do) {
              if (!have_mi) {
                brick_image(g, q, oi, mi);
                have_mi = true;
              }
              int mj[3];
              brick_image(g, q, oj, mj);
              n1 += mi[0] - mj[0];
              n2 += mi[1] - mj[1];
              n3 += mi[2] - mj[2];
            }
            double dd[3];
            bool accept = true;
            if (PRECISE || r2 >= lo) {
              double cr2 = canon_r2(g, q, oi, oj, n1, n2, n3, dd);
              if (r2 >= lo) {
                nre++;
                accept = cr2 < g->rc2;
              }
              if (PRECISE && accept) {
                double inv = 1.0 / cr2;
                double s2 = pp.sig2d * inv;
                double s6 = s2 * s2 * s2;
                double fr = pp.eps24d * inv * s6 * (2.0 * s6 - 1.0);
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
              }
            }
            if (!accept) continue;
            npair++;
            if (!PRECISE) {
              // add back the residuals: d = (x_j - t) + (r_j - T), accurate to a
              // rounding of d itself
              const float4 pjr = posr[j];
              dx += pjr.x - Tx;
              dy += pjr.y - Ty;
              dz += pjr.z - Tz;
              const float r2c = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
              const float inv = __frcp_rn(r2c);
              const float s2 = pp.sig2 * inv;
              const float s6 = s2 * s2 * s2;
              const float fr = pp.eps24 * inv * s6 * (2.0f * s6 - 1.0f);
              uu += fmaf(pp.eps4 * s6, s6 - 1.0f, -pp.ushift);
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
            }
            if (RECORD) {
              if (is_do && !have_mi) {
                brick_image(g, q, oi, mi);
                have_mi = true;
              }
              bool canon = (oi < oj) || (oi == oj && (n1 != 0 ? n1 > 0 : (n2 != 0 ? n2 > 0 : n3 > 0)));
              if (canon) {
                unsigned long long slot = atomicAdd(pair_count, 1ull);
                if ((long long)slot < pair_cap) {
                  int32_t *p = pair_buf + 5 * slot;
                  p[0] = oi;
                  p[1] = oj;
                  p[2] = n1;
                  p[3] = n2;
                  p[4] = n3;
                }
              }
            }
          }
        }
        tx -= sx;
        ty -= sy;
        tz -= sz;
        Tx -= srx;
        Ty -= sry;
        Tz -= srz;
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
        ox = Qm[0] * fx + Qm[1] * fy + Qm[2] * fz;
        oy = Qm[3] * fx + Qm[4] * fy + Qm[5] * fz;
        oz = Qm[6] * fx + Qm[7] * fy + Qm[8] * fz;
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
    v[0] = uu;
    v[1] = wxx;
    v[2] = wyy;
    v[3] = wzz;
    v[4] = wxy;
    v[5] = wxz;
    v[6] = wyz;
  }
  v[7] = npair;
  v[8] = ncand;
  v[9] = nre;
  block_reduce_store<NT>(v, partials);
}

// Single block: sums the per-block partials in a fixed order (deterministic),
// halves the full-neighbourhood double count, rotates the virial of the
// dynamic offset frame back to Cartesian (W = Q W_R Q^T) and publishes
// U, W and the counters.
__global__ void k_reduce_final(Geo *__restrict__ g, const double *__restrict__ partials, int nblocks,
                               int frame_is_cartesian, double *__restrict__ uw,
                               unsigned long long *__restrict__ counters) {
  __shared__ double sh[256][kPartials];
  double acc[kPartials];
#pragma unroll
  for (int k = 0; k < kPartials; k++) acc[k] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < kPartials; k++) acc[k] += partials[(size_t)b * kPartials + k];
#pragma unroll
  for (int k = 0; k < kPartials; k++) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < kPartials; k++) sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const bool ok = !(g->error & (ERRB_BOX | ERRB_CAPACITY));
    double U = 0.5 * sh[0][0];
    double Wr[9];
    Wr[0] = 0.5 * sh[0][1];
    Wr[4] = 0.5 * sh[0][2];
    Wr[8] = 0.5 * sh[0][3];
    Wr[1] = Wr[3] = 0.5 * sh[0][4];
    Wr[2] = Wr[6] = 0.5 * sh[0][5];
    Wr[5] = Wr[7] = 0.5 * sh[0][6];
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
    counters[0] = (unsigned long long)(0.5 * sh[0][7] + 0.25);
    counters[1] = (unsigned long long)(sh[0][8] + 0.5);
    counters[2] = (unsigned long long)(sh[0][9] + 0.5);
    g->sticky |= g->error;
  }
}

static Pot make_pot(const nemd_ctx *c) {
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
#define NEMD_ARGS                                                                                         \
  c->geo, c->pos4, c->posr, c->cell_sorted, c->start, c->rows, c->rowcnt, c->q_dev, n, pp, F, c->partials, \
      c->pair_buf, c->pair_count, (long long)c->record_cap
  if (rec && pre)
    k_force_plain<NT, true, true><<<nblocks, NT, 0, c->stream>>>(NEMD_ARGS);
  else if (rec)
    k_force_plain<NT, true, false><<<nblocks, NT, 0, c->stream>>>(NEMD_ARGS);
  else if (pre)
    k_force_plain<NT, false, true><<<nblocks, NT, 0, c->stream>>>(NEMD_ARGS);
  else
    k_force_plain<NT, false, false><<<nblocks, NT, 0, c->stream>>>(NEMD_ARGS);
#undef NEMD_ARGS
}

cudaError_t launch_forces(nemd_ctx *c, float *F_dev, double *UW_dev) {
  const Pot pp = make_pot(c);
  const int NT = 128;
  int nblocks = (int)((c->n + NT - 1) / NT);
  if (nblocks < 1) nblocks = 1;
  if (c->record_cap > 0) {
    cudaError_t e = cudaMemsetAsync(c->pair_count, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
  }
  const bool timed = c->timing && c->ev && c->ev_n < c->ev_cap;
  if (timed) cudaEventRecord(c->ev[2 * c->ev_n], c->stream);
  launch_plain<NT>(c, nblocks, pp, F_dev);
  if (timed) {
    cudaEventRecord(c->ev[2 * c->ev_n + 1], c->stream);
    c->ev_n++;
  }
  c->launches += 2;
  k_reduce_final<<<1, 256, 0, c->stream>>>(c->geo, c->partials, nblocks, c->precise ? 1 : 0, UW_dev, c->counters);
  return cudaGetLastError();
}

}  // namespace nemd
