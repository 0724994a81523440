// lattice.cu -- lattice evolution and remap (Sec. 2.1, 2.2), cell grid (Sec. 4.1,
// 4.2, 5.1, 5.2) and neighbour stencil (Sec. 4.1, 4.2) on the device, in FP64.
//
//   tau = t - T floor(t / T)                 remap L <- L M^-1 at every period (Eq. kr);
//   or centred, tau = t - T floor(t/T + 1/2), remapping half way through a period
//   (Sec. 2.2: shear remapped at half a lattice spacing)
//   L   = exp(tau A) L0                      (Sec. 2.1, dL/dt = A L)
//   exp by Taylor series with scaling and squaring, products spread over lanes
//   L^-1 by the adjugate, V = det L, heights h_i = 1 / |row_i(L^-1)|
//   QR by Cholesky of L^T L (R upper triangular, r_ii > 0), Q = L R^-1
//   dynamic size:   c_i = floor((1 - 1e-12) k h_i / rc)     (Sec. 4.1)
//   dynamic offset: l_i = floor((1 - 1e-12) k r_ii / rc)    (Sec. 5.2)
#include <math.h>

#include "batch_internal.cuh"

namespace {
// float-float (hi, lo) form of a float64 value: hi rounded, lo the rounded rest
__device__ __forceinline__ float2 to_ff2(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}
}  // namespace

namespace nemd {

namespace {

__device__ __forceinline__ int floordiv_i(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
  return q;
}

// c = a * b for 3x3 row-major matrices in shared memory; lanes 0..8 each
// produce one entry.  c may alias a or b.
__device__ __forceinline__ void mm3(const double *a, const double *b, double *c, int lane) {
  double v = 0.0;
  if (lane < 9) {
    int i = lane / 3, j = lane % 3;
    v = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
  }
  __syncwarp();
  if (lane < 9) c[lane] = v;
  __syncwarp();
}

}  // namespace

// Shared scratch of one warp's lattice.
struct LatScratch {
  double B[9], P[9], E[9], Ls[9], Gm[9], Rm[9], Ri[9], Lt[9], cof[9];
  double det;
  int s;
};

// One warp (sc its shared scratch).  validate != 0: compute exp(tau_in A) L0
// only (for the KR check).
__device__ __forceinline__ void lattice_body(Geo *g, const LatIn &in, LatScratch &sc) {
  const int validate = in.validate;
  const double tau_in = in.tau;
  double *B = sc.B, *P = sc.P, *E = sc.E, *Ls = sc.Ls, *Gm = sc.Gm, *Rm = sc.Rm, *Ri = sc.Ri, *Lt = sc.Lt;
  int &sh_s = sc.s;
  const int lane = threadIdx.x & 31;

  double tau;
  if (validate) {
    tau = tau_in;
  } else {
    const double T = in.T, t = in.t_dev ? *in.t_dev : in.t;
    if (!(T > 0.0))
      tau = t;
    else if (in.centered)
      tau = t - T * floor(t / T + 0.5);
    else
      tau = t - T * floor(t / T);
  }
  if (lane < 9) {
    g->A[lane] = in.A[lane];
    g->L0[lane] = in.L0[lane];
  }
  if (lane == 0) {
    g->T = in.T;
    g->t = in.t_dev ? *in.t_dev : in.t;
    if (!validate) g->error = 0;
  }

  // scaled argument B = tau A / 2^s with |B|_1 <= 1/8
  if (lane < 9) B[lane] = tau * in.A[lane];
  __syncwarp();
  if (lane == 0) {
    double nrm = 0.0;
    for (int j = 0; j < 3; j++) {
      double cs = fabs(B[j]) + fabs(B[3 + j]) + fabs(B[6 + j]);
      nrm = fmax(nrm, cs);
    }
    // smallest s with 8 nrm <= 2^s (from the exponent: 8 nrm = f 2^e, f in [1/2, 1))
    int s = 0;
    if (nrm > 0.125) frexp(nrm * 8.0, &s);
    sh_s = s;
  }
  __syncwarp();
  const int s = sh_s;
  if (lane < 9) B[lane] = ldexp(B[lane], -s);
  __syncwarp();

  // Taylor polynomial of degree 12 by Horner: P = I + B/12, P = I + B P / k ...
  // (1/k as constants: a float64 division costs many float64 operations here)
  const int deg = 12;
  const double inv_k[deg + 1] = {0.0,       1.0,       1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5, 1.0 / 6,
                                 1.0 / 7,   1.0 / 8,   1.0 / 9,  1.0 / 10, 1.0 / 11, 1.0 / 12};
  if (lane < 9) P[lane] = ((lane % 4) == 0 ? 1.0 : 0.0) + B[lane] * inv_k[deg];
  __syncwarp();
#pragma unroll
  for (int k = deg - 1; k >= 1; k--) {
    mm3(B, P, P, lane);
    if (lane < 9) P[lane] = ((lane % 4) == 0 ? 1.0 : 0.0) + P[lane] * inv_k[k];
    __syncwarp();
  }
  for (int k = 0; k < s; k++) mm3(P, P, P, lane);
  if (lane < 9) E[lane] = P[lane];
  __syncwarp();

  // L = E L0
  if (lane < 9) Ls[lane] = in.L0[lane];
  __syncwarp();
  mm3(E, Ls, Ls, lane);

  if (validate) {
    if (lane < 9) g->L[lane] = Ls[lane];
    if (lane == 0) g->tau = tau;
    return;
  }

  // inverse by the adjugate
  double *cof = sc.cof;
  double &det_s = sc.det;
  if (lane < 9) {
    const double *a = Ls;
    double c;
    switch (lane) {
      case 0: c = a[4] * a[8] - a[5] * a[7]; break;
      case 1: c = a[2] * a[7] - a[1] * a[8]; break;
      case 2: c = a[1] * a[5] - a[2] * a[4]; break;
      case 3: c = a[5] * a[6] - a[3] * a[8]; break;
      case 4: c = a[0] * a[8] - a[2] * a[6]; break;
      case 5: c = a[2] * a[3] - a[0] * a[5]; break;
      case 6: c = a[3] * a[7] - a[4] * a[6]; break;
      case 7: c = a[1] * a[6] - a[0] * a[7]; break;
      default: c = a[0] * a[4] - a[1] * a[3]; break;
    }
    cof[lane] = c;
  }
  __syncwarp();
  if (lane == 0) det_s = Ls[0] * cof[0] + Ls[1] * cof[3] + Ls[2] * cof[6];
  __syncwarp();
  const double det = det_s;
  if (lane < 9) {
    g->L[lane] = Ls[lane];
    g->Linv[lane] = cof[lane] / det;
    g->Linvff[lane] = to_ff2(cof[lane] / det);
  }
  // Gram matrix L^T L for the Cholesky QR
  if (lane < 9) Lt[lane] = Ls[(lane % 3) * 3 + lane / 3];
  __syncwarp();
  mm3(Lt, Ls, Gm, lane);

  if (lane == 0) {
    g->tau = tau;
    g->V = fabs(det);
    // heights 1 / |row_i(L^-1)| = |det| / |row_i(cof)|, by the reciprocal square
    // root (float64 division and square root are each ~0.3 us of latency here)
    const double adet = fabs(det);
    for (int i = 0; i < 3; i++) {
      const double r0 = cof[3 * i], r1 = cof[3 * i + 1], r2 = cof[3 * i + 2];
      g->h[i] = adet * rsqrt(r0 * r0 + r1 * r1 + r2 * r2);
    }
    // Cholesky of the Gram matrix, each pivot's reciprocal formed once
    double r11 = sqrt(Gm[0]);
    const double i11 = 1.0 / r11;
    double r12 = Gm[1] * i11, r13 = Gm[2] * i11;
    double r22 = sqrt(Gm[4] - r12 * r12);
    const double i22 = 1.0 / r22;
    double r23 = (Gm[5] - r12 * r13) * i22;
    double r33 = sqrt(Gm[8] - r13 * r13 - r23 * r23);
    const double i33 = 1.0 / r33;
    double R[9] = {r11, r12, r13, 0.0, r22, r23, 0.0, 0.0, r33};
    for (int k = 0; k < 9; k++) Rm[k] = R[k];
    Ri[0] = i11;
    Ri[1] = -r12 * i11 * i22;
    Ri[2] = (r12 * r23 - r13 * r22) * i11 * i22 * i33;
    Ri[3] = 0.0;
    Ri[4] = i22;
    Ri[5] = -r23 * i22 * i33;
    Ri[6] = 0.0;
    Ri[7] = 0.0;
    Ri[8] = i33;
  }
  __syncwarp();
  if (lane < 9) {
    g->R[lane] = Rm[lane];
    g->Rff[lane] = to_ff2(Rm[lane]);
  }
  if (lane < 3) {
    const double ri = Ri[4 * lane];  // 1 / r_ii, from the Cholesky above
    g->rinv[lane] = ri;
    g->rinvff[lane] = to_ff2(ri);
  }
  mm3(Ls, Ri, Ri, lane);  // Q = L R^-1
  if (lane < 9) g->Q[lane] = Ri[lane];
  __syncwarp();
}

__global__ void k_lattice(Geo *g, LatIn in) {
  __shared__ LatScratch sc;
  lattice_body(g, in, sc);
}

// Single thread: cell counts of both variants at k = 1, their neighbourhood
// volumes (Sec. 5.1: V_DS = 27 V / (c1 c2 c3); Sec. 5.2: V_DO = avg r11 r22 r33 /
// (l1 l2 l3) with avg = 27 + 14/l3 + 6/l2 - 4/(l2 l3)), the variant of this step,
// its grid at cell factor k, and the float32 guard band.
__device__ void grid_body(Geo *g, const GridIn &in) {
  g->rc = in.rc;
  g->req_variant = in.variant;
  g->kfac = in.kfac;
  g->max_cells = in.max_cells;
  double Ls[9], Rm[9], Ri[9];
  for (int k = 0; k < 9; k++) {
    Ls[k] = g->L[k];
    Rm[k] = g->R[k];
    Ri[k] = g->Q[k];
  }
  const double rc = g->rc;
  const double V = g->V;
  const double fac = (1.0 - kMargin);
  // one reciprocal instead of a division per count (a float64 division is
  // ~0.3 us of latency on this part, and this thread's work is serial): the
  // product differs from the quotient by a rounding, which moves a count only
  // within 2^-52 of an integer, inside the 1e-12 margin of fac
  const double irc = 1.0 / rc;
  int cds1[3], cdo1[3];
  for (int a = 0; a < 3; a++) {
    cds1[a] = (int)floor(fac * g->h[a] * irc);
    cdo1[a] = (int)floor(fac * Rm[4 * a] * irc);
  }
  // neighbourhood volumes at k = 1 (Sec. 5.1, 5.2)
  double vds = 1e300, vdo = 1e300;
  if (cds1[0] > 0 && cds1[1] > 0 && cds1[2] > 0)
    vds = 27.0 * V / ((double)cds1[0] * (double)cds1[1] * (double)cds1[2]);
  if (cdo1[0] > 0 && cdo1[1] > 0 && cdo1[2] > 0) {
    double l2 = cdo1[1], l3 = cdo1[2];
    double avg = (cdo1[1] >= 2 && cdo1[2] >= 2) ? 27.0 + 14.0 / l3 + 6.0 / l2 - 4.0 / (l2 * l3) : 36.0;
    vdo = avg * V / ((double)cdo1[0] * l2 * l3);
  }
  g->vol_ds = vds;
  g->vol_do = vdo;
  for (int a = 0; a < 3; a++) {
    g->counts_ds[a] = cds1[a];
    g->counts_do[a] = cdo1[a];
  }
  int variant = g->req_variant;
  int kf = g->kfac;
  if (variant == NEMD_AUTO_LEARNED && g->learned_choice >= 0) {
    // the learned selector's option for this step: variant and cell factor
    variant = g->learned_choice & 1;
    kf = 1 + (g->learned_choice >> 1);
    g->kfac = kf;
  } else if (variant != NEMD_DS && variant != NEMD_DO) {
    variant = (vdo < vds) ? NEMD_DO : NEMD_DS;
  }
  g->variant = variant;

  int nc[3];
  double Gd[9];
  float step[3];
  int reach[3];
  int maxrows;
  // bound on the float-float wrap's position error: fractional coordinates
  // within 2^-42 (16 + 1) of the definition's, then a few dozen operations of
  // relative error ~2^-45 on values up to the box's extent; the dynamic offset
  // windows reach this much further, so a particle binned a rounding outside
  // its cell still finds every partner
  double lsum = 0.0;
  for (int k = 0; k < 9; k++) lsum += fabs(Ls[k]) + fabs(Rm[k]);
  const double wtol = ldexp(lsum + 1.0, -36);
  g->wrap_tol = wtol;
  const double rce = rc * (1.0 + kMargin) + (variant == NEMD_DS ? 0.0 : 2.0 * wtol);
  if (variant == NEMD_DS) {
    for (int a = 0; a < 3; a++) nc[a] = (int)floor(fac * (double)kf * g->h[a] * irc);
    double inc[3];
    for (int b = 0; b < 3; b++) inc[b] = nc[b] > 0 ? 1.0 / (double)nc[b] : 0.0;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) Gd[3 * a + b] = Ls[3 * a + b] * inc[b];
    for (int a = 0; a < 3; a++) {
      g->Ginv_scale[a] = (double)nc[a];
      g->w[a] = 0.0;
      reach[a] = kf;
    }
    maxrows = (2 * kf + 1) * (2 * kf + 1);
    for (int k = 0; k < 9; k++) g->Qf[k] = (k % 4 == 0) ? 1.0f : 0.0f;
  } else {
    for (int a = 0; a < 3; a++) nc[a] = (int)floor(fac * (double)kf * Rm[4 * a] * irc);
    for (int k = 0; k < 9; k++) Gd[k] = 0.0;
    // the stencil forms its window bounds in float-float (error below 2^-40
    // lsum, a sixteenth of wrap_tol) from this reach, one wrap_tol longer
    const double rcs = rce + wtol;
    g->rceff = to_ff2(rcs);
    for (int a = 0; a < 3; a++) {
      const double w = (nc[a] > 0) ? Rm[4 * a] / (double)nc[a] : 1.0;
      const double iw = 1.0 / w;  // the one reciprocal of the side: binning, windows and reach
      g->w[a] = w;
      g->Ginv_scale[a] = iw;
      g->wff[a] = to_ff2(w);
      g->Ginvff[a] = to_ff2(iw);
      Gd[4 * a] = w;
      reach[a] = (int)ceil(rcs * iw);
    }
    maxrows = (2 * reach[2] + 1) * (2 * reach[1] + 2);
    for (int k = 0; k < 9; k++) g->Qf[k] = (float)Ri[k];
  }
  int err = 0;
  long long ncells = (long long)nc[0] * nc[1] * nc[2];
  if (nc[0] < 1 || nc[1] < 1 || nc[2] < 1) err |= ERRB_BOX;
  if (ncells > (long long)g->max_cells || maxrows > in.row_stride) err |= ERRB_CAPACITY;
  g->error |= err;
  for (int a = 0; a < 3; a++) {
    g->nc[a] = nc[a];
    g->reach[a] = reach[a];
  }
  g->ncells = err ? 0 : (int)ncells;
  g->maxrows = maxrows;
  // chunks of up to 32 particles of one x-row span at most kMaxSpan cells, or
  // more (up to kMaxSpanCap) where the cells hold on average fewer than 6
  // particles, so that a chunk still fills most of a warp
  int span = kMaxSpan;
  if (ncells > 0 && in.n > 0) span = min(kMaxSpanCap, max(kMaxSpan, (int)ceil(48.0 * (double)ncells / in.n)));
  g->span = span;
  for (int k = 0; k < 9; k++) {
    g->G[k] = Gd[k];
    g->Gf[k] = (float)Gd[k];
    g->Gff[k] = to_ff2(Gd[k]);
  }
  // Quantum: float32 positions and offsets are stored as exact multiples of a
  // power of two q, chosen so that every intermediate (|rel| + |offset| bounded
  // by M) has at most 24 significant bits.  Then t = x_i - o and d = x_j - t are
  // exact in float32; only the residuals (each < q/2, carried separately) are
  // missing from the distance test, and they are added back for accepted pairs.
  double gmax = 0.0;
  for (int a = 0; a < 3; a++) gmax = fmax(gmax, fabs(Gd[3 * a]) + fabs(Gd[3 * a + 1]) + fabs(Gd[3 * a + 2]));
  const int rmax = max(reach[0], max(reach[1], reach[2]));
  // offsets reach (rmax + 2 + span) cells and the warp kernel's staged
  // positions (Sec. 3 union windows) up to (span + 2 rmax + 3) cells from a
  // chunk's first cell; positions half a cell, distances rc
  const double M = (double)(3 * rmax + 6 + span) * gmax + 2.0 * rc;
  int e2;
  frexp(M, &e2);             // M < 2^e2
  const double q = ldexp(1.0, e2 - 23);
  g->quantum = q;
  g->quantum_inv = ldexp(1.0, 23 - e2);
  g->quantum_f = (float)q;
  g->quantum_inv_f = (float)g->quantum_inv;
  // frame vector between consecutive x-cells: G e_x (dynamic size), (w1, 0, 0) (dynamic offset)
  for (int a = 0; a < 3; a++) {
    double sv = Gd[3 * a];
    double sq = rint(sv * g->quantum_inv) * q;  // q a power of two: exact
    step[a] = (float)sq;
    g->step_r[a] = (float)(sv - sq);
  }
  // Coarse band (quantised test): the omitted residuals of x_i, x_j, the row
  // shift and (dx + sxi) steps, at most (rmax + 6 + span) q / 2 per component,
  // plus the rounding of r^2.  Fine band (test with residuals added back): one
  // rounding of each corrected component and of r^2.
  const double u = 5.9604644775390625e-08;  // 2^-24
  const double E = (double)(rmax + 6 + span) * 0.5 * q;
  const double s3 = 1.7320508075688772;
  // Both bands also cover the wrap's float-float error: each position within
  // dw of its float64 value (wrap_tol, plus a rounding of the residual), so
  // |d| within 2 dw and r^2 within 4 rc dw + 4 dw^2.
  const double dw = wtol + ldexp(q, -20);
  const double wterm = 4.0 * rc * dw + 4.0 * dw * dw;
  double band = 2.0 * (2.0 * s3 * rc * E + 3.0 * E * E + 3.0 * u * rc * rc) + 1e-12 * rc * rc + wterm;
  const double E2 = 2.0 * u * (rc + q);
  double band2 = 2.0 * (2.0 * s3 * rc * E2 + 3.0 * E2 * E2 + 3.0 * u * rc * rc) + 1e-12 * rc * rc + wterm;
  for (int a = 0; a < 3; a++) g->step[a] = step[a];
  g->band = (float)band;
  {
    // kappa = (G^-1 rel)_1: dynamic size c1 (row 1 of L^-1) . rel, dynamic offset x / w1
    double k3[3];
    if (variant == NEMD_DS) {
      for (int a = 0; a < 3; a++) k3[a] = (double)nc[0] * g->Linv[a];
    } else {
      k3[0] = nc[0] > 0 ? g->Ginv_scale[0] : 0.0;
      k3[1] = k3[2] = 0.0;
    }
    const double kn = sqrt(k3[0] * k3[0] + k3[1] * k3[1] + k3[2] * k3[2]);
    for (int a = 0; a < 3; a++) g->kap[a] = (float)k3[a];
    // |d . n1| = |delta kappa| h_cell <= |d| < rc, with room for float32 rounding
    g->rho1 = (float)(rc * kn * (1.0 + 1e-4) + 1e-4);
  }
  g->rc2 = rc * rc;
  g->rc2f = (float)(rc * rc);
  g->rc2_lo = __double2float_rd(rc * rc - band);
  g->rc2_lo2 = __double2float_rd(rc * rc - band2);
  g->rc2_hi2 = __double2float_ru(rc * rc + band2);
  g->rc2_hi = __double2float_ru(rc * rc + band);
}

__global__ void k_grid(Geo *g, GridIn in) {
  if (threadIdx.x == 0) grid_body(g, in);
}

// ---- the stencil in float-float: a class's window bounds and row shifts take
// a few dozen operations, and float64 runs at a small fraction of the float32
// rate here ----
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ int ff_floor_int(ff x) { return (int)ff_floor(x); }
__device__ __forceinline__ int ff_ceil_int(ff x) { return -(int)ff_floor(ff_neg(x)); }

// Nearest integer to hi + lo (|hi| < 2^22; halves as round-half-even on hi).
__device__ __forceinline__ float ff_rint(ff x) {
  const float r = rintf(x.hi);
  const float d = __fadd_rn(__fsub_rn(x.hi, r), x.lo);  // x.hi - r is exact
  return d > 0.5f ? __fadd_rn(r, 1.f) : (d < -0.5f ? __fsub_rn(r, 1.f) : r);
}

// One component o of a row shift split as the rows store it: the nearest
// multiple sh of the quantum q (a power of two; qi = 1 / q) and the rest
// o - sh rounded once to float32 (o.hi - sh is exact: both lie within a factor
// two of each other, or sh = 0).
__device__ __forceinline__ void split_shift_ff(ff o, float q, float qi, float &sh, float &sr) {
  const ff t = {__fmul_rn(o.hi, qi), __fmul_rn(o.lo, qi)};  // exact scaling
  sh = __fmul_rn(ff_rint(t), q);
  sr = __fadd_rn(__fsub_rn(o.hi, sh), o.lo);
}

// The neighbour rows of one home (iy, iz) class, written to out[0..maxrows) by
// the lanes of one warp (one row per lane); returns their number on every
// lane.  Row order: dz (jz) outer, dy (jy) inner.  cell_base is added to every
// row's first cell (the system's first cell slot in a batch).
__device__ int stencil_class_warp(Geo *g, int cls, int cell_base, Row *out, int lane) {
  constexpr int kMaxZ = 2 * kMaxFactor + 4;  // bound on the z-rows of a dynamic offset class
  const int l1 = g->nc[0], l2 = g->nc[1], l3 = g->nc[2];
  const int maxrows = g->maxrows;
  const float qf = g->quantum_f, qif = g->quantum_inv_f;
  const int iy = cls % l2, iz = cls / l2;
  int nr;
  if (g->variant == NEMD_DS) {
    const int K = g->kfac, side = 2 * K + 1;
    nr = side * side;
    for (int e = lane; e < nr && e < maxrows; e += 32) {
      const int dz = e / side - K, dy = e % side - K;
      const int jyu = iy + dy, jzu = iz + dz;
      const int ky = floordiv_i(jyu, l2), kz = floordiv_i(jzu, l3);
      const int jy = jyu - ky * l2, jz = jzu - kz * l3;
      const float c1 = (float)dy, c2 = (float)dz;
      Row r;
      ff o[3];
#pragma unroll
      for (int a = 0; a < 3; a++)
        o[a] = ff_add(ff_mul_f(ff_of(g->Gff[3 * a + 1]), c1), ff_mul_f(ff_of(g->Gff[3 * a + 2]), c2));
      split_shift_ff(o[0], qf, qif, r.shx, r.srx);
      split_shift_ff(o[1], qf, qif, r.shy, r.sry);
      split_shift_ff(o[2], qf, qif, r.shz, r.srz);
      r.cbase = cell_base + l1 * (jy + l2 * jz);
      r.sxi = 0;
      r.dxlo = -K;
      r.cnt = 2 * K + 1;
      r.ky = (short)ky;
      r.kz = (short)kz;
      r.dir = dz > 0 || (dz == 0 && dy > 0) ? 1 : (dz == 0 && dy == 0 ? 0 : -1);
      out[e] = r;
    }
  } else {
    // window bounds in units of the cell sides (the grid's reciprocals): the
    // reach rce includes rc (1 + 1e-12), the wrap's tolerance on both sides and
    // one more wrap_tol for the float-float roundings here, so a bound that
    // moves by a rounding only adds or drops a cell lying farther than rc
    const ff rce = ff_of(g->rceff);
    const ff w1 = ff_of(g->wff[0]), w2 = ff_of(g->wff[1]), w3 = ff_of(g->wff[2]);
    const ff iw1 = ff_of(g->Ginvff[0]), iw2 = ff_of(g->Ginvff[1]), iw3 = ff_of(g->Ginvff[2]);
    const ff r12 = ff_of(g->Rff[1]), r13 = ff_of(g->Rff[2]), r23 = ff_of(g->Rff[5]);
    const int zlo = ff_floor_int(ff_mul(ff_sub(ff_mul_f(w3, (float)iz), rce), iw3));
    int zhi = ff_ceil_int(ff_mul(ff_add(ff_mul_f(w3, (float)(iz + 1)), rce), iw3)) - 1;
    if (zhi - zlo + 1 > kMaxZ) {
      if (lane == 0) atomicOr(&g->error, ERRB_CAPACITY);
      zhi = zlo + kMaxZ - 1;
    }
    // lane z: the y-window of z-row zlo + z; rows numbered z-row by z-row
    const int nz = zhi - zlo + 1;
    int ycnt_l = 0, ylo_l = 0;
    if (lane < nz) {
      const int jzu = zlo + lane;
      const int kz = floordiv_i(jzu, l3);
      const ff yshift = ff_mul_f(r23, (float)kz);
      ylo_l = ff_floor_int(ff_mul(ff_sub(ff_sub(ff_mul_f(w2, (float)iy), rce), yshift), iw2));
      const int hi = ff_ceil_int(ff_mul(ff_sub(ff_add(ff_mul_f(w2, (float)(iy + 1)), rce), yshift), iw2)) - 1;
      ycnt_l = hi - ylo_l + 1;
    }
    int ylo[kMaxZ], ycnt[kMaxZ];
    nr = 0;
#pragma unroll
    for (int z = 0; z < kMaxZ; z++) {
      ylo[z] = __shfl_sync(0xffffffffu, ylo_l, z);
      ycnt[z] = z < nz ? __shfl_sync(0xffffffffu, ycnt_l, z) : 0;
      nr += ycnt[z];
    }
    for (int e = lane; e < nr && e < maxrows; e += 32) {
      int z = 0, base = 0;
      while (z < kMaxZ - 1 && e >= base + ycnt[z]) base += ycnt[z++];
      const int jzu = zlo + z, jyu = ylo[z] + (e - base);
      const int kz = floordiv_i(jzu, l3), jz = jzu - kz * l3;
      const int ky = floordiv_i(jyu, l2), jy = jyu - ky * l2;
      const ff sx = ff_add(ff_mul_f(r12, (float)ky), ff_mul_f(r13, (float)kz));
      const int xlo = ff_floor_int(ff_mul(ff_sub(ff_neg(rce), sx), iw1));
      const int xhi = ff_ceil_int(ff_mul(ff_sub(ff_add(w1, rce), sx), iw1)) - 1;
      const float sxi = ff_rint(ff_mul(sx, iw1));
      Row r;
      split_shift_ff(ff_sub(sx, ff_mul_f(w1, sxi)), qf, qif, r.shx, r.srx);
      split_shift_ff(ff_add(ff_mul_f(w2, (float)(jyu - iy)), ff_mul_f(r23, (float)kz)), qf, qif, r.shy, r.sry);
      split_shift_ff(ff_mul_f(w3, (float)(jzu - iz)), qf, qif, r.shz, r.srz);
      r.cbase = cell_base + l1 * (jy + l2 * jz);
      r.sxi = (int)sxi;
      r.dxlo = xlo;
      r.cnt = xhi - xlo + 1;
      r.ky = (short)ky;
      r.kz = (short)kz;
      {
        const int dz = jzu - iz, dy = jyu - iy;
        r.dir = dz > 0 || (dz == 0 && dy > 0) ? 1 : (dz == 0 && dy == 0 ? 0 : -1);
      }
      out[e] = r;
    }
  }
  if (nr > maxrows) {
    if (lane == 0) atomicOr(&g->error, ERRB_CAPACITY);
    nr = maxrows;
  }
  return nr;
}

// One warp per home (iy, iz) class: the neighbour rows of that class.
__global__ void k_stencil(Geo *g, Row *rows, int *rowcnt) {
  if (g->error) return;
  const int ncls = g->nc[1] * g->nc[2];
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int cls = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; cls < ncls; cls += nw) {
    const int nr = stencil_class_warp(g, cls, 0, rows + (size_t)cls * g->maxrows, lane);
    if (lane == 0) rowcnt[cls] = nr;
  }
}

cudaError_t launch_lattice(nemd_ctx *c, int validate, double tau) {
  LatIn in;
  for (int k = 0; k < 9; k++) {
    in.A[k] = c->A[k];
    in.L0[k] = c->L0[k];
  }
  in.T = c->T;
  in.t = c->t;
  in.tau = tau;
  in.validate = validate;
  in.centered = c->remap_centered;
  in.t_dev = c->t_dev;
  k_lattice<<<1, 32, 0, c->stream>>>(c->geo, in);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_grid(nemd_ctx *c) {
  GridIn in;
  in.rc = c->rc;
  in.variant = c->variant_req;
  in.kfac = c->kfac;
  in.n = (int)c->n;
  in.max_cells = (int)c->cap_cells;
  const int ka = c->kfac_alloc > c->kfac ? c->kfac_alloc : c->kfac;
  in.row_stride = (2 * ka + 1) * (2 * ka + 2);
  k_grid<<<1, 32, 0, c->stream>>>(c->geo, in);
  c->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_stencil(nemd_ctx *c) {
  int64_t classes = c->cap_cells;  // l2 * l3 <= ncells <= cap
  int threads = 128;               // four classes per block
  int64_t blocks = (classes + 3) / 4;
  if (blocks > 8 * (int64_t)c->sms) blocks = 8 * (int64_t)c->sms;
  if (blocks < 1) blocks = 1;
  k_stencil<<<(int)blocks, threads, 0, c->stream>>>(c->geo, c->rows, c->rowcnt);
  c->launches += 1;
  return cudaGetLastError();
}


// ---- batches: one launch over every system (or every sampled state) ----

// One system per block (one warp).
__global__ void k_b_lattice(Geo *geo, const LatIn *__restrict__ lat, const double *__restrict__ t) {
  __shared__ LatScratch sc;
  LatIn in = lat[blockIdx.x];
  if (t) in.t = t[blockIdx.x];
  lattice_body(geo + blockIdx.x, in, sc);
}

// One thread per system, 128 per block: the grid is long straight-line
// float64 code run once, so few SMs (each fetching it once) do it fastest.
__global__ void k_b_grid(Geo *geo, const GridIn *__restrict__ grid, const SysInfo *__restrict__ sys, int count) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  Geo *g = geo + e;
  grid_body(g, grid[e]);
  // the batch sizes a system's row classes from its states over one period
  if (sys && !(g->error & ERRB_BOX) && (long long)g->nc[1] * g->nc[2] > (long long)sys[e].clcap) {
    g->error |= ERRB_CAPACITY;
    g->ncells = 0;
  }
}

// blockIdx.y = system; warps stride over its classes.
__global__ void k_b_stencil(BatchView v) {
  const int s = blockIdx.y;
  Geo *g = v.geo + s;
  if (g->error) return;
  const SysInfo si = v.sys[s];
  const int ncls = g->nc[1] * g->nc[2];
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int cls = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; cls < ncls; cls += nw) {
    const int slot = si.clo + cls;
    const int nr = stencil_class_warp(g, cls, si.coff, v.rows + (size_t)slot * kBatchRowStride, lane);
    if (lane == 0) v.rowcnt[slot] = nr;
  }
}

cudaError_t launch_batch_lattice(cudaStream_t st, Geo *geo, const LatIn *lat, const double *t, int count) {
  if (count <= 0) return cudaSuccess;
  k_b_lattice<<<count, 32, 0, st>>>(geo, lat, t);
  return cudaGetLastError();
}

cudaError_t launch_batch_grid(cudaStream_t st, Geo *geo, const GridIn *grid, const SysInfo *sys, int count) {
  if (count <= 0) return cudaSuccess;
  k_b_grid<<<(count + 127) / 128, 128, 0, st>>>(geo, grid, sys, count);
  return cudaGetLastError();
}

cudaError_t launch_batch_stencil(cudaStream_t st, const BatchView &v, int max_clcap) {
  const int threads = 128;  // four classes per block
  int bx = (max_clcap + 3) / 4;
  if (bx < 1) bx = 1;
  if (bx > 64) bx = 64;
  k_b_stencil<<<dim3(bx, v.nsys), threads, 0, st>>>(v);
  return cudaGetLastError();
}

}  // namespace nemd
