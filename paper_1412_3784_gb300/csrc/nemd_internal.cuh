// nemd_internal.cuh -- device data layout shared by the CUDA translation units.
//
// Geometry of one evaluation lives in a device-resident Geo record written by
// the lattice kernel (Sec. 2.1-2.2 lattice, Sec. 4.1/4.2 cell grid) and read by
// every later kernel, so the host never waits for the device between steps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nemd.h"

namespace nemd {

// Relative safety margin of the cell counts and stencil intervals: counts are
// floor((1 - kMargin) k h / rc) and intervals use rc (1 + kMargin), so FP64
// rounding of positions can never drop a pair.
constexpr double kMargin = 1e-12;
constexpr int kMaxFactor = 3;          // largest cell-size factor k
constexpr int kMaxSpan = 8;            // x-span (cells) of a chunk of the grouped and row kernels ...
constexpr int kMaxSpanCap = 32;        // ... widened up to this where cells hold few particles
constexpr int kRecheckCap = 1 << 14;   // fine-band candidates per evaluation (~1e-7 of candidates)
constexpr int kFixupBlocks = 16;       // blocks of the float64 fix-up pass (when partial slots allow)
constexpr int kMaxRowsPerClass = 64;   // (2k+2)^2 for k = 3

// Device error word bits (deferred errors).
enum : int {
  ERRB_BOX = 1,
  ERRB_NONFINITE = 2,
  ERRB_CAPACITY = 4,
  ERRB_TIMEOUT = 8,
};

struct Geo {
  // ---- inputs (host-written) ----
  double A[9], L0[9];
  double T;
  double t;
  double rc, rc2;
  int variant;   // NEMD_DS / NEMD_DO actually used for this step
  int req_variant;
  int kfac;
  int max_cells;  // host bound on the number of cells (allocation size)
  // ---- lattice (a1) ----
  double tau;
  double L[9], Linv[9], V, h[3], Q[9], R[9];
  double rinv[3];  // 1 / r_ii
  // ---- grid (a3) ----
  int nc[3];
  int ncells;
  int maxrows;        // row stride per (iy, iz) class
  int span;           // largest x-span (cells) of a chunk this step
  int reach[3];       // stencil reach in cells per axis
  double G[9];        // frame position of cell corner = G * (ix, iy, iz)
  double Ginv_scale[3];  // DS: c_i ; DO: 1 / w_i
  double w[3];        // DO cell sides
  float Gf[9];
  float step[3];      // frame vector from one x-cell to the next: quantised part
  float step_r[3];    //   and its residual
  float Qf[9];        // rotation frame -> Cartesian (identity for DS)
  float rc2_lo, rc2_hi, rc2f;   // coarse band: quantised test without residuals
  float rc2_lo2, rc2_hi2;       // fine band: float32 test with residuals added back
  float band;
  // coordinate along the x-rows in cell units: kappa = kap . rel is in
  // [-1/2, 1/2] inside a cell (dynamic size: u1 - 1/2; dynamic offset: x / w1);
  // two particles whose kappa positions along a row differ by more than rho1
  // are farther apart than rc
  float kap[3];
  float rho1;
  // float-float (hi, lo) copies of the wrap's frame data: R, 1 / r_ii, G, the
  // dynamic offset 1 / w_i and w_i.  The wrap works in float-float after the
  // float64 fractional coordinates; wrap_tol bounds its position error.
  // rceff: the dynamic offset stencil's reach rc (1 + 1e-12) + 3 wrap_tol.
  float2 Rff[9], rinvff[3], Gff[9], Ginvff[3], wff[3], Linvff[9], rceff;
  double wrap_tol;
  float quantum_f, quantum_inv_f;  // the quantum and its inverse (powers of two) as float
  double quantum;     // float32 coordinates and offsets are multiples of this power of 2
  double quantum_inv;  // 1 / quantum (exact)
  double vol_ds, vol_do;  // neighbourhood volumes (Sec. 5.1, 5.2) of both variants
  int counts_ds[3], counts_do[3];
  int error;   // this step's error bits
  int sticky;  // error bits accumulated until the host reads them (nemd_sync)
  int learned_choice;  // option picked by the learned selector this step, -1 if none
  int pad_lc;
};

// Launch inputs, passed by value so that asynchronous launches and captured
// graphs see the values of the call that issued them.
struct LatIn {
  double A[9], L0[9];
  double T, t, tau;
  int validate;
  int centered;  // remap half way through the period: tau in [-T/2, T/2)
  const double *t_dev = nullptr;  // when set, t is read here (device memory: captured steps)
};

struct GridIn {
  double rc;
  int variant, kfac, max_cells, row_stride;
  int n;  // particles of the system (0: unknown, Geo::span = kMaxSpan)
};

// One neighbour row of a home (iy, iz) class: the x-cells ix+dxlo ... ix+dxlo+cnt-1
// of the wrapped row (jy, jz), reached through lattice image (kx, ky, kz) where kx
// follows from the x wrap.  The frame vector from the home cell's centre to the
// centre of the cell ix+dx of this row is  shift + (dx + sxi) * step  (step =
// Geo::step); shift is split into an exact multiple of Geo::quantum (shx, shy,
// shz) and a float32 residual (srx, sry, srz), and kept within half a cell
// along x by the integer sxi.  The home cell's own row has shift 0 and sxi 0,
// so the offset of the home cell itself is exactly 0.  dir orders the rows for
// half neighbourhoods: +1 when the row lies ahead of the home row (dz > 0, or
// dz = 0 and dy > 0, in unwrapped cell offsets), 0 for the home row itself,
// -1 behind; a pair met through a +1 row is met through a -1 row from its
// partner's side, so a half neighbourhood visits +1 rows and the forward half
// of the home row.
struct __align__(16) Row {
  float shx, shy, shz;
  int cbase;   // l1 * (jy + l2 * jz)
  float srx, sry, srz;
  int dxlo;
  int cnt;
  short ky, kz;
  int sxi;
  int dir;
};
static_assert(sizeof(Row) == 48, "Row is 48 bytes");

// Geometry of the Verlet-list force at one step (verlet.cu): the list's
// dynamic size grid c (cells at least rc + skin wide, fixed at the build), the
// current cell vectors G = L(t) / c (float64, and as an exact multiple of the
// quantum plus a float32 residual), and the float32 bands of the cut-off.
struct VlGeo {
  int c[3];
  int pad;
  double G[9];
  float Gq[9], Gr[9];
  float quantum_f, quantum_inv_f;
  double quantum, quantum_inv;
  float rc2_lo, rc2_hi, rc2_lo2, rc2_hi2;
  double rl;  // rc + skin
  float2 Gff[9];  // G in float-float (hi, lo)
  float Lf[9];    // L(t) rounded to float (peculiar displacements)
};

// Per-block partial sums of the force kernel (float64): U, W (6 symmetric
// components xx yy zz xy xz yz), interacting pairs, candidates, rechecks.
constexpr int kPartials = 10;

// Learned selector: 12 inputs -> 64 -> 64 -> 4 outputs (float32).
constexpr int kMlpIn = 12, kMlpHidden = 64, kMlpOut = 4;
constexpr int kMlpParams = kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden +
                           kMlpOut * kMlpHidden + kMlpOut;

// Autotuner cache: per shape class, the summed mean time and the number of
// measurements of every candidate configuration.
constexpr int kTuneCandidates = 13;
constexpr int kMaxTuneClasses = 64;
struct TuneEntry {
  int32_t key[2];
  double sum_ms[kTuneCandidates];
  int64_t count[kTuneCandidates];
};

}  // namespace nemd

// Context (opaque to callers).
struct nemd_ctx {
  int device;
  cudaStream_t stream;
  int sms;
  // flow / potential
  double A[9], L0[9], T;
  int64_t M[9];
  bool have_flow, have_pot, have_state, have_cells;
  int pot_kind;
  double eps, sigma;
  int shift;
  int remap_centered;  // NEMD_OPT_REMAP
  // state
  int64_t n;
  double t;
  const double *q_dev;  // device positions (user's or internal copy)
  double rc;
  int variant_req;
  // options
  int precise;
  int64_t record_cap;
  int kernel;
  int kfac;
  int kfac_alloc;  // cell factor the buffers of the current step are sized for
  int block;
  // device memory
  nemd::Geo *geo;
  int64_t cap_n;
  int64_t cap_cells;
  int64_t cap_rows;
  double *q_copy;
  float4 *relc;          // per input particle: frame rel position + cell (bits) in w
  int *rank;
  int *count;            // cap_cells + 1
  int *start;            // cap_cells + 1
  int *block_sums;
  int *perm;
  float4 *relr;          // per input particle: residual of the quantised rel position
  float4 *pos4;          // sorted: quantised rel position + original index (bits)
  float4 *posr;          // sorted: residual of the quantised rel position
  int *cell_sorted;
  nemd::Row *rows;
  int *rowcnt;
  double *partials;
  int64_t cap_partials;
  double *uw_out;        // device U (1) + W (9)
  unsigned long long *fix_f;  // 3 per particle: the fix-up's forces in 64-bit fixed point (kept zero between uses)
  unsigned long long *fix_uw; // 8: the fix-up's U, W and pair count in fixed point (kept zero between uses)
  int64_t fix_cap;            // particles fix_f holds
  float *f_dev;          // internal F buffer (host outputs)
  int32_t *pair_buf;
  unsigned long long *pair_count;
  unsigned long long *counters;  // [0] pairs [1] candidates [2] rechecks
  // force-kernel timing (CUDA events on the context's stream)
  int timing;
  cudaEvent_t *ev;
  int ev_cap, ev_n;
  int64_t launches;
  // host staging
  int *h_error;  // pinned
  // grouped force kernel
  int4 *chunks;
  int *nchunks;
  int *chunk_cnt, *chunk_off;  // per class slot: chunks, their scan (total at [cap_cells])
  int group;
  // candidates left within float32 rounding of rc, decided by the float64 fix-up
  int4 *recheck;
  int *nrecheck;
  // learned selector: params | input mean, std | target mean, std | Adam state (device)
  float *model;
  int have_model;
  float model_norm_host[2 * nemd::kMlpIn + 2];
  // autotuner cache (host)
  int autotuned;
  int ntune;
  nemd::TuneEntry tune[nemd::kMaxTuneClasses];
  char msg[512];
  double last_stats_band;
  // asynchronous host input/output (NEMD_OPT_ASYNC_HOST): double-buffered device
  // copies on a copy stream, ordered against the context's stream by events
  int async_host;
  int aslot;                  // buffer pair of the current evaluation
  int64_t acap;               // particles the async buffers hold
  cudaStream_t copy_stream;   // host -> device
  cudaStream_t copy_back;     // device -> host (a separate queue: an output copy waits for
                              // its evaluation, the next input copy must not wait behind it)
  cudaEvent_t ev_q[2], ev_done[2], ev_out[2];
  bool done_valid[2], out_valid[2];
  double *aq[2];              // positions copied from the host
  float *af[2];               // forces copied to the host
  double *auw[2];             // U, W copied to the host
  // time integration (nemd_integrate): propagators and thermostat state,
  // per-block sums of |p|^2, forces of the current step
  double *int_state;
  double *int_part;
  float *f_int;
  int64_t f_int_cap;
  const double *t_dev;  // while integrating: the lattice reads the time from here
  int int_graph;        // NEMD_OPT_INT_GRAPH: replay a captured step (default 1)
  cudaStream_t cap_stream;  // private stream the step is captured on
  // Verlet list of nemd_integrate (nemd_set_verlet): pairs within rc + skin of
  // the last build, per sorted particle in ELL layout (entry e of particle k at
  // vl_ent[e * vl_n + k])
  double vl_skin;           // 0: off
  int64_t vl_capn;          // particles the per-particle buffers hold
  int64_t vl_capent;        // entries vl_ent holds
  int64_t vl_n;             // particles of the current list
  int vl_maxk;              // most entries of one particle in the current list
  int *vl_cnt;              // per sorted particle: its entries
  int2 *vl_ent;             // (sorted j, packed cell offset)
  int *vl_slot;             // per input particle: its sorted slot at the build
  double *vl_sb;            // per sorted particle: fractional position at the build (3)
  int4 *vl_idx;             // per sorted particle: list cell (x, y, z), brick image (packed) in w
  float4 *vl_pos, *vl_res;  // per sorted particle, per step: position in its cell and residual
                            // interleaved in vl_pos (vl_res unused)
  nemd::VlGeo *vl_geo;      // device
  unsigned *vl_disp;        // device: largest displacement (float bits), its maximum entry count
  unsigned *h_vl;           // pinned host copy of vl_disp[0..1]
  int64_t vl_builds, vl_steps;
  double vl_tb;             // time of the last build
  double vl_delta;          // largest displacement measured at the last check
  long long vl_period;      // remap period of the last build
};

namespace nemd {

// ---- kernels (launch wrappers implemented in the .cu files) ----
cudaError_t launch_lattice(nemd_ctx *c, int validate, double tau);
cudaError_t launch_grid(nemd_ctx *c);
cudaError_t launch_stencil(nemd_ctx *c);
cudaError_t launch_bin(nemd_ctx *c);
cudaError_t launch_forces(nemd_ctx *c, float *F_dev, double *UW_dev);
cudaError_t launch_recheck_fixup(nemd_ctx *c, float *F_dev, double *UW_dev, int nblocks, bool half,
                                 bool frame_is_cartesian);
// Verlet list of nemd_integrate (verlet.cu): forces of the current state
int verlet_forces(nemd_ctx *c, float *F, int variant, double rc, double t);
// grouped force kernel: chunk list, then the kernel (returns the number of
// blocks whose partials it wrote)
bool chunk_kernel_applies(const nemd_ctx *c);
bool warp_kernel_applies(const nemd_ctx *c);
cudaError_t launch_chunk_build(nemd_ctx *c, int gs, bool wide);
cudaError_t launch_force_warp(nemd_ctx *c, float *F_dev, int *nblocks, bool half);
// row kernel (per-lane kappa windows, half-precision coarse test)
bool row_kernel_applies(const nemd_ctx *c);
cudaError_t launch_force_row(nemd_ctx *c, float *F_dev, int *nblocks);
// autotuner cache lookup (autotune.cu)
void tune_apply(nemd_ctx *c, double rc);
// learned selector inference for this step (mlp.cu)
cudaError_t launch_learned_choice(nemd_ctx *c, double rc);
cudaError_t launch_force_chunk(nemd_ctx *c, float *F_dev, int *nblocks);
// status code and message of a set of device error bits (capi.cu)
int status_from_bits(int bits, const char **what);

}  // namespace nemd
