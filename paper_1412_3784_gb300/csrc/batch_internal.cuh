// batch_internal.cuh -- device layout of a batch of independent systems
// (nemd_batch_* in include/nemd.h) and the batched launch wrappers.
//
// All systems live in concatenated arrays.  System s owns
//   input particles  [poff, poff + n)            (q, F, sys_of)
//   cell slots       [coff, coff + ccap)         (count, start)
//   row classes      [clo, clo + clcap)          (rows, rowcnt, class_sys)
// and sorted particles [start[coff], start[coff + ncells]) after binning.  Every
// stage of a step is one launch over all systems; launch shapes depend only on
// the capacities, so the step is captured once into a CUDA graph and replayed.
#pragma once

#include "force_common.cuh"

struct nemd_batch;

namespace nemd {

// Rows per class the batch tables hold: (2k + 1)(2k + 2) at cell factor k = 2.
constexpr int kBatchMaxFactor = 2;
constexpr int kBatchRowStride = (2 * kBatchMaxFactor + 1) * (2 * kBatchMaxFactor + 2);

struct SysInfo {
  int n;      // particles
  int poff;   // first input particle
  int coff;   // first cell slot
  int ccap;   // cell slots
  int clo;    // first row class slot
  int clcap;  // row class slots
  int pad[2];
};

// Blocks per system of the batch's final reduction, and the sums each writes
// (U, six virial components, pairs).
constexpr int kReduceSplit = 4;
constexpr int kReduceSums = 8;

// Pointers and totals one batched step uses (passed by value to the kernels).
struct BatchView {
  int nsys, ntot, ncells, nclasses;  // systems; totals of particles, cell and class slots
  int gs;                            // particles per chunk (16 or 32)
  int wide;                          // chunks span up to Geo::span cells (row kernel), else kMaxSpan
  Geo *geo;
  const SysInfo *sys;
  const Pot *pot;
  const LatIn *lat;
  const GridIn *grid;
  const double *t;
  const int *sys_of;     // per input particle
  const int *class_sys;  // per class slot
  const double *q;
  float4 *relc, *relr;
  int *rank, *count, *start, *perm;
  float4 *pos4, *posr;
  int *cell_sorted;
  Row *rows;
  int *rowcnt;
  int *chunk_off;  // [nclasses]: the length of the chunk list
  int4 *chunks;
  int *work;     // dynamic chunk counter of the force kernel
  float4 *ppart;  // per sorted particle: {u, wxx, wyy, wzz}, {wxy, wxz, wyz, pairs (int bits)}
  int4 *recheck;
  int *nrecheck;
  unsigned long long *sys_counters;  // per system: candidates, band candidates
  unsigned long long *sys_pairs;     // per system: interacting pairs
  double *red_part;      // per system and reduction block: its kReduceSums sums
  unsigned *red_ticket;  // per system: reduction blocks finished (0 between steps)
  float *F;
  double *UW;  // per system: U, W[9]
};


// lattice.cu: one warp per entry; t (may be null) overrides lat[e].t
cudaError_t launch_batch_lattice(cudaStream_t st, Geo *geo, const LatIn *lat, const double *t, int count);
// lattice.cu: one thread per entry; sys (may be null) adds the class capacity check
cudaError_t launch_batch_grid(cudaStream_t st, Geo *geo, const GridIn *grid, const SysInfo *sys, int count);
// lattice.cu: rows of every class of every system
cudaError_t launch_batch_stencil(cudaStream_t st, const BatchView &v, int max_clcap);
// bin.cu: wrap, scan, scatter, rank within the cell and pack
cudaError_t launch_batch_bin(cudaStream_t st, const BatchView &v, int sms);
// One block: exclusive scan of the per-class chunk counts (c2 c3 classes from
// the grid), total at out[cap].
cudaError_t launch_class_scan(nemd_ctx *c, const int *in, int *out, int cap);
// force_chunk.cu: per-class chunk counts, their scan, the chunk list
cudaError_t launch_batch_chunks(cudaStream_t st, const BatchView &v, int sms);
// force_warp.cu: the persistent force kernel over every chunk of every system
// (blocks from batch_force_blocks, which must be called outside stream capture)
int batch_force_blocks(int sms);
cudaError_t launch_batch_force(cudaStream_t st, const BatchView &v, int blocks);
// the same with the row kernel (force_row.cu)
int batch_row_blocks(int sms);
cudaError_t launch_batch_force_row(cudaStream_t st, const BatchView &v, int blocks);
// force.cu: float64 fix-up of deferred candidates, per-system reductions
cudaError_t launch_batch_finish(cudaStream_t st, const BatchView &v);

}  // namespace nemd
