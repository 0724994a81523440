// batch.cu -- batches of independent systems (nemd_batch_* in include/nemd.h).
// The paper treats one system at a time; here every stage of a step is one
// launch over all systems (layout in batch_internal.cuh), the whole step is
// captured once into a CUDA graph and replayed.  This file is host code only:
// validation, sizing, allocation, capture and the C ABI.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "batch_internal.cuh"

using nemd::BatchView;
using nemd::Geo;
using nemd::GridIn;
using nemd::LatIn;
using nemd::Pot;
using nemd::Row;
using nemd::SysInfo;

struct nemd_batch {
  int device;
  cudaStream_t stream;      // the caller's stream: every step runs on it
  cudaStream_t cap_stream;  // internal stream the graph is captured on
  int sms;
  nemd_ctx *check;  // validates flows and potentials exactly as a context does
  std::vector<nemd_system> systems;
  std::vector<Pot> pots;
  std::vector<GridIn> grid_host;  // per system: rc, requested variant, cell factor, capacities
  bool finalized;
  int kfac, gs, use_graph;
  int force_kernel;  // 2 warp kernel, 4 row kernel
  int force_blocks, row_blocks;
  int max_clcap;
  std::vector<int64_t> offsets;
  // device tables
  BatchView v;
  SysInfo *sys_dev;
  LatIn *lat_dev;
  GridIn *grid_dev;
  Pot *pot_dev;
  double *t_dev;
  double *q_copy;
  float *f_int;
  double *uw_int;
  int *err_dev;
  int *h_err;  // pinned, nsys
  bool have_state;
  const double *q_cur;
  // captured step
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  const void *key[3];
  int key_cfg[3];
  int64_t launches;  // kernel launches of one step
  char msg[512];
};

namespace {

int set_err(nemd_batch *b, int code, const char *fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->msg, sizeof b->msg, fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_err(nemd_batch *b, cudaError_t e, const char *where) {
  return set_err(b, NEMD_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CKB(call)                                         \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_err(b, e_, #call); \
  } while (0)

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
int alloc(nemd_batch *b, T **p, int64_t count, const char *what) {
  if (count <= 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_err(b, NEMD_ERR_NOMEM, "cudaMalloc of %s (%lld elements) failed", what, (long long)count);
  }
  return NEMD_OK;
}

double det3(const double *a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
}

__global__ void k_b_errors(Geo *geo, int *out, int nsys, int clear) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    out[s] = geo[s].sticky | geo[s].error;
    if (clear) {
      geo[s].sticky = 0;
      geo[s].error = 0;
    }
  }
}

void drop_graph(nemd_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// The kernels of one step on stream st (also what the graph captures).
cudaError_t enqueue_step(nemd_batch *b, cudaStream_t st) {
  BatchView &v = b->v;
  cudaError_t e;
  if ((e = nemd::launch_batch_lattice(st, v.geo, b->lat_dev, b->t_dev, v.nsys)) != cudaSuccess) return e;
  if ((e = nemd::launch_batch_grid(st, v.geo, b->grid_dev, b->sys_dev, v.nsys)) != cudaSuccess) return e;
  if ((e = nemd::launch_batch_stencil(st, v, b->max_clcap)) != cudaSuccess) return e;
  if ((e = nemd::launch_batch_bin(st, v, b->sms)) != cudaSuccess) return e;
  if ((e = nemd::launch_batch_chunks(st, v, b->sms)) != cudaSuccess) return e;
  if ((e = (b->force_kernel == 4 ? nemd::launch_batch_force_row(st, v, b->row_blocks)
                                  : nemd::launch_batch_force(st, v, b->force_blocks))) != cudaSuccess)
    return e;
  return nemd::launch_batch_finish(st, v);
}

// lattice, grid, stencil, bin (wrap, scan, scatter, rank-and-pack), chunk
// list, force, fix-up, reduce
constexpr int64_t kStepLaunches = 3 + 4 + 1 + 1 + 2;

}  // namespace

extern "C" {

int nemd_batch_create(nemd_batch **out, int device, void *stream) {
  if (!out) return NEMD_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return NEMD_ERR_CUDA;
  }
  nemd_batch *b = new nemd_batch();
  b->device = device;
  b->stream = (cudaStream_t)stream;
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, device);
  b->kfac = 1;
  b->gs = 32;
  b->force_kernel = 4;
  b->use_graph = 1;
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      nemd_create(&b->check, device, stream) != NEMD_OK) {
    cudaGetLastError();
    nemd_batch_destroy(b);
    return NEMD_ERR_CUDA;
  }
  snprintf(b->msg, sizeof b->msg, "ok");
  *out = b;
  return NEMD_OK;
}

int nemd_batch_destroy(nemd_batch *b) {
  if (!b) return NEMD_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  BatchView &v = b->v;
  void *ptrs[] = {v.geo,      (void *)v.sys_of,  (void *)v.class_sys, v.relc,       v.relr,      v.rank,   v.count,     v.start,
                  v.perm,    v.pos4,      v.posr,       v.cell_sorted, v.rows, v.rowcnt,
                  v.chunk_off, v.chunks, v.work,     v.ppart,     v.recheck, v.nrecheck, v.sys_counters,
                  v.sys_pairs, v.red_part, v.red_ticket, b->sys_dev, b->lat_dev, b->grid_dev, b->pot_dev,  b->t_dev, b->q_copy,   b->f_int,
                  b->uw_int,  b->err_dev};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (b->h_err) cudaFreeHost(b->h_err);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->check) nemd_destroy(b->check);
  cudaGetLastError();
  delete b;
  return NEMD_OK;
}

const char *nemd_batch_last_error(const nemd_batch *b) { return b ? b->msg : "null batch"; }

int nemd_batch_add(nemd_batch *b, const nemd_system *sys, int64_t *index) {
  if (!b || !sys) return set_err(b, NEMD_ERR_ARG, "batch_add: null argument");
  if (b->finalized) return set_err(b, NEMD_ERR_ORDER, "batch_add after finalize");
  if (sys->n < 0 || sys->n > (int64_t)1 << 21)
    return set_err(b, NEMD_ERR_ARG, "batch_add: N = %lld outside 0 .. 2^21", (long long)sys->n);
  if (sys->variant != NEMD_DS && sys->variant != NEMD_DO && sys->variant != NEMD_AUTO_HEURISTIC)
    return set_err(b, NEMD_ERR_ARG, "batch_add: variant %d (DS, DO or AUTO_HEURISTIC)", sys->variant);
  if (sys->remap != 0 && sys->remap != 1) return set_err(b, NEMD_ERR_ARG, "batch_add: remap %d", sys->remap);
  const double rc = sys->rc;
  if (!(rc > 0.0) || !isfinite(rc)) return set_err(b, NEMD_ERR_ARG, "batch_add: rc must be > 0");
  if (sys->kind == NEMD_WCA && fabs(rc - pow(2.0, 1.0 / 6.0) * sys->sigma) > 1e-12 * sys->sigma)
    return set_err(b, NEMD_ERR_ARG, "batch_add: WCA needs rc = 2^(1/6) sigma");
  int r = nemd_set_flow(b->check, sys->A, sys->L0, sys->M, sys->T);
  if (!r) r = nemd_set_potential(b->check, sys->kind, sys->eps, sys->sigma, sys->shift);
  if (r) return set_err(b, r, "batch_add (system %zu): %s", b->systems.size(), nemd_last_error(b->check));
  const double V = fabs(det3(sys->L0));
  const double k = nemd::kBatchMaxFactor;
  if (k * k * k * V / (rc * rc * rc) > 1.0e8)
    return set_err(b, NEMD_ERR_ARG, "batch_add: %g cell slots is too many", k * k * k * V / (rc * rc * rc));
  // potential constants of this system, as a context computes them
  b->check->rc = rc;
  b->pots.push_back(nemd::make_pot(b->check));
  b->systems.push_back(*sys);
  // a context keeps T = 1 for A = 0 (the period plays no part then)
  double amax = 0.0;
  for (int q = 0; q < 9; q++) amax = fmax(amax, fabs(sys->A[q]));
  if (amax == 0.0 && !(sys->T > 0.0)) b->systems.back().T = 1.0;
  if (index) *index = (int64_t)b->systems.size() - 1;
  return NEMD_OK;
}

int nemd_batch_finalize(nemd_batch *b) {
  if (!b) return NEMD_ERR_ARG;
  if (b->finalized) return set_err(b, NEMD_ERR_ORDER, "batch already finalized");
  const int S = (int)b->systems.size();
  if (S < 1) return set_err(b, NEMD_ERR_ARG, "batch_finalize: no systems");
  if (S > 65535) return set_err(b, NEMD_ERR_ARG, "batch_finalize: %d systems (at most 65535)", S);
  CKB(cudaSetDevice(b->device));
  // ---- particles and cell slots ----
  std::vector<SysInfo> si(S);
  b->offsets.assign(S + 1, 0);
  int64_t ntot = 0, ncells = 0;
  for (int s = 0; s < S; s++) {
    const nemd_system &y = b->systems[s];
    const double k = nemd::kBatchMaxFactor;
    const double V = fabs(det3(y.L0));
    // c1 c2 c3 <= k^3 h1 h2 h3 / rc^3 <= k^3 V / rc^3 at every strain (the same for l_i)
    const int64_t ccap = (int64_t)(k * k * k * V / (y.rc * y.rc * y.rc) * (1.0 + 1e-9)) + 2;
    memset(&si[s], 0, sizeof si[s]);
    si[s].n = (int)y.n;
    si[s].poff = (int)ntot;
    si[s].coff = (int)ncells;
    si[s].ccap = (int)ccap;
    ntot += y.n;
    ncells += ccap;
    b->offsets[s + 1] = ntot;
    if (ntot > (int64_t)1 << 29 || ncells > (int64_t)1 << 30)
      return set_err(b, NEMD_ERR_ARG, "batch_finalize: %lld particles / %lld cell slots is too many",
                     (long long)ntot, (long long)ncells);
  }
  // ---- row classes: largest l2 l3 (c2 c3) over states of one period, both variants, k = 2 ----
  const int K = 256;
  const int ne = S * (K + 1);
  std::vector<LatIn> lat(ne);
  std::vector<GridIn> gin(ne);
  for (int s = 0; s < S; s++) {
    const nemd_system &y = b->systems[s];
    for (int k = 0; k <= K; k++) {
      LatIn &L = lat[(size_t)s * (K + 1) + k];
      memcpy(L.A, y.A, sizeof L.A);
      memcpy(L.L0, y.L0, sizeof L.L0);
      L.T = y.T;
      // K evenly spaced states and the state just before the remap (largest skew)
      L.t = (k < K) ? y.T * (double)k / K : y.T * (1.0 - ldexp(1.0, -20));
      L.tau = 0.0;
      L.validate = 0;
      L.centered = y.remap;
      GridIn &G = gin[(size_t)s * (K + 1) + k];
      G.rc = y.rc;
      G.n = (int)y.n;
      G.kfac = nemd::kBatchMaxFactor;
      G.max_cells = 0x7fffffff;
      G.row_stride = 1 << 20;
    }
  }
  Geo *gs_dev = nullptr;
  LatIn *lat_tmp = nullptr;
  GridIn *gin_tmp = nullptr;
  int r = alloc(b, &gs_dev, ne, "sample geometry");
  if (!r) r = alloc(b, &lat_tmp, ne, "sample lattice inputs");
  if (!r) r = alloc(b, &gin_tmp, ne, "sample grid inputs");
  std::vector<int64_t> maxcls(S, 1);
  cudaError_t e = cudaSuccess;
  if (!r) {
    std::vector<Geo> host(ne);
    e = cudaMemcpyAsync(lat_tmp, lat.data(), sizeof(LatIn) * ne, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(gs_dev, 0, sizeof(Geo) * ne, b->stream);
    if (e == cudaSuccess) e = nemd::launch_batch_lattice(b->stream, gs_dev, lat_tmp, nullptr, ne);
    for (int variant = NEMD_DS; variant <= NEMD_DO && e == cudaSuccess; variant++) {
      for (auto &G : gin) G.variant = variant;
      e = cudaMemcpyAsync(gin_tmp, gin.data(), sizeof(GridIn) * ne, cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess) e = nemd::launch_batch_grid(b->stream, gs_dev, gin_tmp, nullptr, ne);
      if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), gs_dev, sizeof(Geo) * ne, cudaMemcpyDeviceToHost, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) break;
      for (int s = 0; s < S; s++)
        for (int k = 0; k <= K; k++) {
          const Geo &g = host[(size_t)s * (K + 1) + k];
          const int64_t c = (int64_t)(g.nc[1] > 0 ? g.nc[1] : 0) * (g.nc[2] > 0 ? g.nc[2] : 0);
          if (c > maxcls[s]) maxcls[s] = c;
        }
    }
  }
  if (gs_dev) cudaFree(gs_dev);
  if (lat_tmp) cudaFree(lat_tmp);
  if (gin_tmp) cudaFree(gin_tmp);
  if (r) return r;
  if (e != cudaSuccess) return cuda_err(b, e, "batch_finalize sampling");
  int64_t nclasses = 0;
  b->max_clcap = 1;
  for (int s = 0; s < S; s++) {
    int64_t cl = (int64_t)ceil(1.25 * (double)maxcls[s]) + 16;
    if (cl > si[s].ccap) cl = si[s].ccap;
    si[s].clo = (int)nclasses;
    si[s].clcap = (int)cl;
    nclasses += cl;
    if (cl > b->max_clcap) b->max_clcap = (int)cl;
    if (nclasses * nemd::kBatchRowStride > (int64_t)1 << 31)
      return set_err(b, NEMD_ERR_ARG, "batch_finalize: %lld row classes is too many", (long long)nclasses);
  }
  // ---- host-built maps ----
  std::vector<int> sys_of(ntot > 0 ? ntot : 1), class_sys(nclasses);
  for (int s = 0; s < S; s++) {
    for (int i = 0; i < si[s].n; i++) sys_of[si[s].poff + i] = s;
    for (int c = 0; c < si[s].clcap; c++) class_sys[si[s].clo + c] = s;
  }
  lat.resize(S);
  gin.resize(S);
  for (int s = 0; s < S; s++) {
    const nemd_system &y = b->systems[s];
    memcpy(lat[s].A, y.A, sizeof lat[s].A);
    memcpy(lat[s].L0, y.L0, sizeof lat[s].L0);
    lat[s].T = y.T;
    lat[s].t = 0.0;
    lat[s].tau = 0.0;
    lat[s].validate = 0;
    lat[s].centered = y.remap;
    gin[s].rc = y.rc;
    gin[s].n = (int)y.n;
    gin[s].variant = y.variant;
    gin[s].kfac = b->kfac;
    gin[s].max_cells = si[s].ccap;
    gin[s].row_stride = nemd::kBatchRowStride;
  }
  // ---- allocation ----
  BatchView &v = b->v;
  v.nsys = S;
  v.ntot = (int)ntot;
  v.ncells = (int)ncells;
  v.nclasses = (int)nclasses;
  v.gs = b->gs;
  v.wide = b->force_kernel == 4;
  const int64_t np = ntot > 0 ? ntot : 1;
  // clang-format off
  if ((r = alloc(b, &v.geo, S, "geo")) || (r = alloc(b, &b->sys_dev, S, "systems")) ||
      (r = alloc(b, &b->lat_dev, S, "lattice inputs")) || (r = alloc(b, &b->grid_dev, S, "grid inputs")) ||
      (r = alloc(b, &b->pot_dev, S, "potentials")) || (r = alloc(b, &b->t_dev, S, "times")) ||
      (r = alloc(b, (int **)&v.sys_of, np, "sys_of")) || (r = alloc(b, (int **)&v.class_sys, nclasses, "class_sys")) ||
      (r = alloc(b, &v.relc, np, "relc")) || (r = alloc(b, &v.relr, np, "relr")) ||
      (r = alloc(b, &v.rank, np, "rank")) || (r = alloc(b, &v.perm, np, "perm")) ||
      (r = alloc(b, &v.pos4, np, "pos4")) || (r = alloc(b, &v.posr, np, "posr")) ||
      (r = alloc(b, &v.cell_sorted, np, "cell_sorted")) || (r = alloc(b, &v.ppart, 2 * np, "pair sums")) ||
      (r = alloc(b, &v.chunks, np, "chunks")) ||
      (r = alloc(b, &v.count, ncells + 1, "count")) || (r = alloc(b, &v.start, ncells + 1, "start")) ||
      (r = alloc(b, &v.rows, nclasses * nemd::kBatchRowStride, "rows")) ||
      (r = alloc(b, &v.rowcnt, nclasses, "rowcnt")) ||
      (r = alloc(b, &v.chunk_off, nclasses + 1, "chunk offsets")) ||
      (r = alloc(b, &v.work, 1, "work")) ||
      (r = alloc(b, &v.recheck, nemd::kRecheckCap, "recheck")) || (r = alloc(b, &v.nrecheck, 1, "nrecheck")) ||
      (r = alloc(b, &v.sys_counters, 2 * S, "counters")) || (r = alloc(b, &v.sys_pairs, S, "pairs")) ||
      (r = alloc(b, &v.red_part, (int64_t)nemd::kReduceSums * nemd::kReduceSplit * S, "reduction partials")) || (r = alloc(b, &v.red_ticket, S, "tickets")) ||
      (r = alloc(b, &b->uw_int, 10 * S, "UW")) || (r = alloc(b, &b->err_dev, S, "errors")))
    return r;
  // clang-format on
  if (cudaMallocHost((void **)&b->h_err, sizeof(int) * S) != cudaSuccess) {
    cudaGetLastError();
    return set_err(b, NEMD_ERR_NOMEM, "pinned error words");
  }
  v.sys = b->sys_dev;
  v.pot = b->pot_dev;
  v.lat = b->lat_dev;
  v.grid = b->grid_dev;
  v.t = b->t_dev;
  CKB(cudaMemsetAsync(v.geo, 0, sizeof(Geo) * S, b->stream));
  CKB(cudaMemsetAsync(v.sys_pairs, 0, sizeof(unsigned long long) * S, b->stream));
  CKB(cudaMemsetAsync(v.red_ticket, 0, sizeof(unsigned) * S, b->stream));
  CKB(cudaMemsetAsync(v.sys_counters, 0, 2 * sizeof(unsigned long long) * S, b->stream));
  CKB(cudaMemcpyAsync(b->sys_dev, si.data(), sizeof(SysInfo) * S, cudaMemcpyHostToDevice, b->stream));
  CKB(cudaMemcpyAsync(b->lat_dev, lat.data(), sizeof(LatIn) * S, cudaMemcpyHostToDevice, b->stream));
  b->grid_host = gin;
  CKB(cudaMemcpyAsync(b->grid_dev, b->grid_host.data(), sizeof(GridIn) * S, cudaMemcpyHostToDevice, b->stream));
  CKB(cudaMemcpyAsync(b->pot_dev, b->pots.data(), sizeof(Pot) * S, cudaMemcpyHostToDevice, b->stream));
  CKB(cudaMemcpyAsync((int *)v.sys_of, sys_of.data(), sizeof(int) * sys_of.size(), cudaMemcpyHostToDevice, b->stream));
  CKB(cudaMemcpyAsync((int *)v.class_sys, class_sys.data(), sizeof(int) * nclasses, cudaMemcpyHostToDevice,
                      b->stream));
  CKB(cudaStreamSynchronize(b->stream));
  b->force_blocks = nemd::batch_force_blocks(b->sms);
  b->row_blocks = nemd::batch_row_blocks(b->sms);
  b->launches = kStepLaunches;
  b->finalized = true;
  return NEMD_OK;
}

int nemd_batch_offsets(const nemd_batch *b, int64_t *offsets, int64_t *nsys) {
  if (!b) return NEMD_ERR_ARG;
  if (nsys) *nsys = (int64_t)b->systems.size();
  if (offsets) {
    int64_t acc = 0;
    offsets[0] = 0;
    for (size_t s = 0; s < b->systems.size(); s++) offsets[s + 1] = (acc += b->systems[s].n);
  }
  return NEMD_OK;
}

int nemd_batch_set_state(nemd_batch *b, const double *q, const double *t) {
  if (!b) return NEMD_ERR_ARG;
  if (!b->finalized) return set_err(b, NEMD_ERR_ORDER, "batch_set_state before finalize");
  if (!t || (!q && b->v.ntot > 0)) return set_err(b, NEMD_ERR_ARG, "batch_set_state: null argument");
  const int S = b->v.nsys;
  for (int s = 0; s < S; s++)
    if (!isfinite(t[s])) return set_err(b, NEMD_ERR_ARG, "batch_set_state: non-finite t of system %d", s);
  CKB(cudaSetDevice(b->device));
  CKB(cudaMemcpyAsync(b->t_dev, t, sizeof(double) * S, cudaMemcpyHostToDevice, b->stream));
  if (b->v.ntot > 0) {
    if (is_device_ptr(q)) {
      b->q_cur = q;
    } else {
      if (!b->q_copy) {
        int r = alloc(b, &b->q_copy, 3 * (int64_t)b->v.ntot, "q copy");
        if (r) return r;
      }
      CKB(cudaMemcpyAsync(b->q_copy, q, sizeof(double) * 3 * (size_t)b->v.ntot, cudaMemcpyHostToDevice, b->stream));
      b->q_cur = b->q_copy;
    }
  }
  b->have_state = true;
  return NEMD_OK;
}

int nemd_batch_compute(nemd_batch *b, float *F, double *UW) {
  if (!b) return NEMD_ERR_ARG;
  if (!b->have_state) return set_err(b, NEMD_ERR_ORDER, "batch_compute before batch_set_state");
  CKB(cudaSetDevice(b->device));
  BatchView &v = b->v;
  float *Fd = nullptr;
  bool f_host = false, uw_host = false;
  if (F && v.ntot > 0) {
    if (is_device_ptr(F)) {
      Fd = F;
    } else {
      if (!b->f_int) {
        int r = alloc(b, &b->f_int, 3 * (int64_t)v.ntot, "F copy");
        if (r) return r;
      }
      Fd = b->f_int;
      f_host = true;
    }
  }
  double *UWd = b->uw_int;
  if (UW && is_device_ptr(UW)) UWd = UW;
  else if (UW) uw_host = true;
  v.q = b->q_cur;
  v.F = Fd;
  v.UW = UWd;
  v.gs = b->gs;
  v.wide = b->force_kernel == 4;
  if (b->use_graph) {
    const bool same = b->exec && b->key[0] == (const void *)v.q && b->key[1] == (const void *)Fd &&
                      b->key[2] == (const void *)UWd && b->key_cfg[0] == b->kfac && b->key_cfg[1] == b->gs &&
                      b->key_cfg[2] == b->force_kernel;
    if (!same) {
      drop_graph(b);
      CKB(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed));
      cudaError_t e = enqueue_step(b, b->cap_stream);
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return cuda_err(b, e != cudaSuccess ? e : e2, "batch graph capture");
      }
      b->graph = g;
      CKB(cudaGraphInstantiate(&b->exec, g, 0));
      b->key[0] = v.q;
      b->key[1] = Fd;
      b->key[2] = UWd;
      b->key_cfg[0] = b->kfac;
      b->key_cfg[1] = b->gs;
      b->key_cfg[2] = b->force_kernel;
    }
    CKB(cudaGraphLaunch(b->exec, b->stream));
  } else {
    cudaError_t e = enqueue_step(b, b->stream);
    if (e != cudaSuccess) return cuda_err(b, e, "batch step");
  }
  if (f_host)
    CKB(cudaMemcpyAsync(F, Fd, sizeof(float) * 3 * (size_t)v.ntot, cudaMemcpyDeviceToHost, b->stream));
  if (uw_host)
    CKB(cudaMemcpyAsync(UW, UWd, sizeof(double) * 10 * (size_t)v.nsys, cudaMemcpyDeviceToHost, b->stream));
  if (f_host || uw_host) return nemd_batch_sync(b, nullptr);
  return NEMD_OK;
}

int nemd_batch_sync(nemd_batch *b, int32_t *status) {
  if (!b) return NEMD_ERR_ARG;
  if (!b->finalized) return set_err(b, NEMD_ERR_ORDER, "batch_sync before finalize");
  CKB(cudaSetDevice(b->device));
  const int S = b->v.nsys;
  k_b_errors<<<(S + 255) / 256, 256, 0, b->stream>>>(b->v.geo, b->err_dev, S, 1);
  CKB(cudaGetLastError());
  CKB(cudaMemcpyAsync(b->h_err, b->err_dev, sizeof(int) * S, cudaMemcpyDeviceToHost, b->stream));
  CKB(cudaStreamSynchronize(b->stream));
  int first = NEMD_OK;
  for (int s = 0; s < S; s++) {
    const char *what;
    const int code = nemd::status_from_bits(b->h_err[s], &what);
    if (status) status[s] = code;
    if (code && !first) {
      first = code;
      set_err(b, code, "system %d: %s (device error bits 0x%x)", s, what, b->h_err[s]);
    }
  }
  return first;
}

int nemd_batch_set_option(nemd_batch *b, int key, int64_t value) {
  if (!b) return NEMD_ERR_ARG;
  switch (key) {
    case NEMD_BATCH_OPT_CELL_FACTOR: {
      if (value < 1 || value > nemd::kBatchMaxFactor)
        return set_err(b, NEMD_ERR_ARG, "batch cell factor %lld (1 or 2)", (long long)value);
      b->kfac = (int)value;
      if (b->finalized) {
        // ordered on the stream: steps already queued keep the factor they were issued with
        for (auto &g : b->grid_host) g.kfac = b->kfac;
        CKB(cudaSetDevice(b->device));
        CKB(cudaMemcpyAsync(b->grid_dev, b->grid_host.data(), sizeof(GridIn) * b->grid_host.size(),
                            cudaMemcpyHostToDevice, b->stream));
      }
      return NEMD_OK;
    }
    case NEMD_BATCH_OPT_TILE:
      if (value != 16 && value != 32) return set_err(b, NEMD_ERR_ARG, "batch tile %lld (16 or 32)", (long long)value);
      b->gs = (int)value;
      return NEMD_OK;
    case NEMD_BATCH_OPT_GRAPH:
      b->use_graph = value ? 1 : 0;
      return NEMD_OK;
    case NEMD_BATCH_OPT_KERNEL:
      if (value != 2 && value != 4) return set_err(b, NEMD_ERR_ARG, "batch force kernel %lld (2 or 4)", (long long)value);
      b->force_kernel = (int)value;
      return NEMD_OK;
    default:
      return set_err(b, NEMD_ERR_ARG, "batch option %d", key);
  }
}

int nemd_batch_get_stats(nemd_batch *b, nemd_batch_stats *out, int64_t *launches) {
  if (!b) return NEMD_ERR_ARG;
  if (!b->finalized) return set_err(b, NEMD_ERR_ORDER, "batch_get_stats before finalize");
  if (launches) *launches = b->launches;
  if (!out) return NEMD_OK;
  CKB(cudaSetDevice(b->device));
  const int S = b->v.nsys;
  std::vector<Geo> g(S);
  std::vector<unsigned long long> pairs(S), cnt(2 * S);
  CKB(cudaMemcpyAsync(g.data(), b->v.geo, sizeof(Geo) * S, cudaMemcpyDeviceToHost, b->stream));
  CKB(cudaMemcpyAsync(pairs.data(), b->v.sys_pairs, sizeof(unsigned long long) * S, cudaMemcpyDeviceToHost,
                      b->stream));
  CKB(cudaMemcpyAsync(cnt.data(), b->v.sys_counters, 2 * sizeof(unsigned long long) * S, cudaMemcpyDeviceToHost,
                      b->stream));
  CKB(cudaStreamSynchronize(b->stream));
  for (int s = 0; s < S; s++) {
    nemd_batch_stats &o = out[s];
    memset(&o, 0, sizeof o);
    o.pairs = (int64_t)pairs[s];
    o.candidates = (int64_t)cnt[2 * s];
    o.band = (int64_t)cnt[2 * s + 1];
    for (int a = 0; a < 3; a++) o.counts[a] = g[s].nc[a];
    o.variant = g[s].variant;
    o.cell_factor = g[s].kfac;
    o.status = nemd::status_from_bits(g[s].sticky | g[s].error, nullptr);
  }
  return NEMD_OK;
}

int nemd_batch_autotune(nemd_batch *b, int reps, nemd_tune_entry *times, int cap, int *ntimes) {
  if (!b) return NEMD_ERR_ARG;
  if (!b->have_state) return set_err(b, NEMD_ERR_ORDER, "batch_autotune before batch_set_state");
  if (reps < 1 || reps > 1000) return set_err(b, NEMD_ERR_ARG, "batch_autotune: reps %d", reps);
  CKB(cudaSetDevice(b->device));
  static const int cand[4][2] = {{1, 32}, {1, 16}, {2, 32}, {2, 16}};
  cudaEvent_t e0, e1;
  CKB(cudaEventCreate(&e0));
  CKB(cudaEventCreate(&e1));
  int best = -1, nt = 0, rc = NEMD_OK;
  double best_ms = 0.0;
  for (int k = 0; k < 4 && !rc; k++) {
    if ((rc = nemd_batch_set_option(b, NEMD_BATCH_OPT_CELL_FACTOR, cand[k][0]))) break;
    if ((rc = nemd_batch_set_option(b, NEMD_BATCH_OPT_TILE, cand[k][1]))) break;
    if ((rc = nemd_batch_compute(b, nullptr, nullptr))) break;
    cudaEventRecord(e0, b->stream);
    for (int q = 0; q < reps && !rc; q++) rc = nemd_batch_compute(b, nullptr, nullptr);
    cudaEventRecord(e1, b->stream);
    if (rc) break;
    if ((rc = nemd_batch_sync(b, nullptr))) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double mean = (double)ms / reps;
    if (times && nt < cap) {
      times[nt].cfg.kernel = b->force_kernel;
      times[nt].cfg.group = cand[k][1];
      times[nt].cfg.cell_factor = cand[k][0];
      times[nt].cfg.pad = 0;
      times[nt].ms = mean;
    }
    nt++;
    if (best < 0 || mean < best_ms) {
      best = k;
      best_ms = mean;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ntimes) *ntimes = nt;
  if (rc) return rc;
  nemd_batch_set_option(b, NEMD_BATCH_OPT_CELL_FACTOR, cand[best][0]);
  nemd_batch_set_option(b, NEMD_BATCH_OPT_TILE, cand[best][1]);
  return NEMD_OK;
}

}  // extern "C"
