// capi.cu -- the C ABI declared in include/nemd.h: context, validation of the
// flow (Sec. 2.2, Eq. kr), buffer management and the launch sequence of one
// force evaluation.  No arithmetic of the method happens here; every step of
// the evaluation is a kernel launched on the context's stream.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "nemd_internal.cuh"

using nemd::Geo;
using nemd::Row;

namespace {

int set_err(nemd_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->msg, sizeof c->msg, fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_err(nemd_ctx *c, cudaError_t e, const char *where) {
  return set_err(c, NEMD_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_err(c, e_, #call); \
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
int grow(nemd_ctx *c, T **p, int64_t count, const char *what) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_err(c, NEMD_ERR_NOMEM, "cudaMalloc of %s (%lld elements) failed", what, (long long)count);
  }
  return NEMD_OK;
}

double det3(const double *a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
}

int rows_stride_bound(int kfac) { return (2 * kfac + 1) * (2 * kfac + 2); }

int ensure_particles(nemd_ctx *c, int64_t n) {
  if (n <= c->cap_n && c->partials) return NEMD_OK;
  int64_t cap = n + n / 8 + 1024;
  int r;
  if ((r = grow(c, &c->relc, cap, "relc"))) return r;
  if ((r = grow(c, &c->rank, cap, "rank"))) return r;
  if ((r = grow(c, &c->perm, cap, "perm"))) return r;
  if ((r = grow(c, &c->pos4, cap, "pos4"))) return r;
  if ((r = grow(c, &c->relr, cap, "relr"))) return r;
  if ((r = grow(c, &c->posr, cap, "posr"))) return r;
  if ((r = grow(c, &c->cell_sorted, cap, "cell_sorted"))) return r;
  if ((r = grow(c, &c->chunks, cap, "chunks"))) return r;
  int64_t nblocks = (cap + 31) / 32 + 2;  // any block size >= 32, plus the fix-up slot
  if ((r = grow(c, &c->partials, nblocks * nemd::kPartials, "partials"))) return r;
  c->cap_partials = nblocks;
  if (c->q_copy) {
    cudaFree(c->q_copy);
    c->q_copy = nullptr;
  }
  if (c->f_dev) {
    cudaFree(c->f_dev);
    c->f_dev = nullptr;
  }
  c->cap_n = cap;
  return NEMD_OK;
}

int ensure_cells(nemd_ctx *c, int64_t cells, int kfac) {
  const int64_t stride = rows_stride_bound(kfac);
  if (cells <= c->cap_cells && stride * cells <= c->cap_rows) return NEMD_OK;
  int64_t cap = cells > c->cap_cells ? cells + cells / 8 + 64 : c->cap_cells;
  int r;
  if ((r = grow(c, &c->count, cap + 1, "count"))) return r;
  if ((r = grow(c, &c->start, cap + 1, "start"))) return r;
  if ((r = grow(c, &c->block_sums, cap / 4096 + 2, "block_sums"))) return r;
  if ((r = grow(c, &c->rowcnt, cap, "rowcnt"))) return r;
  if ((r = grow(c, &c->rows, cap * stride, "rows"))) return r;
  if ((r = grow(c, &c->chunk_cnt, cap + 1, "chunk counts"))) return r;
  if ((r = grow(c, &c->chunk_off, cap + 1, "chunk offsets"))) return r;
  c->cap_cells = cap;
  c->cap_rows = cap * stride;
  return NEMD_OK;
}

// Stream, events and double buffers of the asynchronous host path.
int ensure_async(nemd_ctx *c) {
  if (!c->copy_stream) {
    CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->copy_back, cudaStreamNonBlocking));
    for (int k = 0; k < 2; k++) {
      CK(cudaEventCreateWithFlags(&c->ev_q[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&c->ev_done[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&c->ev_out[k], cudaEventDisableTiming));
      c->done_valid[k] = c->out_valid[k] = false;
    }
  }
  if (c->acap < c->cap_n || !c->aq[0]) {
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaStreamSynchronize(c->copy_stream));
    CK(cudaStreamSynchronize(c->copy_back));
    for (int k = 0; k < 2; k++) {
      int r;
      if ((r = grow(c, &c->aq[k], 3 * c->cap_n, "async q"))) return r;
      if ((r = grow(c, &c->af[k], 3 * c->cap_n, "async F"))) return r;
      if ((r = grow(c, &c->auw[k], 10, "async UW"))) return r;
    }
    c->acap = c->cap_n;
  }
  return NEMD_OK;
}

int take_device_error(nemd_ctx *c) {
  int bits = *c->h_error;
  *c->h_error = 0;
  if (!bits) return NEMD_OK;
  const char *what;
  const int code = nemd::status_from_bits(bits, &what);
  return set_err(c, code, "%s (device error bits 0x%x)", what, bits);
}

__global__ void k_fetch_error(Geo *g, int *out, int clear) {
  int v = g->sticky | g->error;
  *out = v;
  if (clear) {
    g->sticky = 0;
    g->error = 0;
  }
}

}  // namespace

namespace nemd {

int status_from_bits(int bits, const char **what) {
  const char *w = "device error";
  int code = bits ? NEMD_ERR_CUDA : NEMD_OK;
  if (!bits) {
    w = "ok";
  } else if (bits & ERRB_NONFINITE) {
    code = NEMD_ERR_NONFINITE;
    w = "non-finite particle coordinate";
  } else if (bits & ERRB_BOX) {
    code = NEMD_ERR_BOX_TOO_SMALL;
    w = "box too small for the cut-off: a cell count is 0";
  } else if (bits & ERRB_CAPACITY) {
    code = NEMD_ERR_CAPACITY;
    w = "device table capacity exceeded";
  } else if (bits & ERRB_TIMEOUT) {
    code = NEMD_ERR_TIMEOUT;
    w = "bounded device wait ran out";
  }
  if (what) *what = w;
  return code;
}

}  // namespace nemd

extern "C" {

int nemd_create(nemd_ctx **out, int device, void *stream) {
  if (!out) return NEMD_ERR_ARG;
  *out = nullptr;
  nemd_ctx *c = (nemd_ctx *)calloc(1, sizeof(nemd_ctx));
  if (!c) return NEMD_ERR_NOMEM;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  c->int_graph = 1;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    free(c);
    return NEMD_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc((void **)&c->geo, sizeof(Geo)) != cudaSuccess ||
      cudaMalloc((void **)&c->uw_out, 10 * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void **)&c->counters, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc((void **)&c->pair_count, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc((void **)&c->nchunks, sizeof(int)) != cudaSuccess ||
      cudaMalloc((void **)&c->nrecheck, sizeof(int)) != cudaSuccess ||
      cudaMalloc((void **)&c->recheck, sizeof(int4) * nemd::kRecheckCap) != cudaSuccess ||
      cudaMallocHost((void **)&c->h_error, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    nemd_destroy(c);
    return NEMD_ERR_NOMEM;
  }
  cudaMemset(c->geo, 0, sizeof(Geo));
  cudaMemset(c->counters, 0, 4 * sizeof(unsigned long long));
  *c->h_error = 0;
  c->pot_kind = NEMD_LJ;
  c->eps = 1.0;
  c->sigma = 1.0;
  c->shift = 1;
  c->have_pot = true;
  c->kfac = 1;
  c->kernel = 0;
  c->block = 128;
  c->group = 16;
  snprintf(c->msg, sizeof c->msg, "ok");
  *out = c;
  return NEMD_OK;
}

int nemd_destroy(nemd_ctx *c) {
  if (!c) return NEMD_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->model) cudaFree(c->model);
  void *ptrs[] = {c->geo,  c->q_copy, c->relc,     c->relr, c->posr, c->rank,     c->count,    c->start, c->chunks, c->nchunks, c->recheck, c->nrecheck,
                  c->block_sums, c->perm, c->pos4, c->cell_sorted, c->rows, c->rowcnt,
                  c->partials, c->uw_out, c->f_dev, c->pair_buf, c->pair_count, c->counters,
                  c->chunk_cnt, c->chunk_off, c->int_state, c->int_part, c->f_int};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  void *vptrs[] = {c->vl_cnt, c->vl_ent, c->vl_slot, c->vl_sb, c->vl_idx, c->vl_pos, c->vl_res, c->vl_geo, c->vl_disp,
                   c->fix_f, c->fix_uw};
  for (void *p : vptrs)
    if (p) cudaFree(p);
  if (c->h_vl) cudaFreeHost(c->h_vl);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamSynchronize(c->copy_back);
    for (int k = 0; k < 2; k++) {
      cudaEventDestroy(c->ev_q[k]);
      cudaEventDestroy(c->ev_done[k]);
      cudaEventDestroy(c->ev_out[k]);
      if (c->aq[k]) cudaFree(c->aq[k]);
      if (c->af[k]) cudaFree(c->af[k]);
      if (c->auw[k]) cudaFree(c->auw[k]);
    }
    cudaStreamDestroy(c->copy_stream);
    cudaStreamDestroy(c->copy_back);
  }
  if (c->h_error) cudaFreeHost(c->h_error);
  if (c->ev) {
    for (int k = 0; k < 2 * c->ev_cap; k++)
      if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    free(c->ev);
  }
  cudaGetLastError();
  free(c);
  return NEMD_OK;
}

const char *nemd_last_error(const nemd_ctx *c) { return c ? c->msg : "null context"; }

int nemd_set_flow(nemd_ctx *c, const double A[9], const double L0[9], const int64_t M[9], double T) {
  if (!c || !A || !L0 || !M) return set_err(c, NEMD_ERR_ARG, "set_flow: null argument");
  for (int k = 0; k < 9; k++)
    if (!isfinite(A[k]) || !isfinite(L0[k])) return set_err(c, NEMD_ERR_ARG, "set_flow: non-finite A or L0");
  // M in SL(3,Z): integer entries (int64 by type) and det M = 1 in exact integer arithmetic
  const int64_t *m = M;
  int64_t dm = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
               m[2] * (m[3] * m[7] - m[4] * m[6]);
  if (dm != 1) return set_err(c, NEMD_ERR_NOT_SL3Z, "set_flow: det M = %lld, not 1", (long long)dm);
  double amax = 0.0;
  for (int k = 0; k < 9; k++) amax = fmax(amax, fabs(A[k]));
  if (fabs(A[0] + A[4] + A[8]) > 1e-12 * amax)
    return set_err(c, NEMD_ERR_TRACE, "set_flow: tr A = %g is not 0 (flow must be incompressible)", A[0] + A[4] + A[8]);
  double dl = det3(L0);
  if (!(fabs(dl) > 0.0)) return set_err(c, NEMD_ERR_ARG, "set_flow: L0 is singular");
  if (amax == 0.0) {
    for (int k = 0; k < 9; k++)
      if (M[k] != ((k % 4 == 0) ? 1 : 0)) return set_err(c, NEMD_ERR_NOT_KR, "set_flow: A = 0 requires M = I");
  } else if (!(T > 0.0)) {
    return set_err(c, NEMD_ERR_ARG, "set_flow: the period T must be > 0");
  }
  memcpy(c->A, A, sizeof c->A);
  memcpy(c->L0, L0, sizeof c->L0);
  memcpy(c->M, M, sizeof c->M);
  c->T = (amax == 0.0 && !(T > 0.0)) ? 1.0 : T;
  CK(cudaSetDevice(c->device));
  if (amax != 0.0) {
    // Kraynik-Reinelt condition exp(A T) L0 = L0 M (Eq. kr), on the device
    cudaError_t e = nemd::launch_lattice(c, 1, c->T);
    if (e != cudaSuccess) return cuda_err(c, e, "set_flow lattice");
    double L[9];
    CK(cudaMemcpyAsync(L, c->geo->L, sizeof L, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double lmax = 0.0, res = 0.0;
    for (int k = 0; k < 9; k++) lmax = fmax(lmax, fabs(L0[k]));
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        double lm = L0[3 * i] * (double)M[j] + L0[3 * i + 1] * (double)M[3 + j] + L0[3 * i + 2] * (double)M[6 + j];
        res = fmax(res, fabs(L[3 * i + j] - lm));
      }
    if (!(res <= 1e-9 * lmax)) {
      c->have_flow = false;
      return set_err(c, NEMD_ERR_NOT_KR, "set_flow: |exp(T A) L0 - L0 M| = %g > 1e-9 |L0|", res);
    }
  }
  c->have_flow = true;
  c->have_state = false;
  c->have_cells = false;
  return NEMD_OK;
}

int nemd_set_potential(nemd_ctx *c, int kind, double eps, double sigma, int shift) {
  if (!c) return NEMD_ERR_ARG;
  if (kind != NEMD_LJ && kind != NEMD_WCA) return set_err(c, NEMD_ERR_ARG, "set_potential: unknown kind %d", kind);
  if (!(eps > 0.0) || !(sigma > 0.0)) return set_err(c, NEMD_ERR_ARG, "set_potential: eps and sigma must be > 0");
  if (kind == NEMD_WCA && !shift) return set_err(c, NEMD_ERR_ARG, "set_potential: WCA is shifted by definition");
  c->pot_kind = kind;
  c->eps = eps;
  c->sigma = sigma;
  c->shift = shift ? 1 : 0;
  c->have_pot = true;
  return NEMD_OK;
}

int nemd_set_state(nemd_ctx *c, const double *q, int64_t n, double t) {
  if (!c) return NEMD_ERR_ARG;
  if (!c->have_flow) return set_err(c, NEMD_ERR_ORDER, "set_state before set_flow");
  if (n < 0 || n > (int64_t)0x7fffffff / 4) return set_err(c, NEMD_ERR_ARG, "set_state: bad N = %lld", (long long)n);
  if (n > 0 && !q) return set_err(c, NEMD_ERR_ARG, "set_state: null q");
  if (!isfinite(t)) return set_err(c, NEMD_ERR_ARG, "set_state: non-finite t");
  CK(cudaSetDevice(c->device));
  int r = ensure_particles(c, n);
  if (r) return r;
  c->n = n;
  c->t = t;
  if (c->async_host) {
    if ((r = ensure_async(c))) return r;
    c->aslot ^= 1;
  }
  if (n > 0) {
    if (is_device_ptr(q)) {
      c->q_dev = q;
    } else if (c->async_host) {
      // copy on the copy stream once the evaluation that last read this buffer is done
      const int k = c->aslot;
      if (c->done_valid[k]) CK(cudaStreamWaitEvent(c->copy_stream, c->ev_done[k], 0));
      CK(cudaMemcpyAsync(c->aq[k], q, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, c->copy_stream));
      CK(cudaEventRecord(c->ev_q[k], c->copy_stream));
      CK(cudaStreamWaitEvent(c->stream, c->ev_q[k], 0));
      c->q_dev = c->aq[k];
    } else {
      if (!c->q_copy) {
        if ((r = grow(c, &c->q_copy, 3 * c->cap_n, "q_copy"))) return r;
      }
      CK(cudaMemcpyAsync(c->q_copy, q, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, c->stream));
      c->q_dev = c->q_copy;
    }
  } else {
    c->q_dev = nullptr;
  }
  cudaError_t e = nemd::launch_lattice(c, 0, 0.0);
  if (e != cudaSuccess) return cuda_err(c, e, "set_state lattice");
  c->have_state = true;
  c->have_cells = false;
  return NEMD_OK;
}

int nemd_build_cells(nemd_ctx *c, int variant, double rc) {
  if (!c) return NEMD_ERR_ARG;
  if (!c->have_state) return set_err(c, NEMD_ERR_ORDER, "build_cells before set_state");
  if (variant < NEMD_DS || variant > NEMD_AUTO_LEARNED) return set_err(c, NEMD_ERR_ARG, "build_cells: variant %d", variant);
  if (!(rc > 0.0) || !isfinite(rc)) return set_err(c, NEMD_ERR_ARG, "build_cells: rc must be > 0");
  if (c->pot_kind == NEMD_WCA && fabs(rc - pow(2.0, 1.0 / 6.0) * c->sigma) > 1e-12 * c->sigma)
    return set_err(c, NEMD_ERR_ARG, "build_cells: WCA needs rc = 2^(1/6) sigma");
  CK(cudaSetDevice(c->device));
  if (c->autotuned) nemd::tune_apply(c, rc);
  // the learned selector may pick cell factor 2 on the device: size for it
  const bool learned = variant == NEMD_AUTO_LEARNED && c->have_model;
  const int kalloc = learned && c->kfac < 2 ? 2 : c->kfac;
  // bound on the number of cells: c1 c2 c3 <= k^3 h1 h2 h3 / rc^3 <= k^3 V / rc^3
  const double V = fabs(det3(c->L0));
  const double k3 = (double)kalloc * kalloc * kalloc;
  double bound = k3 * V / (rc * rc * rc) * (1.0 + 1e-9) + 1.0;
  if (bound > 2.0e9) return set_err(c, NEMD_ERR_ARG, "build_cells: %g cells is too many", bound);
  int r = ensure_cells(c, (int64_t)bound, kalloc);
  if (r) return r;
  c->rc = rc;
  c->variant_req = variant;
  c->kfac_alloc = kalloc;
  cudaError_t e = cudaSuccess;
  if (variant == NEMD_AUTO_LEARNED) {
    e = nemd::launch_learned_choice(c, rc);
    if (e != cudaSuccess) return cuda_err(c, e, "build_cells learned choice");
  }
  e = nemd::launch_grid(c);
  if (e != cudaSuccess) return cuda_err(c, e, "build_cells grid");
  e = nemd::launch_stencil(c);
  if (e != cudaSuccess) return cuda_err(c, e, "build_cells stencil");
  e = nemd::launch_bin(c);
  if (e != cudaSuccess) return cuda_err(c, e, "build_cells bin");
  c->have_cells = true;
  return NEMD_OK;
}

// Asynchronous host outputs: the evaluation writes the current buffer pair,
// which the copy stream then moves to the host; nothing waits on the host.
static int compute_forces_async(nemd_ctx *c, float *F, double *U, double *W) {
  const int k = c->aslot;
  const bool fd = F && is_device_ptr(F), ud = U && is_device_ptr(U), wd = W && is_device_ptr(W);
  // the buffers of this pair are free once their previous copies to the host are done
  if (c->out_valid[k]) CK(cudaStreamWaitEvent(c->stream, c->ev_out[k], 0));
  float *Fd = (F && c->n > 0) ? (fd ? F : c->af[k]) : nullptr;
  cudaError_t e = nemd::launch_forces(c, Fd, c->auw[k]);
  if (e != cudaSuccess) return cuda_err(c, e, "compute_forces");
  if (ud) CK(cudaMemcpyAsync(U, c->auw[k], sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  if (wd) CK(cudaMemcpyAsync(W, c->auw[k] + 1, 9 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaEventRecord(c->ev_done[k], c->stream));
  c->done_valid[k] = true;
  CK(cudaStreamWaitEvent(c->copy_back, c->ev_done[k], 0));
  if (F && c->n > 0 && !fd)
    CK(cudaMemcpyAsync(F, c->af[k], sizeof(float) * 3 * (size_t)c->n, cudaMemcpyDeviceToHost, c->copy_back));
  if (U && !ud) CK(cudaMemcpyAsync(U, c->auw[k], sizeof(double), cudaMemcpyDeviceToHost, c->copy_back));
  if (W && !wd) CK(cudaMemcpyAsync(W, c->auw[k] + 1, 9 * sizeof(double), cudaMemcpyDeviceToHost, c->copy_back));
  CK(cudaEventRecord(c->ev_out[k], c->copy_back));
  c->out_valid[k] = true;
  return NEMD_OK;
}

int nemd_compute_forces(nemd_ctx *c, float *F, double *U, double *W) {
  if (!c) return NEMD_ERR_ARG;
  if (!c->have_cells) return set_err(c, NEMD_ERR_ORDER, "compute_forces before build_cells");
  CK(cudaSetDevice(c->device));
  if (c->async_host) return compute_forces_async(c, F, U, W);
  float *Fd = nullptr;
  bool host_out = false;
  if (F && c->n > 0) {
    if (is_device_ptr(F)) {
      Fd = F;
    } else {
      if (!c->f_dev) {
        int r = grow(c, &c->f_dev, 3 * c->cap_n, "f_dev");
        if (r) return r;
      }
      Fd = c->f_dev;
      host_out = true;
    }
  }
  cudaError_t e = nemd::launch_forces(c, Fd, c->uw_out);
  if (e != cudaSuccess) return cuda_err(c, e, "compute_forces");
  if (F && host_out)
    CK(cudaMemcpyAsync(F, Fd, sizeof(float) * 3 * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
  if (U) {
    bool dev = is_device_ptr(U);
    host_out |= !dev;
    CK(cudaMemcpyAsync(U, c->uw_out, sizeof(double), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream));
  }
  if (W) {
    bool dev = is_device_ptr(W);
    host_out |= !dev;
    CK(cudaMemcpyAsync(W, c->uw_out + 1, 9 * sizeof(double), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream));
  }
  if (host_out) return nemd_sync(c);
  return NEMD_OK;
}

int nemd_sync(nemd_ctx *c) {
  if (!c) return NEMD_ERR_ARG;
  CK(cudaSetDevice(c->device));
  k_fetch_error<<<1, 1, 0, c->stream>>>(c->geo, c->h_error, 1);
  c->launches += 1;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  if (c->copy_stream) {
    CK(cudaStreamSynchronize(c->copy_stream));
    CK(cudaStreamSynchronize(c->copy_back));
  }
  return take_device_error(c);
}

int nemd_set_option(nemd_ctx *c, int key, int64_t value) {
  if (!c) return NEMD_ERR_ARG;
  switch (key) {
    case NEMD_OPT_PRECISE:
      c->precise = value ? 1 : 0;
      return NEMD_OK;
    case NEMD_OPT_RECORD_PAIRS: {
      if (value < 0) return set_err(c, NEMD_ERR_ARG, "record capacity < 0");
      CK(cudaSetDevice(c->device));
      CK(cudaStreamSynchronize(c->stream));
      if (c->pair_buf) cudaFree(c->pair_buf);
      c->pair_buf = nullptr;
      c->record_cap = 0;
      if (value > 0) {
        int r = grow(c, &c->pair_buf, 5 * value, "pair record");
        if (r) return r;
        c->record_cap = value;
      }
      return NEMD_OK;
    }
    case NEMD_OPT_ASYNC_HOST:
      CK(cudaSetDevice(c->device));
      CK(cudaStreamSynchronize(c->stream));
      if (c->copy_stream) {
        CK(cudaStreamSynchronize(c->copy_stream));
        CK(cudaStreamSynchronize(c->copy_back));
      }
      c->async_host = value ? 1 : 0;
      return NEMD_OK;
    case NEMD_OPT_INT_GRAPH:
      if (value != 0 && value != 1) return set_err(c, NEMD_ERR_ARG, "int_graph %lld (0 or 1)", (long long)value);
      c->int_graph = (int)value;
      return NEMD_OK;
    case NEMD_OPT_REMAP:
      if (value != 0 && value != 1) return set_err(c, NEMD_ERR_ARG, "remap %lld (0 or 1)", (long long)value);
      c->remap_centered = (int)value;
      return NEMD_OK;
    case NEMD_OPT_KERNEL:
      if (value < 0 || value > 4) return set_err(c, NEMD_ERR_ARG, "kernel %lld", (long long)value);
      c->kernel = (int)value;
      return NEMD_OK;
    case NEMD_OPT_CELL_FACTOR:
      if (value < 1 || value > nemd::kMaxFactor) return set_err(c, NEMD_ERR_ARG, "cell factor %lld", (long long)value);
      c->kfac = (int)value;
      return NEMD_OK;
    case NEMD_OPT_GROUP:
      if (value != 4 && value != 8 && value != 16 && value != 32)
        return set_err(c, NEMD_ERR_ARG, "group size %lld (4, 8, 16 or 32)", (long long)value);
      c->group = (int)value;
      return NEMD_OK;
    case NEMD_OPT_AUTOTUNED:
      c->autotuned = value ? 1 : 0;
      return NEMD_OK;
    case NEMD_OPT_TIMING:
      CK(cudaSetDevice(c->device));
      if (value && !c->ev) {
        c->ev_cap = 4096;
        c->ev = (cudaEvent_t *)calloc(2 * (size_t)c->ev_cap, sizeof(cudaEvent_t));
        if (!c->ev) return set_err(c, NEMD_ERR_NOMEM, "timing events");
        for (int k = 0; k < 2 * c->ev_cap; k++) CK(cudaEventCreate(&c->ev[k]));
      }
      c->timing = value ? 1 : 0;
      c->ev_n = 0;
      return NEMD_OK;
    case NEMD_OPT_BLOCK:
      if (value < 32 || value > 1024 || value % 32) return set_err(c, NEMD_ERR_ARG, "block %lld", (long long)value);
      c->block = (int)value;
      return NEMD_OK;
    default:
      return set_err(c, NEMD_ERR_UNSUPPORTED, "unknown option %d", key);
  }
}

int nemd_get_lattice(nemd_ctx *c, double *out) {
  if (!c || !out) return NEMD_ERR_ARG;
  CK(cudaSetDevice(c->device));
  Geo g;
  CK(cudaMemcpyAsync(&g, c->geo, sizeof g, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  memcpy(out, g.L, 9 * sizeof(double));
  memcpy(out + 9, g.Linv, 9 * sizeof(double));
  out[18] = g.V;
  memcpy(out + 19, g.h, 3 * sizeof(double));
  memcpy(out + 22, g.Q, 9 * sizeof(double));
  memcpy(out + 31, g.R, 9 * sizeof(double));
  out[40] = g.tau;
  out[41] = g.band;
  for (int a = 0; a < 3; a++) out[42 + a] = g.nc[a];
  out[45] = g.ncells;
  out[46] = g.variant;
  out[47] = g.maxrows;
  return NEMD_OK;
}

int nemd_get_stats(nemd_ctx *c, nemd_stats *s) {
  if (!c || !s) return NEMD_ERR_ARG;
  CK(cudaSetDevice(c->device));
  Geo g;
  unsigned long long cnt[4];
  CK(cudaMemcpyAsync(&g, c->geo, sizeof g, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(cnt, c->counters, sizeof cnt, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  memset(s, 0, sizeof *s);
  s->n = c->n;
  s->pairs = (int64_t)cnt[0];
  s->candidates = (int64_t)cnt[1];
  s->rechecks = (int64_t)cnt[2];
  s->ncells = g.ncells;
  for (int a = 0; a < 3; a++) s->counts[a] = g.nc[a];
  s->variant = g.variant;
  s->cell_factor = g.kfac;
  s->max_rows = g.maxrows;
  s->tau = g.tau;
  s->band = g.band;
  s->launches = c->launches;
  // stencil size: sum over home classes of cells per neighbourhood times l1
  if (g.ncells > 0) {
    int ncls = g.nc[1] * g.nc[2];
    int *rc = (int *)malloc(sizeof(int) * (size_t)ncls);
    Row *rw = (Row *)malloc(sizeof(Row) * (size_t)ncls * g.maxrows);
    if (rc && rw) {
      cudaMemcpy(rc, c->rowcnt, sizeof(int) * (size_t)ncls, cudaMemcpyDeviceToHost);
      cudaMemcpy(rw, c->rows, sizeof(Row) * (size_t)ncls * g.maxrows, cudaMemcpyDeviceToHost);
      int64_t tot = 0;
      for (int k = 0; k < ncls; k++)
        for (int r = 0; r < rc[k]; r++) tot += rw[(size_t)k * g.maxrows + r].cnt;
      s->stencil_cells = tot * g.nc[0];
    }
    free(rc);
    free(rw);
  }
  return NEMD_OK;
}

int nemd_get_kernel_time(nemd_ctx *c, double *ms_total, int64_t *nlaunch) {
  if (!c || !ms_total || !nlaunch) return NEMD_ERR_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  for (int k = 0; k < c->ev_n; k++) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]));
    tot += ms;
  }
  *ms_total = tot;
  *nlaunch = c->ev_n;
  c->ev_n = 0;
  return NEMD_OK;
}

int nemd_get_pairs(nemd_ctx *c, int32_t *out, int64_t cap, int64_t *count) {
  if (!c || !count) return NEMD_ERR_ARG;
  if (c->record_cap <= 0) return set_err(c, NEMD_ERR_ORDER, "get_pairs: recording is off");
  CK(cudaSetDevice(c->device));
  unsigned long long n = 0;
  CK(cudaMemcpyAsync(&n, c->pair_count, sizeof n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *count = (int64_t)n;
  int64_t avail = (int64_t)n < c->record_cap ? (int64_t)n : c->record_cap;
  int64_t ncopy = avail < cap ? avail : cap;
  if (out && ncopy > 0) CK(cudaMemcpy(out, c->pair_buf, sizeof(int32_t) * 5 * (size_t)ncopy, cudaMemcpyDeviceToHost));
  if ((int64_t)n > c->record_cap || (int64_t)n > cap)
    return set_err(c, NEMD_ERR_CAPACITY, "get_pairs: %lld pairs, record holds %lld, output %lld", (long long)n,
                   (long long)c->record_cap, (long long)cap);
  return NEMD_OK;
}

}  // extern "C"
