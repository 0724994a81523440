// autotune.cu -- the library's autotuner: picks the force kernel, the lanes per
// group and the cell-size factor for a shape class of systems by timing them.
// The paper has no counterpart (its cell size is fixed at the cut-off,
// Sec. 4); every candidate computes the same pair set and forces, so the
// choice changes only the time.
//
// Shape class: (round(log2 N), round(4 log2(rho rc^3))) -- quantities the host
// knows without reading the device, so a cached choice can be applied when a
// step's cells are built.  Per class and candidate the cache keeps the sum and
// count of measured times; the choice is the smallest mean.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "nemd_internal.cuh"

namespace {

struct Candidate {
  int kernel, group, kfac;
};

// plain kernel; warp kernel at k = 1, 2; grouped kernel with 4, 8, 16 lanes at
// k = 1, 2; warp kernel with half neighbourhoods at k = 1, 2; row kernel at k = 1, 2
const Candidate kCandidates[] = {{0, 16, 1}, {2, 32, 1}, {2, 32, 2}, {1, 4, 1},  {1, 8, 1},  {1, 16, 1}, {1, 4, 2},
                                 {1, 8, 2},  {1, 16, 2}, {3, 32, 1}, {3, 32, 2}, {4, 32, 1}, {4, 32, 2}};
constexpr int kNumCandidates = sizeof(kCandidates) / sizeof(kCandidates[0]);
static_assert(kNumCandidates == nemd::kTuneCandidates, "cache layout");

uint64_t fnv1a(const unsigned char *p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; i++) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

namespace nemd {

void tune_class_key(const nemd_ctx *c, double rc, int32_t key[2]) {
  const double V = fabs(c->L0[0] * (c->L0[4] * c->L0[8] - c->L0[5] * c->L0[7]) -
                        c->L0[1] * (c->L0[3] * c->L0[8] - c->L0[5] * c->L0[6]) +
                        c->L0[2] * (c->L0[3] * c->L0[7] - c->L0[4] * c->L0[6]));
  const double n = c->n > 0 ? (double)c->n : 1.0;
  const double nrc = n / V * rc * rc * rc;
  key[0] = (int32_t)lrint(log2(n));
  key[1] = (int32_t)lrint(4.0 * log2(nrc > 1e-30 ? nrc : 1e-30));
}

TuneEntry *tune_find(nemd_ctx *c, const int32_t key[2], bool create) {
  for (int k = 0; k < c->ntune; k++)
    if (c->tune[k].key[0] == key[0] && c->tune[k].key[1] == key[1]) return &c->tune[k];
  if (!create || c->ntune >= kMaxTuneClasses) return nullptr;
  TuneEntry *e = &c->tune[c->ntune++];
  memset(e, 0, sizeof *e);
  e->key[0] = key[0];
  e->key[1] = key[1];
  return e;
}

// Apply the cached choice of the current class, if any (nemd_build_cells).
void tune_apply(nemd_ctx *c, double rc) {
  int32_t key[2];
  tune_class_key(c, rc, key);
  const TuneEntry *e = tune_find(c, key, false);
  if (!e) return;
  int best = -1;
  double bm = 0.0;
  for (int k = 0; k < kNumCandidates; k++) {
    if (e->count[k] <= 0) continue;
    const double m = e->sum_ms[k] / (double)e->count[k];
    if (best < 0 || m < bm) {
      best = k;
      bm = m;
    }
  }
  if (best < 0) return;
  c->kernel = kCandidates[best].kernel;
  c->group = kCandidates[best].group;
  c->kfac = kCandidates[best].kfac;
}

}  // namespace nemd

extern "C" {

int nemd_autotune(nemd_ctx *c, int variant, double rc, int reps, nemd_tune_config *best, nemd_tune_entry *times,
                  int cap, int *ntimes) {
  if (!c) return NEMD_ERR_ARG;
  if (!c->have_state) return NEMD_ERR_ORDER;
  if (reps < 1 || reps > 1000) return NEMD_ERR_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return NEMD_ERR_CUDA;
  if (!c->f_dev && c->n > 0) {
    if (cudaMalloc((void **)&c->f_dev, sizeof(float) * 3 * (size_t)c->cap_n) != cudaSuccess) return NEMD_ERR_NOMEM;
  }
  const int saved_timing = c->timing;
  c->timing = 0;
  int32_t key[2];
  nemd::tune_class_key(c, rc, key);
  nemd::TuneEntry *entry = nemd::tune_find(c, key, true);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return NEMD_ERR_CUDA;
  const int keep_autotuned = c->autotuned;
  c->autotuned = 0;
  int rc_status = NEMD_OK;
  int nt = 0;
  double best_ms = 0.0;
  int best_k = -1;
  for (int k = 0; k < kNumCandidates && rc_status == NEMD_OK; k++) {
    c->kernel = kCandidates[k].kernel;
    c->group = kCandidates[k].group;
    c->kfac = kCandidates[k].kfac;
    // one untimed evaluation (allocations, first-touch), then reps timed ones
    rc_status = nemd_build_cells(c, variant, rc);
    if (!rc_status) rc_status = nemd_compute_forces(c, c->f_dev, nullptr, nullptr);
    if (rc_status) break;
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && !rc_status; r++) {
      rc_status = nemd_build_cells(c, variant, rc);
      if (!rc_status) rc_status = nemd_compute_forces(c, c->f_dev, nullptr, nullptr);
    }
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc_status = NEMD_ERR_CUDA;
    if (rc_status) break;
    rc_status = nemd_sync(c);
    if (rc_status) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double mean = (double)ms / reps;
    if (entry) {
      entry->sum_ms[k] += mean;
      entry->count[k] += 1;
    }
    if (times && nt < cap) {
      times[nt].cfg.kernel = kCandidates[k].kernel;
      times[nt].cfg.group = kCandidates[k].group;
      times[nt].cfg.cell_factor = kCandidates[k].kfac;
      times[nt].cfg.pad = 0;
      times[nt].ms = mean;
    }
    nt++;
    if (best_k < 0 || mean < best_ms) {
      best_k = k;
      best_ms = mean;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timing = saved_timing;
  c->autotuned = keep_autotuned;
  if (ntimes) *ntimes = nt;
  if (rc_status) return rc_status;
  // apply the class's best mean (over every call so far) and leave the cells built with it
  nemd::tune_apply(c, rc);
  if (best) {
    best->kernel = c->kernel;
    best->group = c->group;
    best->cell_factor = c->kfac;
    best->pad = 0;
  }
  return nemd_build_cells(c, variant, rc);
}

// File: "NEMDTUNE" | u32 version | u32 count | count x {i32 key[2], f64 sum_ms[K], i64 n[K]} |
// u64 FNV-1a of everything before it.
int nemd_tune_save(nemd_ctx *c, const char *path) {
  if (!c || !path) return NEMD_ERR_ARG;
  const uint32_t version = 2, count = (uint32_t)c->ntune, ncand = kNumCandidates;
  size_t n = 8 + 12 + (size_t)count * sizeof(nemd::TuneEntry);
  unsigned char *buf = (unsigned char *)malloc(n + 8);
  if (!buf) return NEMD_ERR_NOMEM;
  memcpy(buf, "NEMDTUNE", 8);
  memcpy(buf + 8, &version, 4);
  memcpy(buf + 12, &count, 4);
  memcpy(buf + 16, &ncand, 4);
  memcpy(buf + 20, c->tune, (size_t)count * sizeof(nemd::TuneEntry));
  const uint64_t h = fnv1a(buf, n);
  memcpy(buf + n, &h, 8);
  FILE *f = fopen(path, "wb");
  if (!f) {
    free(buf);
    return NEMD_ERR_ARG;
  }
  const size_t w = fwrite(buf, 1, n + 8, f);
  fclose(f);
  free(buf);
  return w == n + 8 ? NEMD_OK : NEMD_ERR_ARG;
}

int nemd_tune_load(nemd_ctx *c, const char *path) {
  if (!c || !path) return NEMD_ERR_ARG;
  FILE *f = fopen(path, "rb");
  if (!f) return NEMD_ERR_ARG;
  unsigned char head[20];
  if (fread(head, 1, 20, f) != 20 || memcmp(head, "NEMDTUNE", 8) != 0) {
    fclose(f);
    return NEMD_ERR_ARG;
  }
  uint32_t version, count, ncand;
  memcpy(&version, head + 8, 4);
  memcpy(&count, head + 12, 4);
  memcpy(&ncand, head + 16, 4);
  if (version != 2 || ncand != (uint32_t)kNumCandidates || count > (uint32_t)nemd::kMaxTuneClasses) {
    fclose(f);
    return NEMD_ERR_ARG;
  }
  const size_t n = 20 + (size_t)count * sizeof(nemd::TuneEntry);
  unsigned char *buf = (unsigned char *)malloc(n + 8);
  if (!buf) {
    fclose(f);
    return NEMD_ERR_NOMEM;
  }
  memcpy(buf, head, 20);
  const size_t got = fread(buf + 20, 1, n + 8 - 20, f);
  fclose(f);
  uint64_t h = 0;
  if (got == n + 8 - 20) memcpy(&h, buf + n, 8);
  if (got != n + 8 - 20 || h != fnv1a(buf, n)) {
    free(buf);
    return NEMD_ERR_ARG;
  }
  memcpy(c->tune, buf + 20, (size_t)count * sizeof(nemd::TuneEntry));
  c->ntune = (int)count;
  free(buf);
  return NEMD_OK;
}

}  // extern "C"
