// noalloc.cu -- nemd_forces_noalloc: the whole force evaluation with no memory
// allocation at all, for callers that cannot call cudaMalloc (for example a
// host loop that must never allocate after start-up, or a plug-in that has no
// access to the CUDA allocator of the process that hosts it).
//
// All scratch lives in one file-scope device array of fixed size, carved into
// the same buffers the context path uses; the evaluation then runs the same
// kernels through the same launch wrappers as nemd_set_state /
// nemd_build_cells / nemd_compute_forces.  The array is created when the
// library is loaded and every GPU that loads the library holds it until the
// process exits.
//
// In host code the name of a __device__ array is only a host-side stand-in, not
// a device address; the device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <math.h>
#include <mutex>
#include <string.h>

#include "nemd_internal.cuh"

namespace {

constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

constexpr int64_t kMaxN = NEMD_NOALLOC_MAX_N;
constexpr int64_t kMaxCells = NEMD_NOALLOC_MAX_CELLS;
constexpr int64_t kRowStride = 12;  // (2k + 1)(2k + 2) rows per class at cell factor k = 1
constexpr int64_t kMaxBlocks = (kMaxN + 127) / 128 + 1;  // force blocks + the fix-up slot

// byte offsets of the buffers inside the array
constexpr size_t kOffGeo = 0;
constexpr size_t kOffRelc = align_up(kOffGeo + sizeof(nemd::Geo));
constexpr size_t kOffRelr = align_up(kOffRelc + 16 * kMaxN);
constexpr size_t kOffPos4 = align_up(kOffRelr + 16 * kMaxN);
constexpr size_t kOffPosr = align_up(kOffPos4 + 16 * kMaxN);
constexpr size_t kOffRank = align_up(kOffPosr + 16 * kMaxN);
constexpr size_t kOffPerm = align_up(kOffRank + 4 * kMaxN);
constexpr size_t kOffCellSorted = align_up(kOffPerm + 4 * kMaxN);
constexpr size_t kOffCount = align_up(kOffCellSorted + 4 * kMaxN);
constexpr size_t kOffStart = align_up(kOffCount + 4 * (kMaxCells + 1));
constexpr size_t kOffBlockSums = align_up(kOffStart + 4 * (kMaxCells + 1));
constexpr size_t kOffRowcnt = align_up(kOffBlockSums + 4 * (kMaxCells / 4096 + 2));
constexpr size_t kOffRows = align_up(kOffRowcnt + 4 * kMaxCells);
constexpr size_t kOffPartials = align_up(kOffRows + sizeof(nemd::Row) * kRowStride * kMaxCells);
constexpr size_t kOffCounters = align_up(kOffPartials + 8 * nemd::kPartials * kMaxBlocks);
constexpr size_t kOffPairCount = align_up(kOffCounters + 8 * 4);
constexpr size_t kOffRecheck = align_up(kOffPairCount + 8);
constexpr size_t kOffNRecheck = align_up(kOffRecheck + sizeof(int4) * nemd::kRecheckCap);
constexpr size_t kScratchBytes = align_up(kOffNRecheck + 4);
static_assert(kScratchBytes == NEMD_NOALLOC_SCRATCH_BYTES, "header constant must match the layout");

// The scratch array.  Shared by every call on a device; it keeps the contents
// of the last call, so each call clears what must start at zero.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices];
int g_sms[kMaxDevices];

// Once per device, with that device current: the device address of the array.
int setup_device(int dev, unsigned char **ptr, int *sms) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return NEMD_ERR_CUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NEMD_ERR_CUDA;
    g_sms[dev] = n;
    g_scratch_ptr[dev] = (unsigned char *)p;
  }
  *ptr = g_scratch_ptr[dev];
  *sms = g_sms[dev];
  return NEMD_OK;
}

// p is device (or managed) memory of device dev, the device the call runs on.
bool on_device(const void *p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int nemd_forces_noalloc(const double A[9], const double L0[9], double T, double t, const double *q,
                                   int64_t n, int variant, double rc, int kind, double eps, double sigma, int shift,
                                   float *F, double *UW, int *status, void *stream) {
  // ---- argument checks (host only, nothing is launched on failure) ----
  if (!A || !L0 || !UW || (n > 0 && (!q || !F))) return NEMD_ERR_ARG;
  if (n < 0) return NEMD_ERR_ARG;
  if (n > kMaxN) return NEMD_ERR_CAPACITY;  // more particles than the static scratch holds
  if (variant != NEMD_DS && variant != NEMD_DO && variant != NEMD_AUTO_HEURISTIC) return NEMD_ERR_ARG;
  if (!(rc > 0.0) || !isfinite(rc) || !isfinite(t) || !(eps > 0.0) || !(sigma > 0.0)) return NEMD_ERR_ARG;
  if (kind != NEMD_LJ && kind != NEMD_WCA) return NEMD_ERR_ARG;
  if (kind == NEMD_WCA && (!shift || fabs(rc - pow(2.0, 1.0 / 6.0) * sigma) > 1e-12 * sigma)) return NEMD_ERR_ARG;
  const double V = fabs(L0[0] * (L0[4] * L0[8] - L0[5] * L0[7]) - L0[1] * (L0[3] * L0[8] - L0[5] * L0[6]) +
                        L0[2] * (L0[3] * L0[7] - L0[4] * L0[6]));
  if (!(V > 0.0)) return NEMD_ERR_ARG;
  const double cell_bound = V / (rc * rc * rc) * (1.0 + 1e-9) + 1.0;
  if (cell_bound > (double)kMaxCells) return NEMD_ERR_CAPACITY;  // more cells than the static scratch holds
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NEMD_ERR_CUDA;
  if (n > 0 && (!on_device(q, dev) || !on_device(F, dev))) return NEMD_ERR_ARG;
  if (!on_device(UW, dev) || (status && !on_device(status, dev))) return NEMD_ERR_ARG;
  unsigned char *base = nullptr;
  int sms = 0;
  int r = setup_device(dev, &base, &sms);
  if (r) return r;

  // ---- a context on the stack whose buffers are slices of the scratch array ----
  nemd_ctx c;
  memset(&c, 0, sizeof c);
  c.device = dev;
  c.stream = (cudaStream_t)stream;
  c.sms = sms;
  for (int k = 0; k < 9; k++) {
    c.A[k] = A[k];
    c.L0[k] = L0[k];
  }
  c.T = T;
  c.pot_kind = kind;
  c.eps = eps;
  c.sigma = sigma;
  c.shift = shift ? 1 : 0;
  c.n = n;
  c.t = t;
  c.q_dev = n > 0 ? q : nullptr;
  c.rc = rc;
  c.variant_req = variant;
  c.kfac = 1;
  c.block = 128;
  c.geo = (nemd::Geo *)(base + kOffGeo);
  c.cap_n = kMaxN;
  c.cap_cells = kMaxCells;
  c.cap_rows = kMaxCells * kRowStride;
  c.relc = (float4 *)(base + kOffRelc);
  c.relr = (float4 *)(base + kOffRelr);
  c.pos4 = (float4 *)(base + kOffPos4);
  c.posr = (float4 *)(base + kOffPosr);
  c.rank = (int *)(base + kOffRank);
  c.perm = (int *)(base + kOffPerm);
  c.cell_sorted = (int *)(base + kOffCellSorted);
  c.count = (int *)(base + kOffCount);
  c.start = (int *)(base + kOffStart);
  c.block_sums = (int *)(base + kOffBlockSums);
  c.rowcnt = (int *)(base + kOffRowcnt);
  c.rows = (nemd::Row *)(base + kOffRows);
  c.partials = (double *)(base + kOffPartials);
  c.cap_partials = kMaxBlocks;
  c.counters = (unsigned long long *)(base + kOffCounters);
  c.pair_count = (unsigned long long *)(base + kOffPairCount);
  c.recheck = (int4 *)(base + kOffRecheck);
  c.nrecheck = (int *)(base + kOffNRecheck);

  // the geometry record (including its error words) starts from zero every call;
  // the cell counts are cleared by the binning step itself
  if (cudaMemsetAsync(c.geo, 0, sizeof(nemd::Geo), c.stream) != cudaSuccess) return NEMD_ERR_CUDA;
  cudaError_t e = nemd::launch_lattice(&c, 0, 0.0);
  if (e == cudaSuccess) e = nemd::launch_grid(&c);
  if (e == cudaSuccess) e = nemd::launch_stencil(&c);
  if (e == cudaSuccess) e = nemd::launch_bin(&c);
  if (e == cudaSuccess) e = nemd::launch_forces(&c, n > 0 ? F : nullptr, UW);
  if (e == cudaSuccess && status)
    e = cudaMemcpyAsync(status, &c.geo->sticky, sizeof(int), cudaMemcpyDeviceToDevice, c.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return NEMD_ERR_CUDA;
  }
  return NEMD_OK;
}
