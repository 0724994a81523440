// mlp.cu -- the learned cell-list selector: a small multilayer perceptron that
// predicts, from the deformed lattice, the time of each cell-list option and
// picks the fastest per step.  The paper has no counterpart; its own choice
// rule is the neighbourhood-volume comparison of Sec. 5.1-5.2, which stays the
// fallback (no trained model) and the baseline the learned choice is judged
// against.  The choice changes only the time, never the pair set or forces.
//
// Inputs (12): the 9 entries of L(t) / V^(1/3), the number density N / V, the
// cut-off rc and ln N.  Outputs (4): predicted normalised ln(time / N) of
// option o = (variant o & 1, cell factor 1 + (o >> 1)).  Layers 12 -> 64 (ReLU)
// -> 64 (ReLU) -> 4, float32.  Training minimises the mean squared error of
// the normalised ln(time / N) with Adam; gradients are summed per weight over the
// batch in a fixed order (one thread per weight), so training is deterministic.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "nemd_internal.cuh"

namespace nemd {

namespace {

constexpr int DI = kMlpIn, H = kMlpHidden, DO_ = kMlpOut;
constexpr int OW1 = 0, OB1 = OW1 + H * DI, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + DO_ * H;
static_assert(OB3 + DO_ == kMlpParams, "parameter layout");

// Features of the current step, from the device lattice, in float32 (inputs
// of a float32 network; training and inference both come through here).  No
// float64 division: one costs ~0.3 us of latency on this part, and this runs
// on one thread at every build.
__device__ void step_features(const Geo *g, int64_t n, double rc, float *x) {
  const float V = (float)g->V;
  const float is = 1.0f / cbrtf(V);
  for (int k = 0; k < 9; k++) x[k] = (float)g->L[k] * is;
  x[9] = (float)n / V;
  x[10] = (float)rc;
  x[11] = logf((float)(n > 0 ? n : 1));
}

// One sample's forward pass in a block of H threads; h1, h2 in shared memory.
__device__ void forward_one(const float *p, const float *xn, float *h1, float *h2, float *y) {
  const int t = threadIdx.x;
  if (t < H) {
    float a = p[OB1 + t];
    for (int i = 0; i < DI; i++) a = fmaf(p[OW1 + t * DI + i], xn[i], a);
    h1[t] = fmaxf(a, 0.f);
  }
  __syncthreads();
  if (t < H) {
    float a = p[OB2 + t];
    for (int k = 0; k < H; k++) a = fmaf(p[OW2 + t * H + k], h1[k], a);
    h2[t] = fmaxf(a, 0.f);
  }
  __syncthreads();
  if (t < DO_) {
    float a = p[OB3 + t];
    for (int k = 0; k < H; k++) a = fmaf(p[OW3 + t * H + k], h2[k], a);
    y[t] = a;
  }
  __syncthreads();
}

}  // namespace

// Per step (between the lattice and grid kernels): features, forward pass,
// the option with the smallest predicted time -> g->learned_choice.
__global__ void k_learned_choice(Geo *g, const float *__restrict__ model, int64_t n, double rc, int have_model) {
  __shared__ float xn[DI], h1[H], h2[H], y[DO_];
  if (!have_model) {
    if (threadIdx.x == 0) g->learned_choice = -1;
    return;
  }
  const float *p = model;
  const float *mu = model + kMlpParams, *sd = mu + DI;
  if (threadIdx.x == 0) {
    float x[DI];
    step_features(g, n, rc, x);
    for (int i = 0; i < DI; i++) xn[i] = (x[i] - mu[i]) / sd[i];
  }
  __syncthreads();
  forward_one(p, xn, h1, h2, y);
  if (threadIdx.x == 0) {
    int best = 0;
    for (int o = 1; o < DO_; o++)
      if (y[o] < y[best]) best = o;
    g->learned_choice = best;
  }
}

__global__ void k_features(const Geo *g, int64_t n, double rc, float *out) {
  if (threadIdx.x == 0) step_features(g, n, rc, out);
}

// Training: forward pass of every sample (block per sample), storing activations.
__global__ void k_mlp_forward(const float *__restrict__ p, const float *__restrict__ X, int B,
                              float *__restrict__ H1, float *__restrict__ H2, float *__restrict__ Y) {
  __shared__ float xn[DI], h1[H], h2[H], y[DO_];
  const int b = blockIdx.x;
  if (b >= B) return;
  if (threadIdx.x < DI) xn[threadIdx.x] = X[b * DI + threadIdx.x];
  __syncthreads();
  forward_one(p, xn, h1, h2, y);
  if (threadIdx.x < H) {
    H1[b * H + threadIdx.x] = h1[threadIdx.x];
    H2[b * H + threadIdx.x] = h2[threadIdx.x];
  }
  if (threadIdx.x < DO_) Y[b * DO_ + threadIdx.x] = y[threadIdx.x];
}

// Back-propagated errors of every sample: D3 = dL/dy, D2 = dL/dh2 pre-ReLU,
// D1 = dL/dh1 pre-ReLU, for L = sum (y - t)^2 / (B * DO); and each sample's
// squared error.
__global__ void k_mlp_delta(const float *__restrict__ p, const float *__restrict__ T, int B,
                            const float *__restrict__ H1, const float *__restrict__ H2, const float *__restrict__ Y,
                            float *__restrict__ D1, float *__restrict__ D2, float *__restrict__ D3,
                            float *__restrict__ sqerr) {
  __shared__ float d3[DO_], d2[H];
  const int b = blockIdx.x, t = threadIdx.x;
  if (b >= B) return;
  const float scale = 2.0f / (float)(B * DO_);
  if (t < DO_) {
    const float e = Y[b * DO_ + t] - T[b * DO_ + t];
    d3[t] = scale * e;
    D3[b * DO_ + t] = d3[t];
  }
  if (t == 0) {
    float s = 0.f;
    for (int o = 0; o < DO_; o++) {
      const float e = Y[b * DO_ + o] - T[b * DO_ + o];
      s += e * e;
    }
    sqerr[b] = s;
  }
  __syncthreads();
  if (t < H) {
    float a = 0.f;
    for (int o = 0; o < DO_; o++) a = fmaf(p[OW3 + o * H + t], d3[o], a);
    d2[t] = H2[b * H + t] > 0.f ? a : 0.f;
    D2[b * H + t] = d2[t];
  }
  __syncthreads();
  if (t < H) {
    float a = 0.f;
    for (int k = 0; k < H; k++) a = fmaf(p[OW2 + k * H + t], d2[k], a);
    D1[b * H + t] = H1[b * H + t] > 0.f ? a : 0.f;
  }
}

// One thread per parameter: its gradient summed over the batch in sample order.
__global__ void k_mlp_wgrad(const float *__restrict__ X, const float *__restrict__ H1, const float *__restrict__ H2,
                            const float *__restrict__ D1, const float *__restrict__ D2, const float *__restrict__ D3,
                            int B, float *__restrict__ grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kMlpParams) return;
  float s = 0.f;
  if (k < OB1) {
    const int h = k / DI, i = k % DI;
    for (int b = 0; b < B; b++) s = fmaf(D1[b * H + h], X[b * DI + i], s);
  } else if (k < OW2) {
    const int h = k - OB1;
    for (int b = 0; b < B; b++) s += D1[b * H + h];
  } else if (k < OB2) {
    const int h = (k - OW2) / H, j = (k - OW2) % H;
    for (int b = 0; b < B; b++) s = fmaf(D2[b * H + h], H1[b * H + j], s);
  } else if (k < OW3) {
    const int h = k - OB2;
    for (int b = 0; b < B; b++) s += D2[b * H + h];
  } else if (k < OB3) {
    const int o = (k - OW3) / H, j = (k - OW3) % H;
    for (int b = 0; b < B; b++) s = fmaf(D3[b * DO_ + o], H2[b * H + j], s);
  } else {
    const int o = k - OB3;
    for (int b = 0; b < B; b++) s += D3[b * DO_ + o];
  }
  grad[k] = s;
}

// Adam (Kingma & Ba 2015) with bias correction.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ grad, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kMlpParams) return;
  const float g = grad[k];
  const float mk = b1 * m[k] + (1.f - b1) * g;
  const float vk = b2 * v[k] + (1.f - b2) * g * g;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// Gather a mini-batch (normalised inputs and targets).
__global__ void k_gather_batch(const float *__restrict__ X, const float *__restrict__ T, const int *__restrict__ idx,
                               int B, float *__restrict__ Xb, float *__restrict__ Tb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int r = idx[b];
  for (int i = 0; i < DI; i++) Xb[b * DI + i] = X[r * DI + i];
  for (int o = 0; o < DO_; o++) Tb[b * DO_ + o] = T[r * DO_ + o];
}

cudaError_t launch_learned_choice(nemd_ctx *c, double rc) {
  k_learned_choice<<<1, H, 0, c->stream>>>(c->geo, c->model, c->n, rc, c->have_model);
  c->launches += 1;
  return cudaGetLastError();
}

}  // namespace nemd

// ------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------

namespace {

int ensure_model(nemd_ctx *c) {
  if (c->model) return NEMD_OK;
  // params | input mean | input std | target mean, std | Adam m | Adam v
  const size_t nf = nemd::kMlpParams + 2 * nemd::kMlpIn + 2 + 2 * nemd::kMlpParams;
  if (cudaMalloc((void **)&c->model, nf * sizeof(float)) != cudaSuccess) return NEMD_ERR_NOMEM;
  cudaMemset(c->model, 0, nf * sizeof(float));
  return NEMD_OK;
}

uint64_t splitmix(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double uniform01(uint64_t &s) { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

// Glorot-uniform initial weights, zero biases (host, seeded).
void init_params(float *p, uint64_t seed) {
  using namespace nemd;
  uint64_t s = seed;
  auto fill = [&](int off, int fan_out, int fan_in) {
    const double a = sqrt(6.0 / (fan_in + fan_out));
    for (int k = 0; k < fan_out * fan_in; k++) p[off + k] = (float)((2.0 * uniform01(s) - 1.0) * a);
  };
  memset(p, 0, sizeof(float) * kMlpParams);
  fill(0, kMlpHidden, kMlpIn);
  fill(kMlpHidden * kMlpIn + kMlpHidden, kMlpHidden, kMlpHidden);
  fill(kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden, kMlpOut, kMlpHidden);
}

}  // namespace

extern "C" {

int nemd_model_set_params(nemd_ctx *c, const float *params, const float *norm) {
  if (!c || !params || !norm) return NEMD_ERR_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return NEMD_ERR_CUDA;
  int r = ensure_model(c);
  if (r) return r;
  if (cudaMemcpy(c->model, params, sizeof(float) * nemd::kMlpParams, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->model + nemd::kMlpParams, norm, sizeof(float) * (2 * nemd::kMlpIn + 2), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return NEMD_ERR_CUDA;
  memcpy(c->model_norm_host, norm, sizeof(float) * (2 * nemd::kMlpIn + 2));
  c->have_model = 1;
  return NEMD_OK;
}

int nemd_model_get_params(nemd_ctx *c, float *params, float *norm) {
  if (!c || !params || !norm) return NEMD_ERR_ARG;
  if (!c->model) return NEMD_ERR_ORDER;
  if (cudaSetDevice(c->device) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) return NEMD_ERR_CUDA;
  if (cudaMemcpy(params, c->model, sizeof(float) * nemd::kMlpParams, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(norm, c->model + nemd::kMlpParams, sizeof(float) * (2 * nemd::kMlpIn + 2), cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return NEMD_ERR_CUDA;
  return NEMD_OK;
}

int nemd_model_predict(nemd_ctx *c, const float *X, int64_t rows, float *Y) {
  if (!c || (rows > 0 && (!X || !Y)) || rows < 0 || rows > (1 << 20)) return NEMD_ERR_ARG;
  if (!c->have_model) return NEMD_ERR_ORDER;
  if (rows == 0) return NEMD_OK;
  if (cudaSetDevice(c->device) != cudaSuccess) return NEMD_ERR_CUDA;
  const int DI = nemd::kMlpIn, H = nemd::kMlpHidden, DO_ = nemd::kMlpOut;
  float *xn = (float *)malloc(sizeof(float) * rows * DI);
  if (!xn) return NEMD_ERR_NOMEM;
  const float *mu = c->model_norm_host, *sd = mu + DI;
  for (int64_t b = 0; b < rows; b++)
    for (int i = 0; i < DI; i++) xn[b * DI + i] = (X[b * DI + i] - mu[i]) / sd[i];
  float *d = nullptr;
  const size_t nb = (size_t)rows;
  if (cudaMalloc((void **)&d, sizeof(float) * nb * (DI + 2 * H + DO_)) != cudaSuccess) {
    free(xn);
    return NEMD_ERR_NOMEM;
  }
  float *dX = d, *dH1 = d + nb * DI, *dH2 = dH1 + nb * H, *dY = dH2 + nb * H;
  cudaMemcpy(dX, xn, sizeof(float) * nb * DI, cudaMemcpyHostToDevice);
  nemd::k_mlp_forward<<<(int)rows, H>>>(c->model, dX, (int)rows, dH1, dH2, dY);
  cudaError_t e = cudaMemcpy(Y, dY, sizeof(float) * nb * DO_, cudaMemcpyDeviceToHost);
  cudaFree(d);
  free(xn);
  return e == cudaSuccess ? NEMD_OK : NEMD_ERR_CUDA;
}

// Gradient of L = sum (y - t)^2 / (rows * 4) with respect to the parameters at
// the current parameters, for normalised inputs Xn and targets Tn (host).
int nemd_model_grad(nemd_ctx *c, const float *Xn, const float *Tn, int64_t rows, float *grad, double *loss) {
  if (!c || !Xn || !Tn || !grad || rows < 1 || rows > (1 << 20)) return NEMD_ERR_ARG;
  if (!c->model) return NEMD_ERR_ORDER;
  if (cudaSetDevice(c->device) != cudaSuccess) return NEMD_ERR_CUDA;
  const int DI = nemd::kMlpIn, H = nemd::kMlpHidden, DO_ = nemd::kMlpOut;
  const size_t nb = (size_t)rows;
  float *d = nullptr;
  const size_t nf = nb * (DI + DO_ + 4 * H + 2 * DO_ + 1) + nemd::kMlpParams;
  if (cudaMalloc((void **)&d, sizeof(float) * nf) != cudaSuccess) return NEMD_ERR_NOMEM;
  float *dX = d, *dT = dX + nb * DI, *dH1 = dT + nb * DO_, *dH2 = dH1 + nb * H, *dY = dH2 + nb * H,
        *dD1 = dY + nb * DO_, *dD2 = dD1 + nb * H, *dD3 = dD2 + nb * H, *dE = dD3 + nb * DO_, *dG = dE + nb;
  cudaMemcpy(dX, Xn, sizeof(float) * nb * DI, cudaMemcpyHostToDevice);
  cudaMemcpy(dT, Tn, sizeof(float) * nb * DO_, cudaMemcpyHostToDevice);
  nemd::k_mlp_forward<<<(int)rows, H>>>(c->model, dX, (int)rows, dH1, dH2, dY);
  nemd::k_mlp_delta<<<(int)rows, H>>>(c->model, dT, (int)rows, dH1, dH2, dY, dD1, dD2, dD3, dE);
  nemd::k_mlp_wgrad<<<(nemd::kMlpParams + 127) / 128, 128>>>(dX, dH1, dH2, dD1, dD2, dD3, (int)rows, dG);
  cudaError_t e = cudaMemcpy(grad, dG, sizeof(float) * nemd::kMlpParams, cudaMemcpyDeviceToHost);
  if (loss && e == cudaSuccess) {
    float *err = (float *)malloc(sizeof(float) * nb);
    if (err && cudaMemcpy(err, dE, sizeof(float) * nb, cudaMemcpyDeviceToHost) == cudaSuccess) {
      double s = 0.0;
      for (size_t b = 0; b < nb; b++) s += err[b];
      *loss = s / (double)(nb * DO_);
    }
    free(err);
  }
  cudaFree(d);
  return e == cudaSuccess ? NEMD_OK : NEMD_ERR_CUDA;
}

// Train on (features X, times T in ms, rows x 4) from scratch: inputs and
// ln(time / N) targets are normalised by their mean and standard deviation,
// weights start Glorot-uniform from `seed`, then `steps` Adam steps on
// mini-batches of `batch` rows drawn with replacement.  loss_hist (optional,
// `steps` entries) receives each step's mini-batch loss.
int nemd_model_train(nemd_ctx *c, const float *X, const float *Tms, int64_t rows, int steps, int batch, double lr,
                     uint64_t seed, float *loss_hist) {
  if (!c || !X || !Tms || rows < 2 || rows > (1 << 20) || steps < 1 || batch < 1 || batch > 4096 || !(lr > 0.0))
    return NEMD_ERR_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return NEMD_ERR_CUDA;
  int r = ensure_model(c);
  if (r) return r;
  const int DI = nemd::kMlpIn, H = nemd::kMlpHidden, DO_ = nemd::kMlpOut, P = nemd::kMlpParams;
  const size_t nr = (size_t)rows;
  // normalisation (host): input means / std, one mean / std over all targets.
  // Targets are ln(time / N) (x[11] = ln N): the time per particle depends far
  // less on N than the time itself, so a system larger than every training
  // system is not an extrapolation of the target; the option with the smallest
  // prediction is the same either way.
  float norm[2 * nemd::kMlpIn + 2];
  for (int i = 0; i < DI; i++) {
    double m = 0.0, v = 0.0;
    for (size_t b = 0; b < nr; b++) m += X[b * DI + i];
    m /= (double)nr;
    for (size_t b = 0; b < nr; b++) v += (X[b * DI + i] - m) * (X[b * DI + i] - m);
    v = sqrt(v / (double)nr);
    norm[i] = (float)m;
    norm[DI + i] = (float)(v > 1e-6 ? v : 1.0);
  }
  auto target = [&](size_t k) { return log((double)Tms[k]) - (double)X[(k / DO_) * DI + (DI - 1)]; };
  double tm = 0.0, tv = 0.0;
  for (size_t k = 0; k < nr * DO_; k++) {
    if (!(Tms[k] > 0.f)) return NEMD_ERR_ARG;
    tm += target(k);
  }
  tm /= (double)(nr * DO_);
  for (size_t k = 0; k < nr * DO_; k++) tv += (target(k) - tm) * (target(k) - tm);
  tv = sqrt(tv / (double)(nr * DO_));
  norm[2 * DI] = (float)tm;
  norm[2 * DI + 1] = (float)(tv > 1e-6 ? tv : 1.0);
  float *xn = (float *)malloc(sizeof(float) * nr * (DI + DO_));
  float *p0 = (float *)malloc(sizeof(float) * P);
  int *idx = (int *)malloc(sizeof(int) * batch);
  if (!xn || !p0 || !idx) {
    free(xn);
    free(p0);
    free(idx);
    return NEMD_ERR_NOMEM;
  }
  float *tn = xn + nr * DI;
  for (size_t b = 0; b < nr; b++) {
    for (int i = 0; i < DI; i++) xn[b * DI + i] = (X[b * DI + i] - norm[i]) / norm[DI + i];
    for (int o = 0; o < DO_; o++) tn[b * DO_ + o] = (float)((target(b * DO_ + o) - tm) / norm[2 * DI + 1]);
  }
  init_params(p0, seed);
  r = nemd_model_set_params(c, p0, norm);
  if (r) {
    free(xn);
    free(p0);
    free(idx);
    return r;
  }
  const size_t B = (size_t)batch;
  float *d = nullptr;
  const size_t nf = nr * (DI + DO_) + B * (DI + DO_ + 4 * H + 2 * DO_ + 1) + P;
  int *didx = nullptr;
  if (cudaMalloc((void **)&d, sizeof(float) * nf) != cudaSuccess || cudaMalloc((void **)&didx, sizeof(int) * B) != cudaSuccess) {
    cudaFree(d);
    free(xn);
    free(p0);
    free(idx);
    return NEMD_ERR_NOMEM;
  }
  float *dX = d, *dT = dX + nr * DI, *bX = dT + nr * DO_, *bT = bX + B * DI, *dH1 = bT + B * DO_, *dH2 = dH1 + B * H,
        *dY = dH2 + B * H, *dD1 = dY + B * DO_, *dD2 = dD1 + B * H, *dD3 = dD2 + B * H, *dE = dD3 + B * DO_,
        *dG = dE + B;
  cudaMemcpy(dX, xn, sizeof(float) * nr * DI, cudaMemcpyHostToDevice);
  cudaMemcpy(dT, tn, sizeof(float) * nr * DO_, cudaMemcpyHostToDevice);
  float *m = c->model + P + 2 * DI + 2, *v = m + P;
  cudaMemset(m, 0, sizeof(float) * 2 * P);
  uint64_t s = seed ^ 0xA5A5A5A5ull;
  float *err = (float *)malloc(sizeof(float) * B);
  const float b1 = 0.9f, b2 = 0.999f;
  double c1 = 1.0, c2 = 1.0;
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < steps && e == cudaSuccess; it++) {
    for (size_t b = 0; b < B; b++) idx[b] = (int)(splitmix(s) % nr);
    cudaMemcpy(didx, idx, sizeof(int) * B, cudaMemcpyHostToDevice);
    nemd::k_gather_batch<<<(int)((B + 127) / 128), 128>>>(dX, dT, didx, (int)B, bX, bT);
    nemd::k_mlp_forward<<<(int)B, H>>>(c->model, bX, (int)B, dH1, dH2, dY);
    nemd::k_mlp_delta<<<(int)B, H>>>(c->model, bT, (int)B, dH1, dH2, dY, dD1, dD2, dD3, dE);
    nemd::k_mlp_wgrad<<<(P + 127) / 128, 128>>>(bX, dH1, dH2, dD1, dD2, dD3, (int)B, dG);
    c1 *= b1;
    c2 *= b2;
    nemd::k_adam<<<(P + 127) / 128, 128>>>(c->model, dG, m, v, (float)lr, b1, b2, 1e-8f, (float)(1.0 - c1),
                                           (float)(1.0 - c2));
    e = cudaGetLastError();
    if (loss_hist && err && e == cudaSuccess) {
      e = cudaMemcpy(err, dE, sizeof(float) * B, cudaMemcpyDeviceToHost);
      double acc = 0.0;
      for (size_t b = 0; b < B; b++) acc += err[b];
      loss_hist[it] = (float)(acc / (double)(B * DO_));
    }
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d);
  cudaFree(didx);
  free(err);
  free(xn);
  free(p0);
  free(idx);
  return e == cudaSuccess ? NEMD_OK : NEMD_ERR_CUDA;
}

// Model file: "NEMDMLP1" | u32 inputs | u32 hidden | u32 outputs | params |
// normalisation | u64 FNV-1a of everything before it.
static uint64_t fnv1a64(const unsigned char *p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; i++) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

int nemd_model_save(nemd_ctx *c, const char *path) {
  if (!c || !path) return NEMD_ERR_ARG;
  if (!c->have_model) return NEMD_ERR_ORDER;
  const size_t np = nemd::kMlpParams, nn = 2 * nemd::kMlpIn + 2;
  const size_t n = 8 + 12 + 4 * (np + nn);
  unsigned char *buf = (unsigned char *)malloc(n + 8);
  if (!buf) return NEMD_ERR_NOMEM;
  const uint32_t dims[3] = {nemd::kMlpIn, nemd::kMlpHidden, nemd::kMlpOut};
  memcpy(buf, "NEMDMLP1", 8);
  memcpy(buf + 8, dims, 12);
  int r = nemd_model_get_params(c, (float *)(buf + 20), (float *)(buf + 20 + 4 * np));
  if (r) {
    free(buf);
    return r;
  }
  const uint64_t h = fnv1a64(buf, n);
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

int nemd_model_load(nemd_ctx *c, const char *path) {
  if (!c || !path) return NEMD_ERR_ARG;
  const size_t np = nemd::kMlpParams, nn = 2 * nemd::kMlpIn + 2;
  const size_t n = 8 + 12 + 4 * (np + nn);
  unsigned char *buf = (unsigned char *)malloc(n + 8);
  if (!buf) return NEMD_ERR_NOMEM;
  FILE *f = fopen(path, "rb");
  const size_t got = f ? fread(buf, 1, n + 8, f) : 0;
  if (f) fclose(f);
  const uint32_t dims[3] = {nemd::kMlpIn, nemd::kMlpHidden, nemd::kMlpOut};
  uint64_t h = 0;
  if (got == n + 8) memcpy(&h, buf + n, 8);
  if (got != n + 8 || memcmp(buf, "NEMDMLP1", 8) != 0 || memcmp(buf + 8, dims, 12) != 0 || h != fnv1a64(buf, n)) {
    free(buf);
    return NEMD_ERR_ARG;
  }
  int r = nemd_model_set_params(c, (const float *)(buf + 20), (const float *)(buf + 20 + 4 * np));
  free(buf);
  return r;
}

// Features of the current state (after nemd_set_state; synchronises).
int nemd_features(nemd_ctx *c, double rc, float *out) {
  if (!c || !out) return NEMD_ERR_ARG;
  if (!c->have_state) return NEMD_ERR_ORDER;
  if (cudaSetDevice(c->device) != cudaSuccess) return NEMD_ERR_CUDA;
  float *d = nullptr;
  if (cudaMalloc((void **)&d, sizeof(float) * nemd::kMlpIn) != cudaSuccess) return NEMD_ERR_NOMEM;
  nemd::k_features<<<1, 32, 0, c->stream>>>(c->geo, c->n, rc, d);
  cudaError_t e = cudaMemcpyAsync(out, d, sizeof(float) * nemd::kMlpIn, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  return e == cudaSuccess ? NEMD_OK : NEMD_ERR_CUDA;
}

// Time every option o = (variant o & 1, cell factor 1 + (o >> 1)) on the
// current state: one untimed then `reps` timed nemd_build_cells +
// nemd_compute_forces each, CUDA events on the context's stream.  features[12]
// receives the selector's inputs, ms[4] the mean times.  Synchronises.
int nemd_time_options(nemd_ctx *c, double rc, int reps, float *features, float *ms) {
  if (!c || !features || !ms || reps < 1 || reps > 1000) return NEMD_ERR_ARG;
  if (!c->have_state) return NEMD_ERR_ORDER;
  int r = nemd_features(c, rc, features);
  if (r) return r;
  if (!c->f_dev && c->n > 0) {
    if (cudaMalloc((void **)&c->f_dev, sizeof(float) * 3 * (size_t)c->cap_n) != cudaSuccess) return NEMD_ERR_NOMEM;
  }
  const int kf = c->kfac, tuned = c->autotuned;
  c->autotuned = 0;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return NEMD_ERR_CUDA;
  for (int o = 0; o < nemd::kMlpOut && !r; o++) {
    c->kfac = 1 + (o >> 1);
    const int variant = o & 1;
    r = nemd_build_cells(c, variant, rc);
    if (!r) r = nemd_compute_forces(c, c->f_dev, nullptr, nullptr);
    cudaEventRecord(e0, c->stream);
    for (int k = 0; k < reps && !r; k++) {
      r = nemd_build_cells(c, variant, rc);
      if (!r) r = nemd_compute_forces(c, c->f_dev, nullptr, nullptr);
    }
    cudaEventRecord(e1, c->stream);
    if (!r && cudaEventSynchronize(e1) != cudaSuccess) r = NEMD_ERR_CUDA;
    if (!r) r = nemd_sync(c);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    ms[o] = t / (float)reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->kfac = kf;
  c->autotuned = tuned;
  return r;
}

}  // extern "C"
