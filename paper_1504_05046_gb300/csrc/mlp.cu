// Learned task-cost model: a small MLP trained on the GPU from per-unit timings.
//
// The paper balances load by over-decomposition and dynamic task scheduling
// (Sec. 3.2) and notes that nonuniform blocking makes block work vary several-fold
// (Sec. 4.4, Table 1). Here the work units are packed statically onto persistent
// CTAs, longest first, so the packing is only as good as the cost estimates. The
// flop count misjudges units made of small or ragged tiles (padding, per-block
// recombination and pipeline overheads do not scale with flops); this MLP learns the
// measured cost of a unit from its features, and bsmm_plan_predict_costs feeds its
// predictions to the packer. Results never depend on it: only the order changes.
//
// Model (F = BSMM_NFEATURES inputs, H = 32): features standardised with stored means
// and deviations, two tanh layers, one linear output = standardised log time.
// Parameters in one float vector: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
// Training: full-batch mean squared error, Adam; every reduction over samples runs in
// a fixed order (per-block partial sums, then a sum over blocks in block order), so
// training is bit-for-bit reproducible.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "bsmm_internal.h"

using namespace bsmm;

namespace {

constexpr int F = BSMM_NFEATURES;
constexpr int H = 32;
constexpr int NP = H * F + H + H * H + H + H + 1;
constexpr int OW1 = 0, OB1 = H * F, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H;
constexpr int TILE = 128;  // samples per block in the gradient kernel

struct Norm {
  float xmu[F], xsd[F];
  float ymu, ysd;
};

__device__ __forceinline__ void mlp_forward_one(const float* __restrict__ w, const float* x, float* h1, float* h2,
                                                float& y) {
#pragma unroll 4
  for (int j = 0; j < H; j++) {
    float z = w[OB1 + j];
#pragma unroll
    for (int f = 0; f < F; f++) z = fmaf(w[OW1 + j * F + f], x[f], z);
    h1[j] = tanhf(z);
  }
#pragma unroll 4
  for (int j = 0; j < H; j++) {
    float z = w[OB2 + j];
    for (int i = 0; i < H; i++) z = fmaf(w[OW2 + j * H + i], h1[i], z);
    h2[j] = tanhf(z);
  }
  float o = w[OB3];
  for (int i = 0; i < H; i++) o = fmaf(w[OW3 + i], h2[i], o);
  y = o;
}

__global__ void mlp_predict_kernel(const float* __restrict__ params, Norm nm, const float* __restrict__ X, int64_t n,
                                   float* __restrict__ y) {
  __shared__ float w[NP];
  for (int p = threadIdx.x; p < NP; p += blockDim.x) w[p] = params[p];
  __syncthreads();
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[F], h1[H], h2[H], o;
#pragma unroll
  for (int f = 0; f < F; f++) x[f] = (X[s * F + f] - nm.xmu[f]) / nm.xsd[f];
  mlp_forward_one(w, x, h1, h2, o);
  y[s] = o * nm.ysd + nm.ymu;  // log time in the caller's units
}

// Per block: the loss and gradient contributions of its TILE samples, summed in
// sample order, written to part[block][0..NP] (entry NP = sum of squared residuals).
__global__ void __launch_bounds__(TILE) mlp_grad_kernel(const float* __restrict__ params, Norm nm,
                                                        const float* __restrict__ X, const float* __restrict__ t,
                                                        int64_t n, float* __restrict__ part) {
  extern __shared__ float sm[];
  float* w = sm;                 // NP
  float* xs = w + NP;            // TILE x F
  float* h1s = xs + TILE * F;    // TILE x H
  float* h2s = h1s + TILE * H;   // TILE x H
  float* d1s = h2s + TILE * H;   // TILE x H  (dL/dz1)
  float* d2s = d1s + TILE * H;   // TILE x H  (dL/dz2)
  float* dys = d2s + TILE * H;   // TILE      (dL/dy)
  float* r2s = dys + TILE;       // TILE      squared residuals
  for (int p = threadIdx.x; p < NP; p += blockDim.x) w[p] = params[p];
  __syncthreads();
  const int tid = threadIdx.x;
  const int64_t s = (int64_t)blockIdx.x * TILE + tid;
  float* x = xs + tid * F;
  float* h1 = h1s + tid * H;
  float* h2 = h2s + tid * H;
  float* d1 = d1s + tid * H;
  float* d2 = d2s + tid * H;
  if (s < n) {
#pragma unroll
    for (int f = 0; f < F; f++) x[f] = (X[s * F + f] - nm.xmu[f]) / nm.xsd[f];
    float y;
    mlp_forward_one(w, x, h1, h2, y);
    const float r = y - (t[s] - nm.ymu) / nm.ysd;
    const float dy = 2.0f * r / (float)n;
    dys[tid] = dy;
    r2s[tid] = r * r;
    for (int j = 0; j < H; j++) d2[j] = dy * w[OW3 + j] * (1.0f - h2[j] * h2[j]);
    for (int i = 0; i < H; i++) {
      float g = 0.0f;
      for (int j = 0; j < H; j++) g = fmaf(w[OW2 + j * H + i], d2[j], g);
      d1[i] = g * (1.0f - h1[i] * h1[i]);
    }
  } else {
    for (int f = 0; f < F; f++) x[f] = 0.0f;
    for (int j = 0; j < H; j++) h1[j] = h2[j] = d1[j] = d2[j] = 0.0f;
    dys[tid] = 0.0f;
    r2s[tid] = 0.0f;
  }
  __syncthreads();
  float* out = part + (int64_t)blockIdx.x * (NP + 1);
  for (int p = tid; p <= NP; p += blockDim.x) {
    float g = 0.0f;
    if (p < OB1) {
      const int j = p / F, f = p % F;
      for (int q = 0; q < TILE; q++) g = fmaf(d1s[q * H + j], xs[q * F + f], g);
    } else if (p < OW2) {
      const int j = p - OB1;
      for (int q = 0; q < TILE; q++) g += d1s[q * H + j];
    } else if (p < OB2) {
      const int j = (p - OW2) / H, i = (p - OW2) % H;
      for (int q = 0; q < TILE; q++) g = fmaf(d2s[q * H + j], h1s[q * H + i], g);
    } else if (p < OW3) {
      const int j = p - OB2;
      for (int q = 0; q < TILE; q++) g += d2s[q * H + j];
    } else if (p < OB3) {
      const int i = p - OW3;
      for (int q = 0; q < TILE; q++) g = fmaf(dys[q], h2s[q * H + i], g);
    } else if (p == OB3) {
      for (int q = 0; q < TILE; q++) g += dys[q];
    } else {  // p == NP: loss numerator
      for (int q = 0; q < TILE; q++) g += r2s[q];
    }
    out[p] = g;
  }
}

// grad[p] = sum over blocks in block order; grad[NP] = mean squared residual
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int nblocks, int64_t n, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > NP) return;
  float g = 0.0f;
  for (int b = 0; b < nblocks; b++) g += part[(int64_t)b * (NP + 1) + p];
  grad[p] = p == NP ? g / (float)n : g;
}

__global__ void mlp_adam_kernel(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ grad, float lr, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NP) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float g = grad[p];
  const float mm = b1 * m[p] + (1.0f - b1) * g;
  const float vv = b2 * v[p] + (1.0f - b2) * g * g;
  m[p] = mm;
  v[p] = vv;
  params[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double normal(uint64_t& s) {  // Box-Muller on two 53-bit uniforms
  const double u1 = ((splitmix64(s) >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = (splitmix64(s) >> 11) * 0x1.0p-53;
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

struct bsmm_mlp_s {
  Norm norm{};
  int64_t step = 0;
  DevBuf params, m, v, grad, part;
};

namespace {

bsmm_status mlp_alloc(DevBuf& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return BSMM_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e)),
           e == cudaErrorMemoryAllocation ? BSMM_ERR_NOMEM : BSMM_ERR_CUDA;
  }
  b.bytes = bytes ? bytes : 16;
  return BSMM_OK;
}

size_t grad_smem() { return sizeof(float) * (NP + TILE * F + 4 * TILE * H + 2 * TILE); }

bsmm_status loss_grad(bsmm_mlp_s* mlp, const float* X, const float* t, int64_t n, cudaStream_t st) {
  const int nb = (int)((n + TILE - 1) / TILE);
  bsmm_status s = mlp_alloc(mlp->part, sizeof(float) * (size_t)nb * (NP + 1));
  if (s != BSMM_OK) return s;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()) !=
        cudaSuccess)
      return set_error("cudaFuncSetAttribute failed"), BSMM_ERR_CUDA;
    attr = true;
  }
  mlp_grad_kernel<<<nb, TILE, grad_smem(), st>>>((const float*)mlp->params.p, mlp->norm, X, t, n,
                                                 (float*)mlp->part.p);
  mlp_reduce_kernel<<<(NP + 1 + 255) / 256, 256, 0, st>>>((const float*)mlp->part.p, nb, n, (float*)mlp->grad.p);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(std::string("mlp kernels: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  return BSMM_OK;
}

}  // namespace

extern "C" {

bsmm_status bsmm_mlp_create(bsmm_mlp_t* out, uint64_t seed) {
  if (!out) return set_error("out is NULL"), BSMM_ERR_INVALID;
  *out = nullptr;
  bsmm_mlp_s* mlp = new (std::nothrow) bsmm_mlp_s();
  if (!mlp) return set_error("out of host memory"), BSMM_ERR_NOMEM;
  std::vector<float> p(NP, 0.0f);
  uint64_t s = seed;
  for (int i = 0; i < H * F; i++) p[OW1 + i] = (float)(normal(s) / std::sqrt((double)F));
  for (int i = 0; i < H * H; i++) p[OW2 + i] = (float)(normal(s) / std::sqrt((double)H));
  for (int i = 0; i < H; i++) p[OW3 + i] = (float)(normal(s) / std::sqrt((double)H));
  for (int f = 0; f < F; f++) {
    mlp->norm.xmu[f] = 0.0f;
    mlp->norm.xsd[f] = 1.0f;
  }
  mlp->norm.ymu = 0.0f;
  mlp->norm.ysd = 1.0f;
  bsmm_status st;
  if ((st = mlp_alloc(mlp->params, sizeof(float) * NP)) != BSMM_OK || (st = mlp_alloc(mlp->m, sizeof(float) * NP)) != BSMM_OK ||
      (st = mlp_alloc(mlp->v, sizeof(float) * NP)) != BSMM_OK ||
      (st = mlp_alloc(mlp->grad, sizeof(float) * (NP + 1))) != BSMM_OK) {
    bsmm_mlp_destroy(mlp);
    return st;
  }
  if (cudaMemcpy(mlp->params.p, p.data(), sizeof(float) * NP, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(mlp->m.p, 0, sizeof(float) * NP) != cudaSuccess || cudaMemset(mlp->v.p, 0, sizeof(float) * NP) != cudaSuccess) {
    bsmm_mlp_destroy(mlp);
    return set_error("mlp initialisation copy failed"), BSMM_ERR_CUDA;
  }
  *out = mlp;
  return BSMM_OK;
}

int32_t bsmm_mlp_num_params(void) { return NP; }

bsmm_status bsmm_mlp_set_params(bsmm_mlp_t mlp, const float* params, int64_t n) {
  if (!mlp || !params || n != NP) return set_error("bad arguments (n must be bsmm_mlp_num_params())"), BSMM_ERR_INVALID;
  if (cudaMemcpy(mlp->params.p, params, sizeof(float) * NP, cudaMemcpyHostToDevice) != cudaSuccess)
    return set_error("copy failed"), BSMM_ERR_CUDA;
  return BSMM_OK;
}

bsmm_status bsmm_mlp_get_params(bsmm_mlp_t mlp, float* params, int64_t n) {
  if (!mlp || !params || n != NP) return set_error("bad arguments (n must be bsmm_mlp_num_params())"), BSMM_ERR_INVALID;
  if (cudaMemcpy(params, mlp->params.p, sizeof(float) * NP, cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_error("copy failed"), BSMM_ERR_CUDA;
  return BSMM_OK;
}

bsmm_status bsmm_mlp_set_norm(bsmm_mlp_t mlp, const float* xmu, const float* xsd, float ymu, float ysd) {
  if (!mlp || !xmu || !xsd || !(ysd > 0.0f)) return set_error("bad arguments"), BSMM_ERR_INVALID;
  for (int f = 0; f < F; f++) {
    if (!(xsd[f] > 0.0f)) return set_error("deviations must be > 0"), BSMM_ERR_INVALID;
    mlp->norm.xmu[f] = xmu[f];
    mlp->norm.xsd[f] = xsd[f];
  }
  mlp->norm.ymu = ymu;
  mlp->norm.ysd = ysd;
  return BSMM_OK;
}

bsmm_status bsmm_mlp_get_norm(bsmm_mlp_t mlp, float* xmu, float* xsd, float* ymu, float* ysd) {
  if (!mlp) return set_error("mlp is NULL"), BSMM_ERR_INVALID;
  for (int f = 0; f < F; f++) {
    if (xmu) xmu[f] = mlp->norm.xmu[f];
    if (xsd) xsd[f] = mlp->norm.xsd[f];
  }
  if (ymu) *ymu = mlp->norm.ymu;
  if (ysd) *ysd = mlp->norm.ysd;
  return BSMM_OK;
}

bsmm_status bsmm_mlp_loss_grad(bsmm_mlp_t mlp, const float* X, const float* t, int64_t n, float* loss, float* grad,
                               void* stream) {
  if (!mlp || !X || !t || n <= 0) return set_error("bad arguments"), BSMM_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  bsmm_status s = loss_grad(mlp, X, t, n, st);
  if (s != BSMM_OK) return s;
  std::vector<float> g(NP + 1);
  if (cudaMemcpyAsync(g.data(), mlp->grad.p, sizeof(float) * (NP + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return set_error("copy failed"), BSMM_ERR_CUDA;
  if (loss) *loss = g[NP];
  if (grad) std::memcpy(grad, g.data(), sizeof(float) * NP);
  return BSMM_OK;
}

bsmm_status bsmm_mlp_fit(bsmm_mlp_t mlp, const float* X, const float* t, int64_t n, int32_t steps, float lr,
                         float* final_loss, void* stream) {
  if (!mlp || !X || !t || n <= 0 || steps < 0 || !(lr > 0.0f)) return set_error("bad arguments"), BSMM_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  // standardisation from the data (host, FP64 sums in sample order)
  std::vector<float> hx((size_t)n * F), ht(n);
  if (cudaMemcpyAsync(hx.data(), X, sizeof(float) * hx.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(ht.data(), t, sizeof(float) * ht.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return set_error("copy failed"), BSMM_ERR_CUDA;
  for (int f = 0; f < F; f++) {
    double s1 = 0, s2 = 0;
    for (int64_t i = 0; i < n; i++) s1 += hx[i * F + f];
    const double mu = s1 / n;
    for (int64_t i = 0; i < n; i++) s2 += (hx[i * F + f] - mu) * (hx[i * F + f] - mu);
    const double sd = std::sqrt(s2 / n);
    mlp->norm.xmu[f] = (float)mu;
    mlp->norm.xsd[f] = sd > 0 ? (float)sd : 1.0f;
  }
  {
    double s1 = 0, s2 = 0;
    for (int64_t i = 0; i < n; i++) s1 += ht[i];
    const double mu = s1 / n;
    for (int64_t i = 0; i < n; i++) s2 += (ht[i] - mu) * (ht[i] - mu);
    const double sd = std::sqrt(s2 / n);
    mlp->norm.ymu = (float)mu;
    mlp->norm.ysd = sd > 0 ? (float)sd : 1.0f;
  }
  if (cudaMemsetAsync(mlp->m.p, 0, sizeof(float) * NP, st) != cudaSuccess ||
      cudaMemsetAsync(mlp->v.p, 0, sizeof(float) * NP, st) != cudaSuccess)
    return set_error("memset failed"), BSMM_ERR_CUDA;
  double c1 = 1.0, c2 = 1.0;
  for (int32_t k = 1; k <= steps; k++) {
    bsmm_status s = loss_grad(mlp, X, t, n, st);
    if (s != BSMM_OK) return s;
    c1 *= 0.9;
    c2 *= 0.999;
    mlp_adam_kernel<<<(NP + 255) / 256, 256, 0, st>>>((float*)mlp->params.p, (float*)mlp->m.p, (float*)mlp->v.p,
                                                       (const float*)mlp->grad.p, lr, (float)(1.0 - c1),
                                                       (float)(1.0 - c2));
  }
  if (cudaGetLastError() != cudaSuccess) return set_error("adam kernel failed"), BSMM_ERR_CUDA;
  if (final_loss) {
    bsmm_status s = loss_grad(mlp, X, t, n, st);
    if (s != BSMM_OK) return s;
    if (cudaMemcpyAsync(final_loss, (float*)mlp->grad.p + NP, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return set_error("copy failed"), BSMM_ERR_CUDA;
  }
  return BSMM_OK;
}

bsmm_status bsmm_mlp_predict(bsmm_mlp_t mlp, const float* X, int64_t n, float* y, void* stream) {
  if (!mlp || !X || !y || n < 0) return set_error("bad arguments"), BSMM_ERR_INVALID;
  if (n == 0) return BSMM_OK;
  mlp_predict_kernel<<<(int)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>((const float*)mlp->params.p,
                                                                               mlp->norm, X, n, y);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(std::string("predict: ") + cudaGetErrorString(e)), BSMM_ERR_CUDA;
  return BSMM_OK;
}

bsmm_status bsmm_plan_predict_costs(bsmm_plan_t plan, bsmm_mlp_t mlp, void* stream) {
  if (!plan || !mlp) return set_error("NULL argument"), BSMM_ERR_INVALID;
  const int64_t n = plan->n_units;
  if (n == 0) return BSMM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf dx, dy;
  bsmm_status s = mlp_alloc(dx, sizeof(float) * (size_t)n * F);
  if (s == BSMM_OK) s = mlp_alloc(dy, sizeof(float) * (size_t)n);
  std::vector<float> y(n);
  if (s == BSMM_OK) {
    if (cudaMemcpyAsync(dx.p, plan->features.data(), sizeof(float) * plan->features.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
      set_error("copy failed");
      s = BSMM_ERR_CUDA;
    }
  }
  if (s == BSMM_OK) s = bsmm_mlp_predict(mlp, (const float*)dx.p, n, (float*)dy.p, stream);
  if (s == BSMM_OK &&
      (cudaMemcpyAsync(y.data(), dy.p, sizeof(float) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess)) {
    set_error("copy failed");
    s = BSMM_ERR_CUDA;
  }
  if (dx.p) cudaFree(dx.p);
  if (dy.p) cudaFree(dy.p);
  if (s != BSMM_OK) return s;
  std::vector<double> cost(n);
  for (int64_t u = 0; u < n; u++) cost[u] = std::exp(std::min(60.0, std::max(-60.0, (double)y[u])));
  return bsmm_plan_set_costs(plan, cost.data());
}

}  // extern "C"

namespace {

constexpr char kMagic[8] = {'B', 'S', 'M', 'M', 'M', 'L', 'P', '\0'};
constexpr uint32_t kFormatVersion = 1;

// FNV-1a, 64 bits, over a byte string
uint64_t fnv1a(const std::vector<unsigned char>& b) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : b) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

template <class T>
void put_raw(std::vector<unsigned char>& b, const T* v, size_t n) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(v);
  b.insert(b.end(), p, p + sizeof(T) * n);
}

template <class T>
bool get_raw(const std::vector<unsigned char>& b, size_t& pos, T* v, size_t n) {
  if (pos + sizeof(T) * n > b.size()) return false;
  std::memcpy(v, b.data() + pos, sizeof(T) * n);
  pos += sizeof(T) * n;
  return true;
}

}  // namespace

extern "C" {

bsmm_status bsmm_mlp_save(bsmm_mlp_t mlp, const char* path) {
  if (!mlp || !path || !*path) return set_error("NULL model or path"), BSMM_ERR_INVALID;
  std::vector<float> prm(NP);
  bsmm_status st = bsmm_mlp_get_params(mlp, prm.data(), NP);
  if (st != BSMM_OK) return st;
  std::vector<unsigned char> b;
  put_raw(b, kMagic, 8);
  const uint32_t hdr[5] = {kFormatVersion, (uint32_t)BSMM_FEATURE_VERSION, (uint32_t)F, (uint32_t)H, (uint32_t)NP};
  put_raw(b, hdr, 5);
  put_raw(b, prm.data(), NP);
  put_raw(b, mlp->norm.xmu, F);
  put_raw(b, mlp->norm.xsd, F);
  put_raw(b, &mlp->norm.ymu, 1);
  put_raw(b, &mlp->norm.ysd, 1);
  const uint64_t sum = fnv1a(b);
  put_raw(b, &sum, 1);
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return set_error(std::string("cannot write ") + tmp), BSMM_ERR_INVALID;
  const bool ok = std::fwrite(b.data(), 1, b.size(), f) == b.size();
  if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return set_error(std::string("cannot write ") + path), BSMM_ERR_INVALID;
  }
  return BSMM_OK;
}

bsmm_status bsmm_mlp_load(bsmm_mlp_t* out, const char* path) {
  if (!out || !path || !*path) return set_error("NULL output or path"), BSMM_ERR_INVALID;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_error(std::string("cannot open ") + path), BSMM_ERR_INVALID;
  std::vector<unsigned char> b;
  unsigned char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) {
    b.insert(b.end(), buf, buf + n);
    if (b.size() > (1u << 20)) break;  // far larger than any model file
  }
  std::fclose(f);
  if (b.size() < 8 + sizeof(uint64_t) || b.size() > (1u << 20))
    return set_error(std::string("not a cost-model file: ") + path), BSMM_ERR_INVALID;
  uint64_t sum = 0;
  std::memcpy(&sum, b.data() + b.size() - sizeof(uint64_t), sizeof(uint64_t));
  b.resize(b.size() - sizeof(uint64_t));
  if (fnv1a(b) != sum) return set_error(std::string("cost-model file checksum mismatch: ") + path), BSMM_ERR_INVALID;
  size_t pos = 0;
  char magic[8];
  uint32_t hdr[5];
  if (!get_raw(b, pos, magic, 8) || std::memcmp(magic, kMagic, 8) != 0 || !get_raw(b, pos, hdr, 5))
    return set_error(std::string("not a cost-model file: ") + path), BSMM_ERR_INVALID;
  if (hdr[0] != kFormatVersion || hdr[1] != (uint32_t)BSMM_FEATURE_VERSION || hdr[2] != (uint32_t)F ||
      hdr[3] != (uint32_t)H || hdr[4] != (uint32_t)NP)
    return set_error(std::string("cost-model file of another format, feature version or shape: ") + path),
           BSMM_ERR_INVALID;
  std::vector<float> prm(NP);
  Norm nm{};
  if (!get_raw(b, pos, prm.data(), NP) || !get_raw(b, pos, nm.xmu, F) || !get_raw(b, pos, nm.xsd, F) ||
      !get_raw(b, pos, &nm.ymu, 1) || !get_raw(b, pos, &nm.ysd, 1) || pos != b.size())
    return set_error(std::string("truncated cost-model file: ") + path), BSMM_ERR_INVALID;
  bsmm_mlp_t m = nullptr;
  bsmm_status st = bsmm_mlp_create(&m, 0);
  if (st == BSMM_OK) st = bsmm_mlp_set_params(m, prm.data(), NP);
  if (st == BSMM_OK) st = bsmm_mlp_set_norm(m, nm.xmu, nm.xsd, nm.ymu, nm.ysd);
  if (st != BSMM_OK) {
    bsmm_mlp_destroy(m);
    return st;
  }
  *out = m;
  return BSMM_OK;
}

void bsmm_mlp_destroy(bsmm_mlp_t mlp) {
  if (!mlp) return;
  for (DevBuf* b : {&mlp->params, &mlp->m, &mlp->v, &mlp->grad, &mlp->part})
    if (b->p) cudaFree(b->p);
  delete mlp;
}

}  // extern "C"
