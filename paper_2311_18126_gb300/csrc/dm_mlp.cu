// Warm-start network: a 4-layer MLP (in -> 256 -> 256 -> 256 -> out) in BF16
// with FP32 accumulation on the tcgen05 tensor cores (dm_gemm.cu), FP32
// master weights and Adam.  No counterpart in the paper: it predicts the
// Newton initial guess of the implicit step from recent states; Newton still
// runs to the same residual.
//
// Shapes: the input width is padded to 64 and the output width to 64 so that
// every GEMM has K % 64 == 0 and N % 16 == 0; padded weight rows/columns are
// zero and stay zero (their gradients are masked).
#include <cuda_bf16.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "dm_internal.h"

namespace dm {
cudaError_t launch_mlp_fused(int M, const void *X, const void *const W[4], const float *const b[4],
                             float *Y, int *err, cudaStream_t st);
cudaError_t launch_gemm_bf16(int M, int N, int K, const void *A, const void *B, const float *bias,
                             void *C, int relu, int out_f32, int *err, cudaStream_t st,
                             int ksplit = 1, float *work = nullptr);
}

using namespace dm;

namespace {

constexpr int kIn = 64, kHid = 256, kOut = 64, kLayers = 4;
const int kDin[kLayers] = {kIn, kHid, kHid, kHid};
const int kDout[kLayers] = {kHid, kHid, kHid, kOut};

__device__ __forceinline__ uint16_t f2bf(float x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t *>(&b);
}
__device__ __forceinline__ float bf2f(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }

__global__ void k_to_bf16(int n, const float *src, uint16_t *dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = f2bf(src[i]);
}
// dst[c][r] = src[r][c] for a rows x cols bf16 matrix
__global__ void k_transpose_bf16(int rows, int cols, const uint16_t *src, uint16_t *dst) {
  __shared__ uint16_t tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j, c = c0 + threadIdx.x;
    tile[j][threadIdx.x] = (r < rows && c < cols) ? src[(size_t)r * cols + c] : 0;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[(size_t)c * rows + r] = tile[threadIdx.x][j];
  }
}
// dst[c][r] = src[r][c] for fp32 (weight gradient back to [out][in])
__global__ void k_transpose_f32(int rows, int cols, const float *src, float *dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i / cols, c = i - r * cols;
  dst[(size_t)c * rows + r] = src[i];
}
// MSE loss on the first n_valid output columns: dY = 2 (pred - y) / (M n_valid),
// padded columns get 0; loss partial sums per block.
__global__ void k_mse(int M, int n_valid, const float *pred, const float *y, uint16_t *dY,
                      float *dY32, double *loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < M * kOut) {
    const int r = i / kOut, c = i - r * kOut;
    float g = 0.0f;
    if (c < n_valid) {
      const float d = pred[i] - y[(size_t)r * n_valid + c];
      l = (double)d * d;
      g = 2.0f * d / (float)(M * n_valid);
    }
    dY[i] = f2bf(g);
    dY32[i] = g;
  }
  // block reduction, one atomic per block
  __shared__ double red[256];
  red[threadIdx.x] = l;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / (double)(M * n_valid));
}
// gradient through ReLU: dH *= (H > 0), bf16 in place; fp32 copy for bias
__global__ void k_relu_back(int n, const uint16_t *H, uint16_t *dH, float *dH32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = bf2f(H[i]) > 0.0f ? bf2f(dH[i]) : 0.0f;
  dH[i] = f2bf(g);
  dH32[i] = g;
}
// bias gradient: column sums of an M x N fp32 matrix (one thread per column,
// fixed summation order)
// Column sums of G [M][N] in two passes with a fixed summation order:
// k_colsum_part gives block (x, y) columns 32x.. and rows y, y + R, ...
// (R = gridDim.y * 8), 8 row lanes per column, partials [gridDim.y][N];
// k_colsum_final adds the partials.
constexpr int kColChunks = 64;
__global__ void k_colsum_part(int M, int N, const float *G, float *part) {
  __shared__ float red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int stride = gridDim.y * 8;
  float s = 0.0f;
  if (c < N)
    for (int r = blockIdx.y * 8 + threadIdx.y; r < M; r += stride) s += G[(size_t)r * N + c];
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < N) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
    part[(size_t)blockIdx.y * N + c] = t;
  }
}
__global__ void k_colsum_final(int N, int chunks, const float *part, float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.0f;
  for (int z = 0; z < chunks; ++z) s += part[(size_t)z * N + c];
  out[c] = s;
}
// Adam on FP32 master parameters; mask zeroes the padded entries
__global__ void k_adam(int n, float *p, const float *g, float *m, float *v, const float *mask,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i] * (mask ? mask[i] : 1.0f);
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  if (mask) p[i] *= mask[i];
}

inline int nb(int64_t n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

struct dm_mlp {
  int in_dim = 0, out_dim = 0;
  cudaStream_t stream = nullptr;
  // per layer: fp32 master W [out][in], b [out], Adam m/v, bf16 W and W^T
  float *W[kLayers] = {}, *b[kLayers] = {}, *mW[kLayers] = {}, *vW[kLayers] = {},
        *mb[kLayers] = {}, *vb[kLayers] = {}, *gW[kLayers] = {}, *gWt[kLayers] = {},
        *gb[kLayers] = {}, *maskW[kLayers] = {}, *maskb[kLayers] = {};
  uint16_t *Wh[kLayers] = {}, *Wth[kLayers] = {};
  // activations for a batch of up to cap rows
  int cap = 0;
  uint16_t *act[kLayers + 1] = {};  // act[0] = input X (not owned), act[l+1] layer l out
  uint16_t *actT = nullptr, *dA = nullptr, *dAT = nullptr, *dA2 = nullptr;
  float *out32 = nullptr, *dY32 = nullptr, *d32 = nullptr;
  float *splitws = nullptr;  // split-K partial weight gradients [kMaxSplit][256][256]
  double *loss = nullptr;
  bool fused = true;  // inference: the fused 4-layer kernel (else a GEMM per layer)
  int *err = nullptr;
  int64_t step = 0;
  std::vector<void *> allocs;
};

namespace {

template <class T>
dm_status mlp_alloc(dm_mlp *m, T **p, size_t n) {
  void *v = nullptr;
  if (cudaMalloc(&v, n * sizeof(T) + 16) != cudaSuccess) {
    set_error("dm_mlp: cudaMalloc failed");
    return DM_ERR_OOM;
  }
  cudaMemset(v, 0, n * sizeof(T) + 16);
  m->allocs.push_back(v);
  *p = (T *)v;
  return DM_OK;
}

// K chunks of the weight-gradient GEMMs for a batch of M rows: up to
// kMaxSplit chunks of at least two 64-column blocks, dividing M exactly.
constexpr int kMaxSplit = 128;
int split_for(int M) {
  int ks = 1;
  while (ks < kMaxSplit && M % (2 * ks * 128) == 0) ks *= 2;
  return ks;
}

dm_status ensure_batch(dm_mlp *m, int M) {
  if (!m->splitws &&
      cudaMalloc(&m->splitws, (size_t)kMaxSplit * kHid * kHid * sizeof(float)) != cudaSuccess)
    return DM_ERR_OOM;
  if (M <= m->cap) return DM_OK;
  for (int l = 1; l <= kLayers; ++l) {
    if (m->act[l]) {
      cudaFree(m->act[l]);
    }
  }
  auto fr = [](void *p) { if (p) cudaFree(p); };
  fr(m->actT); fr(m->dA); fr(m->dAT); fr(m->dA2); fr(m->out32); fr(m->dY32); fr(m->d32);
  size_t w = (size_t)M * kHid;
  for (int l = 1; l <= kLayers; ++l)
    if (cudaMalloc(&m->act[l], w * 2) != cudaSuccess) return DM_ERR_OOM;
  if (cudaMalloc(&m->actT, w * 2) || cudaMalloc(&m->dA, w * 2) || cudaMalloc(&m->dAT, w * 2) ||
      cudaMalloc(&m->dA2, w * 2) || cudaMalloc(&m->out32, (size_t)M * kOut * 4) ||
      cudaMalloc(&m->dY32, (size_t)M * kOut * 4) || cudaMalloc(&m->d32, w * 4))
    return DM_ERR_OOM;
  m->cap = M;
  return DM_OK;
}

void refresh_bf16(dm_mlp *m) {
  for (int l = 0; l < kLayers; ++l) {
    const int n = kDout[l] * kDin[l];
    k_to_bf16<<<nb(n, 256), 256, 0, m->stream>>>(n, m->W[l], m->Wh[l]);
    dim3 blk(32, 8), grd(nb(kDin[l], 32), nb(kDout[l], 32));
    k_transpose_bf16<<<grd, blk, 0, m->stream>>>(kDout[l], kDin[l], m->Wh[l], m->Wth[l]);
  }
}

// Inference into Y (NULL: the network's own output buffer): the fused
// kernel, or the per-layer GEMMs followed by a copy to Y.
cudaError_t infer(dm_mlp *m, const uint16_t *X, int M, float *Y = nullptr);

cudaError_t forward(dm_mlp *m, const uint16_t *X, int M) {
  m->act[0] = const_cast<uint16_t *>(X);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
    const bool last = l == kLayers - 1;
    e = launch_gemm_bf16(M, kDout[l], kDin[l], m->act[l], m->Wh[l], m->b[l],
                         last ? (void *)m->out32 : (void *)m->act[l + 1], last ? 0 : 1,
                         last ? 1 : 0, m->err, m->stream);
  }
  return e;
}

cudaError_t infer(dm_mlp *m, const uint16_t *X, int M, float *Y) {
  if (!m->fused) {
    cudaError_t e = forward(m, X, M);
    if (e == cudaSuccess && Y)
      e = cudaMemcpyAsync(Y, m->out32, (size_t)M * kOut * 4, cudaMemcpyDeviceToDevice, m->stream);
    return e;
  }
  const void *W[kLayers] = {m->Wh[0], m->Wh[1], m->Wh[2], m->Wh[3]};
  const float *b[kLayers] = {m->b[0], m->b[1], m->b[2], m->b[3]};
  return launch_mlp_fused(M, X, W, b, Y ? Y : m->out32, m->err, m->stream);
}

}  // namespace

namespace dm {
// Forward pass on `st` without synchronisation (used inside dm_step);
// returns the fp32 output [M][64] (owned by the network) or nullptr.
float *mlp_forward_async(dm_mlp *m, const void *X, int M, cudaStream_t st, int *err) {
  if (!m || M <= 0 || M % 128) return nullptr;
  if (ensure_batch(m, M) != DM_OK) return nullptr;
  cudaStream_t keep = m->stream;
  int *keep_err = m->err;
  m->stream = st;
  m->err = err;
  const cudaError_t e = infer(m, (const uint16_t *)X, M);
  m->stream = keep;
  m->err = keep_err;
  return e == cudaSuccess ? m->out32 : nullptr;
}
}  // namespace dm

extern "C" {

dm_status dm_mlp_create(int32_t in_dim, int32_t out_dim, uint64_t seed, void *stream,
                        dm_mlp **out) {
  if (!out || in_dim < 1 || in_dim > kIn || out_dim < 1 || out_dim > kOut) {
    set_error("dm_mlp_create: in_dim in [1, 64], out_dim in [1, 64]");
    return DM_ERR_INVALID_ARG;
  }
  dm_mlp *m = new dm_mlp();
  m->in_dim = in_dim;
  m->out_dim = out_dim;
  m->stream = (cudaStream_t)stream;
  std::mt19937_64 rng(seed);
  dm_status st = DM_OK;
  for (int l = 0; l < kLayers && st == DM_OK; ++l) {
    const int fo = kDout[l], fi = kDin[l];
    const int vi = l == 0 ? in_dim : fi, vo = l == kLayers - 1 ? out_dim : fo;
    std::vector<float> W(fo * fi, 0.0f), b(fo, 0.0f), mw(fo * fi, 0.0f), mb(fo, 0.0f);
    // He-uniform initialisation on the valid block
    const float lim = std::sqrt(6.0f / (float)vi) * (l == kLayers - 1 ? 0.1f : 1.0f);
    std::uniform_real_distribution<float> U(-lim, lim);
    for (int o = 0; o < vo; ++o) {
      for (int i = 0; i < vi; ++i) {
        W[o * fi + i] = U(rng);
        mw[o * fi + i] = 1.0f;
      }
      mb[o] = 1.0f;
    }
    for (auto *p : {&m->W[l], &m->mW[l], &m->vW[l], &m->gW[l], &m->gWt[l], &m->maskW[l]})
      if (st == DM_OK) st = mlp_alloc(m, p, (size_t)fo * fi);
    for (auto *p : {&m->b[l], &m->mb[l], &m->vb[l], &m->gb[l], &m->maskb[l]})
      if (st == DM_OK) st = mlp_alloc(m, p, (size_t)fo);
    if (st == DM_OK) st = mlp_alloc(m, &m->Wh[l], (size_t)fo * fi);
    if (st == DM_OK) st = mlp_alloc(m, &m->Wth[l], (size_t)fo * fi);
    if (st == DM_OK) {
      cudaMemcpy(m->W[l], W.data(), W.size() * 4, cudaMemcpyHostToDevice);
      cudaMemcpy(m->b[l], b.data(), b.size() * 4, cudaMemcpyHostToDevice);
      cudaMemcpy(m->maskW[l], mw.data(), mw.size() * 4, cudaMemcpyHostToDevice);
      cudaMemcpy(m->maskb[l], mb.data(), mb.size() * 4, cudaMemcpyHostToDevice);
    }
  }
  if (st == DM_OK) st = mlp_alloc(m, &m->loss, 1);
  if (st == DM_OK) st = mlp_alloc(m, &m->err, 1);
  if (st != DM_OK) {
    dm_mlp_destroy(m);
    return st;
  }
  refresh_bf16(m);
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
    set_error("dm_mlp_create: CUDA error");
    dm_mlp_destroy(m);
    return DM_ERR_CUDA;
  }
  *out = m;
  return DM_OK;
}

void dm_mlp_destroy(dm_mlp *m) {
  if (!m) return;
  for (void *p : m->allocs) cudaFree(p);
  for (int l = 1; l <= kLayers; ++l)
    if (m->act[l]) cudaFree(m->act[l]);
  for (void *p : {(void *)m->actT, (void *)m->dA, (void *)m->dAT, (void *)m->dA2,
                  (void *)m->out32, (void *)m->dY32, (void *)m->d32, (void *)m->splitws})
    if (p) cudaFree(p);
  delete m;
}

// Parameters as one fp32 host array: for each layer W [out][in] then b [out]
// (padded shapes: 256x64, 256x256, 256x256, 64x256).
int64_t dm_mlp_num_params(void) {
  int64_t n = 0;
  for (int l = 0; l < kLayers; ++l) n += (int64_t)kDout[l] * kDin[l] + kDout[l];
  return n;
}

dm_status dm_mlp_get_params(dm_mlp *m, float *host) {
  if (!m || !host) return DM_ERR_INVALID_ARG;
  cudaStreamSynchronize(m->stream);
  int64_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    cudaMemcpy(host + o, m->W[l], (size_t)kDout[l] * kDin[l] * 4, cudaMemcpyDeviceToHost);
    o += (int64_t)kDout[l] * kDin[l];
    cudaMemcpy(host + o, m->b[l], (size_t)kDout[l] * 4, cudaMemcpyDeviceToHost);
    o += kDout[l];
  }
  return cudaGetLastError() == cudaSuccess ? DM_OK : DM_ERR_CUDA;
}

dm_status dm_mlp_set_params(dm_mlp *m, const float *host) {
  if (!m || !host) return DM_ERR_INVALID_ARG;
  cudaStreamSynchronize(m->stream);
  int64_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    cudaMemcpy(m->W[l], host + o, (size_t)kDout[l] * kDin[l] * 4, cudaMemcpyHostToDevice);
    o += (int64_t)kDout[l] * kDin[l];
    cudaMemcpy(m->b[l], host + o, (size_t)kDout[l] * 4, cudaMemcpyHostToDevice);
    o += kDout[l];
  }
  refresh_bf16(m);
  return cudaStreamSynchronize(m->stream) == cudaSuccess ? DM_OK : DM_ERR_CUDA;
}

dm_status dm_mlp_set_fused(dm_mlp *m, int32_t enable) {
  if (!m) {
    set_error("dm_mlp_set_fused: NULL network");
    return DM_ERR_INVALID_ARG;
  }
  m->fused = enable != 0;
  return DM_OK;
}

// Forward pass: X [M][64] bf16 (device) -> Y [M][64] fp32 (device).
dm_status dm_mlp_forward_async(dm_mlp *m, const void *X, float *Y, int32_t M) {
  if (!m || !X || !Y || M <= 0 || M % 128) {
    set_error("dm_mlp_forward: M must be a positive multiple of 128");
    return DM_ERR_INVALID_ARG;
  }
  // the per-layer path keeps every layer's activations
  if (!m->fused && ensure_batch(m, M) != DM_OK) return DM_ERR_OOM;
  if (infer(m, (const uint16_t *)X, M, Y) != cudaSuccess) {
    set_error("dm_mlp_forward: launch failed");
    return DM_ERR_CUDA;
  }
  return DM_OK;
}

dm_status dm_mlp_check(dm_mlp *m) {
  if (!m) {
    set_error("dm_mlp_check: NULL network");
    return DM_ERR_INVALID_ARG;
  }
  int h = 0;
  cudaMemcpyAsync(&h, m->err, 4, cudaMemcpyDeviceToHost, m->stream);
  const bool ok = cudaStreamSynchronize(m->stream) == cudaSuccess && !h;
  cudaMemsetAsync(m->err, 0, 4, m->stream);
  if (!ok) {
    set_error("dm_mlp: CUDA error or tensor-core barrier timeout");
    return DM_ERR_CUDA;
  }
  return DM_OK;
}

dm_status dm_mlp_forward(dm_mlp *m, const void *X, float *Y, int32_t M) {
  dm_status st = dm_mlp_forward_async(m, X, Y, M);
  if (st != DM_OK) return st;
  return dm_mlp_check(m);
}

// One training step on a minibatch: forward, MSE loss on the first out_dim
// columns of the fp32 targets Y [M][out_dim], backward (tensor-core GEMMs
// for the weight and input gradients), Adam.  grads_out (device, optional)
// receives the fp32 gradients in the dm_mlp_get_params layout; loss_out the
// loss before the update.
dm_status dm_mlp_train_step(dm_mlp *m, const void *X, const float *Y, int32_t M, float lr,
                            float *grads_out, double *loss_out) {
  if (!m || !X || !Y || M <= 0 || M % 128) {
    set_error("dm_mlp_train_step: M must be a positive multiple of 128");
    return DM_ERR_INVALID_ARG;
  }
  if (ensure_batch(m, M) != DM_OK) return DM_ERR_OOM;
  cudaStream_t st = m->stream;
  cudaMemsetAsync(m->err, 0, 4, st);
  cudaMemsetAsync(m->loss, 0, 8, st);
  if (forward(m, (const uint16_t *)X, M) != cudaSuccess) return DM_ERR_CUDA;
  // output gradient (bf16 for the GEMMs, fp32 for the bias)
  uint16_t *dY = m->dA;
  k_mse<<<nb((int64_t)M * kOut, 256), 256, 0, st>>>(M, m->out_dim, m->out32, Y, dY, m->dY32,
                                                     m->loss);
  int width = kOut;
  uint16_t *dcur = dY;
  float *dcur32 = m->dY32;
  for (int l = kLayers - 1; l >= 0; --l) {
    const int fo = kDout[l], fi = kDin[l];
    // weight gradient dW [fo][fi] = dY^T [fo][M] * A_in [M][fi]: the GEMM
    // reduces over the batch; its row count must be a multiple of 128, so
    // the narrow output layer computes dW^T = A_in^T dY and transposes it
    dim3 blk(32, 8);
    k_transpose_bf16<<<dim3(nb(fi, 32), nb(M, 32)), blk, 0, st>>>(M, fi, m->act[l], m->actT);
    k_transpose_bf16<<<dim3(nb(fo, 32), nb(M, 32)), blk, 0, st>>>(M, fo, dcur, m->dAT);
    // the batch reduction is split over K chunks so that the tiny M x N
    // tile grid (two row tiles) still fills the GPU
    const int ks = split_for(M);
    if (fo % 128 == 0) {
      if (launch_gemm_bf16(fo, fi, M, m->dAT, m->actT, nullptr, m->gW[l], 0, 1, m->err, st, ks,
                           m->splitws))
        return DM_ERR_CUDA;
    } else {
      if (launch_gemm_bf16(fi, fo, M, m->actT, m->dAT, nullptr, m->gWt[l], 0, 1, m->err, st, ks,
                           m->splitws))
        return DM_ERR_CUDA;
      k_transpose_f32<<<nb(fi * fo, 256), 256, 0, st>>>(fi, fo, m->gWt[l], m->gW[l]);
    }
    // bias gradient (partials in the split-K workspace, free again here)
    k_colsum_part<<<dim3(nb(fo, 32), kColChunks), dim3(32, 8), 0, st>>>(M, fo, dcur32,
                                                                       m->splitws);
    k_colsum_final<<<nb(fo, 128), 128, 0, st>>>(fo, kColChunks, m->splitws, m->gb[l]);
    if (l > 0) {
      // dA_in [M][fi] = dY [M][fo] * W^T: B = W^T as [fi][fo]
      uint16_t *dnext = (dcur == m->dA) ? m->dA2 : m->dA;
      if (launch_gemm_bf16(M, fi, fo, dcur, m->Wth[l], nullptr, dnext, 0, 0, m->err, st))
        return DM_ERR_CUDA;
      k_relu_back<<<nb((int64_t)M * fi, 256), 256, 0, st>>>(M * fi, m->act[l], dnext, m->d32);
      dcur = dnext;
      dcur32 = m->d32;
    }
    width = fi;
  }
  (void)width;
  if (grads_out) {
    int64_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
      cudaMemcpyAsync(grads_out + o, m->gW[l], (size_t)kDout[l] * kDin[l] * 4,
                      cudaMemcpyDeviceToDevice, st);
      o += (int64_t)kDout[l] * kDin[l];
      cudaMemcpyAsync(grads_out + o, m->gb[l], (size_t)kDout[l] * 4, cudaMemcpyDeviceToDevice, st);
      o += kDout[l];
    }
  }
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)m->step), c2 = 1.0f - std::pow(b2, (float)m->step);
  if (lr > 0.0f) {
    for (int l = 0; l < kLayers; ++l) {
      const int n = kDout[l] * kDin[l];
      k_adam<<<nb(n, 256), 256, 0, st>>>(n, m->W[l], m->gW[l], m->mW[l], m->vW[l], m->maskW[l],
                                          lr, b1, b2, 1e-8f, c1, c2);
      k_adam<<<nb(kDout[l], 256), 256, 0, st>>>(kDout[l], m->b[l], m->gb[l], m->mb[l], m->vb[l],
                                                 m->maskb[l], lr, b1, b2, 1e-8f, c1, c2);
    }
    refresh_bf16(m);
  }
  int h = 0;
  double loss = 0.0;
  cudaMemcpyAsync(&h, m->err, 4, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&loss, m->loss, 8, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || h) {
    set_error("dm_mlp_train_step: CUDA error or tensor-core barrier timeout");
    return DM_ERR_CUDA;
  }
  if (loss_out) *loss_out = loss;
  return DM_OK;
}

}  // extern "C"
