// Inference of the warm-start network (64 -> 256 -> 256 -> 256 -> 64, ReLU
// on the hidden layers; BF16 operands, FP32 accumulation) in one persistent
// kernel: a CTA per SM takes 128-row tiles of the input in turn and runs the
// four layers on chip, so the hidden activations never leave shared memory.
//
//   * operands in shared memory in the tensor core's K-major layout with the
//     128-byte swizzle (8-row groups of 1024 bytes), written by TMA tiled
//     loads (cp.async.bulk.tensor, tensor maps with SWIZZLE_128B) for the
//     input and the weights, and by the epilogue's swizzled stores for the
//     activations;
//   * layer 1's weights (256 x 64) stay resident; the 12 weight blocks of
//     layers 2-4 per tile (4 x [256 x 64] of each hidden layer, 4 x [64 x 64]
//     of the output layer) stream through a 3-stage ring from L2, loaded two
//     blocks ahead of the tensor core;
//   * one elected thread issues TMA and tcgen05.mma (M = 128, K = 16 per
//     instruction, the accumulator of up to 256 fp32 columns in tensor
//     memory); tcgen05.commit signals the ring's free slots and the end of a
//     layer; the four warps read their 32 accumulator lanes back
//     (tcgen05.ld), add the bias, apply ReLU, round to BF16 and store the
//     next layer's operand, or write the FP32 output;
//   * the next tile's input is loaded as soon as layer 1 has consumed the
//     current one.
// Every mbarrier wait is bounded: on timeout the kernel records an error,
// waits (bounded) for its copies in flight, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "dm_internal.h"
#include "dm_tc.cuh"

namespace dm {

namespace {

constexpr int kTM = 128;  // rows per tile
constexpr int kThreadsF = 128;
constexpr int kStages = 3;
constexpr int kBlocksPerTile = 12;  // weight blocks streamed per tile
// shared memory map (bytes from a 1024-aligned base)
constexpr int kOffW1 = 0;                       // [256][64] bf16: 32 KB
constexpr int kOffH = kOffW1 + 256 * 128;       // 4 K-blocks of [128][64]: 64 KB
constexpr int kOffX = kOffH + 4 * kTM * 128;    // [128][64]: 16 KB
constexpr int kOffRing = kOffX + kTM * 128;     // 3 x [256][64]: 96 KB
constexpr int kStageBytes = 256 * 128;
constexpr int kOffBar = kOffRing + kStages * kStageBytes;
constexpr int kSmemFused = kOffBar + 128 + 1024;  // barriers, TMEM slot, alignment slack

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

}  // namespace

__global__ void __launch_bounds__(kThreadsF, 1)
    k_mlp_fused(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_w1,
                const __grid_constant__ CUtensorMap tm_w2, const __grid_constant__ CUtensorMap tm_w3,
                const __grid_constant__ CUtensorMap tm_w4, const float *__restrict__ b1,
                const float *__restrict__ b2, const float *__restrict__ b3,
                const float *__restrict__ b4, float *__restrict__ Y, int ntiles, int *err) {
  using namespace tc;
  extern __shared__ char smem_raw[];
  char *smem = reinterpret_cast<char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  char *W1s = smem + kOffW1, *Hs = smem + kOffH, *Xs = smem + kOffX, *Ring = smem + kOffRing;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kOffBar);
  uint64_t *bar_w1 = bar, *bar_x = bar + 1, *bar_mma = bar + 2;
  uint64_t *bar_full = bar + 3, *bar_free = bar + 3 + kStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 3 + 2 * kStages);
  volatile int *fail = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total_blocks = my_tiles * kBlocksPerTile;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 3 + 2 * kStages; ++i) mbar_init(&bar[i], 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  // weight block g of this CTA's stream: layer 2, 3 (blocks of [256][64]) or
  // 4 ([64][64]), K-block g % 4
  auto block_bytes = [](int b) { return b < 8 ? kStageBytes : 64 * 128; };
  int issued = 0;      // weight blocks whose load was issued (thread 0)
  int x_loads = 0;     // input tiles whose load was issued (thread 0)
  bool x_pending = false;
  auto load_block = [&](int g) -> bool {  // thread 0
    const int s = g % kStages, b = g % kBlocksPerTile;
    if (g >= kStages && !mbar_wait(&bar_free[s], (uint32_t)((g / kStages - 1) & 1))) return false;
    mbar_expect_tx(&bar_full[s], (uint32_t)block_bytes(b));
    const void *map = b < 4 ? (const void *)&tm_w2 : (b < 8 ? (const void *)&tm_w3 : (const void *)&tm_w4);
    tma_load_2d(Ring + s * kStageBytes, map, 64 * (b % 4), 0, &bar_full[s]);
    issued = g + 1;
    return true;
  };

  bool ok = true;
  if (tid == 0 && my_tiles > 0) {
    mbar_expect_tx(bar_w1, 256 * 128);
    tma_load_2d(W1s, &tm_w1, 0, 0, bar_w1);
    mbar_expect_tx(bar_x, kTM * 128);
    tma_load_2d(Xs, &tm_x, 0, (int)blockIdx.x * kTM, bar_x);
    x_pending = true;
    x_loads = 1;
    for (int g = 0; g < 2 && g < total_blocks; ++g) ok = ok && load_block(g);
    ok = ok && mbar_wait(bar_w1, 0);
    if (!ok) *fail = 1;
  }
  const uint32_t id256 = make_idesc(kTM, 256), id64 = make_idesc(kTM, 64);
  uint32_t mma_phase = 0;
  const int row = warp * 32 + lane;  // this thread's accumulator lane / tile row
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);

  // all threads: the end of a layer's MMAs (bounded), agreed by the block
  auto layer_done = [&]() -> bool {
    bool w = mbar_wait(bar_mma, mma_phase);
    mma_phase ^= 1u;
    w = __syncthreads_and(w && !*fail) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    return w;
  };
  // epilogue of a hidden layer: accumulator + bias, ReLU, BF16 into H
  auto hidden_epilogue = [&](const float *bias) {
#pragma unroll 1
    for (int c0 = 0; c0 < 256; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(trow + (uint32_t)c0, r);
      uint32_t p[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float v0 = fmaxf(__uint_as_float(r[2 * j]) + __ldg(bias + c0 + 2 * j), 0.0f);
        const float v1 = fmaxf(__uint_as_float(r[2 * j + 1]) + __ldg(bias + c0 + 2 * j + 1), 0.0f);
        p[j] = pack_bf16(v0, v1);
      }
      // K-block c0 / 64, 16-byte chunks (c0 % 64) / 8 and the next, swizzled
      char *rowp = Hs + (c0 >> 6) * (kTM * 128) + row * 128;
      const int ch = (c0 & 63) >> 3;
      *reinterpret_cast<uint4 *>(rowp + ((ch ^ (row & 7)) << 4)) = make_uint4(p[0], p[1], p[2], p[3]);
      *reinterpret_cast<uint4 *>(rowp + (((ch + 1) ^ (row & 7)) << 4)) =
          make_uint4(p[4], p[5], p[6], p[7]);
    }
    // the generic-proxy stores become visible to the tensor core's reads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  };
  // thread 0: the MMAs of a streamed layer (4 weight blocks from g0 on), A
  // the activations in H; the next loads two blocks ahead
  auto streamed_layer = [&](int g0, uint32_t idesc) -> bool {
    for (int b = 0; b < 4; ++b) {
      const int g = g0 + b, s = g % kStages;
      if (!mbar_wait(&bar_full[s], (uint32_t)((g / kStages) & 1))) return false;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(Hs + b * (kTM * 128)), w0 = smem_u32(Ring + s * kStageBytes);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma_bf16(tmem, make_desc(a0 + 32 * kk, 16, 1024, kSwizzle128B),
                 make_desc(w0 + 32 * kk, 16, 1024, kSwizzle128B), idesc, (b | kk) ? 1u : 0u);
      mma_commit(&bar_free[s]);
      if (g + 2 < total_blocks && !load_block(g + 2)) return false;
    }
    mma_commit(bar_mma);
    return true;
  };

  for (int i = 0; i < my_tiles && ok; ++i) {
    const int tile = (int)blockIdx.x + i * (int)gridDim.x;
    const int g0 = i * kBlocksPerTile;
    // layer 1: A = the input tile, B = the resident weights
    if (tid == 0 && !*fail) {
      if (mbar_wait(bar_x, (uint32_t)(i & 1))) {
        x_pending = false;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = smem_u32(Xs), w0 = smem_u32(W1s);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(tmem, make_desc(a0 + 32 * kk, 16, 1024, kSwizzle128B),
                   make_desc(w0 + 32 * kk, 16, 1024, kSwizzle128B), id256, kk ? 1u : 0u);
        mma_commit(bar_mma);
      } else {
        *fail = 1;
      }
    }
    if (!(ok = layer_done())) break;
    if (tid == 0 && i + 1 < my_tiles) {  // the input buffer is free: next tile's input
      mbar_expect_tx(bar_x, kTM * 128);
      tma_load_2d(Xs, &tm_x, 0, (tile + (int)gridDim.x) * kTM, bar_x);
      x_pending = true;
      ++x_loads;
    }
    hidden_epilogue(b1);
    // layers 2 and 3: A = H, B = streamed blocks
    for (int l = 0; l < 2 && ok; ++l) {
      if (tid == 0 && !*fail && !streamed_layer(g0 + 4 * l, id256)) *fail = 1;
      if (!(ok = layer_done())) break;
      hidden_epilogue(l == 0 ? b2 : b3);
    }
    if (!ok) break;
    // layer 4 (N = 64): FP32 output rows
    if (tid == 0 && !*fail && !streamed_layer(g0 + 8, id64)) *fail = 1;
    if (!(ok = layer_done())) break;
    float *yrow = Y + ((size_t)tile * kTM + row) * 64;
#pragma unroll 1
    for (int c0 = 0; c0 < 64; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(trow + (uint32_t)c0, r);
      float4 *o = reinterpret_cast<float4 *>(yrow + c0);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        o[j] = make_float4(__uint_as_float(r[4 * j]) + __ldg(b4 + c0 + 4 * j),
                           __uint_as_float(r[4 * j + 1]) + __ldg(b4 + c0 + 4 * j + 1),
                           __uint_as_float(r[4 * j + 2]) + __ldg(b4 + c0 + 4 * j + 2),
                           __uint_as_float(r[4 * j + 3]) + __ldg(b4 + c0 + 4 * j + 3));
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // the accumulator is read before the next tile's layer 1
  }
  if (!ok || *fail) {
    if (tid == 0) {
      atomicExch(err, 1);
      // copies in flight land before the CTA leaves (bounded)
      for (int g = (int)(issued > 3 ? issued - 3 : 0); g < issued; ++g)
        mbar_wait(&bar_full[g % kStages], (uint32_t)((g / kStages) & 1));
      if (x_pending) mbar_wait(bar_x, (uint32_t)((x_loads - 1) & 1));
      // every MMA issued so far is done before the tensor memory is freed
      mma_commit(bar_mma);
      mbar_wait(bar_mma, mma_phase);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Row-major [rows][cols] bf16 matrix, boxes of 64 columns x box_rows rows,
// 128-byte swizzle.
bool encode(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {64, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Y [M][64] fp32 = the network on X [M][64] bf16; W[l] the bf16 weights
// [out][in] (256 x 64, 256 x 256, 256 x 256, 64 x 256), b[l] the fp32
// biases.  M % 128 == 0, every pointer 16-byte aligned.  err: device int set
// to 1 on a barrier timeout.
cudaError_t launch_mlp_fused(int M, const void *X, const void *const W[4], const float *const b[4],
                             float *Y, int *err, cudaStream_t st) {
  static int sms = 0;
  static bool attr = false;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFused);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  CUtensorMap tx, t1, t2, t3, t4;
  if (!encode(&tx, X, (uint64_t)M, 64, kTM) || !encode(&t1, W[0], 256, 64, 256) ||
      !encode(&t2, W[1], 256, 256, 256) || !encode(&t3, W[2], 256, 256, 256) ||
      !encode(&t4, W[3], 64, 256, 64))
    return cudaErrorInvalidValue;
  const int ntiles = M / kTM;
  const int grid = ntiles < sms ? ntiles : sms;
  if (grid == 0) return cudaSuccess;
  k_mlp_fused<<<grid, kThreadsF, kSmemFused, st>>>(tx, t1, t2, t3, t4, b[0], b[1], b[2], b[3], Y,
                                                     ntiles, err);
  return cudaGetLastError();
}

}  // namespace dm
