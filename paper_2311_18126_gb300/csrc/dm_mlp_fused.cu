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
//   * the output layer's weights (64 x 256) stay resident; the 9 weight
//     blocks of layers 1-3 per tile ([256 x 64] each: layer 1's, then four
//     K-blocks of each hidden layer) stream through a 3-stage ring from L2,
//     loaded two blocks ahead of the tensor core;
//   * warp 0 issues TMA and tcgen05.mma (M = 128, K = 16 per instruction;
//     lane 0 issues, the whole warp takes the waits, so no lane of it spins
//     while lane 0 has work); the hidden layers accumulate into 256 fp32
//     columns of tensor memory, the output layer into 64 others;
//     tcgen05.commit signals the ring's free slots and the end of a layer;
//   * eight warps read the accumulator back (tcgen05.ld; warp w the lanes
//     32 (w % 4).. and half w / 4 of the columns, all loads before one
//     wait), add the bias, apply ReLU, round to BF16 and store the next
//     layer's operand with the swizzle, or write the FP32 output;
//   * the next tile's input is loaded as soon as layer 1 has consumed the
//     current one, and its layer 1 runs while the output of the current one
//     is written.
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
constexpr int kThreadsF = 256;  // 8 warps: warp w reads lanes 32 (w % 4).., columns half w / 4
constexpr int kStages = 3;
constexpr int kBlocksPerTile = 9;  // streamed weight blocks per tile: W1, 4 of W2, 4 of W3
// shared memory map (bytes from a 1024-aligned base)
constexpr int kOffW4 = 0;                       // 4 K-blocks of [64][64] bf16: 32 KB
constexpr int kOffH = kOffW4 + 4 * 64 * 128;    // 4 K-blocks of [128][64]: 64 KB
constexpr int kOffX = kOffH + 4 * kTM * 128;    // [128][64]: 16 KB
constexpr int kOffRing = kOffX + kTM * 128;     // 3 x [256][64]: 96 KB
constexpr int kStageBytes = 256 * 128;
constexpr int kOffBias = kOffRing + kStages * kStageBytes;  // fp32 biases: 3 x 256 + 64
constexpr int kOffBar = kOffBias + (3 * 256 + 64) * 4;
constexpr int kSmemFused = kOffBar + 128 + 1024;  // barriers, TMEM slot, alignment slack
constexpr uint32_t kTmemCols = 512;  // hidden accumulator at 0, output accumulator at 256

constexpr unsigned kFullMask = 0xffffffffu;

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
  char *W4s = smem + kOffW4, *Hs = smem + kOffH, *Xs = smem + kOffX, *Ring = smem + kOffRing;
  float *sbias = reinterpret_cast<float *>(smem + kOffBias);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kOffBar);
  uint64_t *bar_w4 = bar, *bar_x = bar + 1, *bar_mma = bar + 2;
  uint64_t *bar_full = bar + 3, *bar_free = bar + 3 + kStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 3 + 2 * kStages);
  volatile int *fail = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total_blocks = my_tiles * kBlocksPerTile;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 3 + 2 * kStages; ++i) mbar_init(&bar[i], 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  for (int i = tid; i < 3 * 256 + 64; i += kThreadsF)
    sbias[i] = i < 256 ? b1[i] : (i < 512 ? b2[i - 256] : (i < 768 ? b3[i - 512] : b4[i - 768]));
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot, tmem_out = tmem + 256;

  // Warp 0 issues the copies and the MMAs: it runs the issue path as a
  // whole (every lane takes the same waits, lane 0 issues), so that no lane
  // of it spins on a barrier while lane 0 has work to do.
  int issued = 0;      // weight blocks whose load was issued (warp 0)
  int x_loads = 0;     // input tiles whose load was issued (warp 0)
  bool x_pending = false;
  // weight block g of this CTA's stream: W1 (g % 9 == 0), else K-block
  // (g % 9 - 1) % 4 of W2 (g % 9 <= 4) or W3
  auto load_block = [&](int g) -> bool {  // warp 0
    const int s = g % kStages, b = g % kBlocksPerTile;
    bool w = true;
    if (g >= kStages) w = mbar_wait(&bar_free[s], (uint32_t)((g / kStages - 1) & 1));
    if (!__all_sync(kFullMask, w)) return false;
    if (lane == 0) {
      mbar_expect_tx(&bar_full[s], (uint32_t)kStageBytes);
      const void *map = b == 0 ? (const void *)&tm_w1 : (b <= 4 ? (const void *)&tm_w2 : (const void *)&tm_w3);
      tma_load_2d(Ring + s * kStageBytes, map, b == 0 ? 0 : 64 * ((b - 1) % 4), 0, &bar_full[s]);
    }
    __syncwarp();
    issued = g + 1;
    return true;
  };
  // warp 0: the MMAs of weight blocks g0 .. g0 + nb - 1 from the ring into
  // the hidden accumulator, A = the input tile (layer 1) or the activations
  // in H; the next loads two blocks ahead; then the layer's commit
  auto ring_layer = [&](int g0, int nb, bool from_x) -> bool {
    for (int b = 0; b < nb; ++b) {
      const int g = g0 + b, s = g % kStages;
      if (!__all_sync(kFullMask, mbar_wait(&bar_full[s], (uint32_t)((g / kStages) & 1))))
        return false;
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (lane == 0) {
        const uint32_t a0 = smem_u32(from_x ? Xs : Hs + b * (kTM * 128));
        const uint32_t w0 = smem_u32(Ring + s * kStageBytes);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(tmem, make_desc(a0 + 32 * kk, 16, 1024, kSwizzle128B),
                   make_desc(w0 + 32 * kk, 16, 1024, kSwizzle128B), make_idesc(kTM, 256),
                   (b | kk) ? 1u : 0u);
        mma_commit(&bar_free[s]);
      }
      __syncwarp();
      if (g + 2 < total_blocks && !load_block(g + 2)) return false;
    }
    if (lane == 0) mma_commit(bar_mma);
    __syncwarp();
    return true;
  };
  // warp 0: layer 1 of local tile i (its input and W1 block must land)
  auto issue_layer1 = [&](int i) -> bool {
    if (!__all_sync(kFullMask, mbar_wait(bar_x, (uint32_t)(i & 1)))) return false;
    x_pending = false;
    return ring_layer(i * kBlocksPerTile, 1, true);
  };

  if (warp == 0 && my_tiles > 0) {
    if (lane == 0) {
      mbar_expect_tx(bar_w4, 4 * 64 * 128);
      for (int kb = 0; kb < 4; ++kb) tma_load_2d(W4s + kb * 64 * 128, &tm_w4, 64 * kb, 0, bar_w4);
      mbar_expect_tx(bar_x, kTM * 128);
      tma_load_2d(Xs, &tm_x, 0, (int)blockIdx.x * kTM, bar_x);
    }
    __syncwarp();
    x_pending = true;
    x_loads = 1;
    bool w = true;
    for (int g = 0; g < 2 && g < total_blocks; ++g) w = w && load_block(g);
    w = w && __all_sync(kFullMask, mbar_wait(bar_w4, 0));
    w = w && issue_layer1(0);
    if (!w && lane == 0) *fail = 1;
  }
  __syncthreads();
  bool ok = !*fail;
  uint32_t mma_phase = 0;
  const int quarter = warp & 3, half = warp >> 2;
  const int row = quarter * 32 + lane;  // this thread's accumulator lane / tile row
  const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;

  // all threads: the end of a layer's MMAs (bounded), agreed by the block
  auto layer_done = [&]() -> bool {
    bool w = mbar_wait(bar_mma, mma_phase);
    mma_phase ^= 1u;
    w = __syncthreads_and(w && !*fail) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    return w;
  };
  // epilogue of a hidden layer: accumulator + bias, ReLU, BF16 into H; the
  // thread's row, columns [128 half, 128 half + 128) (eight loads from
  // tensor memory, one wait)
  auto hidden_epilogue = [&](const float *bias) {
    const int cb = 128 * half;
    uint32_t r[128];
#pragma unroll
    for (int q = 0; q < 8; ++q) tmem_ld16_nowait(tmem + lane_off + (uint32_t)(cb + 16 * q), r + 16 * q);
    tmem_wait();
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
      // K-block (cb + 64 kb) / 64 of H, this row's eight 16-byte chunks, swizzled
      char *rowp = Hs + ((cb >> 6) + kb) * (kTM * 128) + row * 128;
#pragma unroll
      for (int ch = 0; ch < 8; ++ch) {
        const int c = 64 * kb + 8 * ch;
        const float4 bl = *reinterpret_cast<const float4 *>(bias + cb + c);
        const float4 bh = *reinterpret_cast<const float4 *>(bias + cb + c + 4);
        const float *a = reinterpret_cast<const float *>(r + c);
        const uint32_t p0 = pack_bf16(fmaxf(a[0] + bl.x, 0.0f), fmaxf(a[1] + bl.y, 0.0f));
        const uint32_t p1 = pack_bf16(fmaxf(a[2] + bl.z, 0.0f), fmaxf(a[3] + bl.w, 0.0f));
        const uint32_t p2 = pack_bf16(fmaxf(a[4] + bh.x, 0.0f), fmaxf(a[5] + bh.y, 0.0f));
        const uint32_t p3 = pack_bf16(fmaxf(a[6] + bh.z, 0.0f), fmaxf(a[7] + bh.w, 0.0f));
        *reinterpret_cast<uint4 *>(rowp + ((ch ^ (row & 7)) << 4)) = make_uint4(p0, p1, p2, p3);
      }
    }
    // the generic-proxy stores become visible to the tensor core's reads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  };

  for (int i = 0; i < my_tiles && ok; ++i) {
    const int tile = (int)blockIdx.x + i * (int)gridDim.x;
    const int g0 = i * kBlocksPerTile;
    // layer 1 was issued before (the prologue, or the previous tile)
    if (!(ok = layer_done())) break;
    if (warp == 0 && i + 1 < my_tiles) {  // the input buffer is free: next tile's input
      if (lane == 0) {
        mbar_expect_tx(bar_x, kTM * 128);
        tma_load_2d(Xs, &tm_x, 0, (tile + (int)gridDim.x) * kTM, bar_x);
      }
      __syncwarp();
      x_pending = true;
      ++x_loads;
    }
    hidden_epilogue(sbias);
    // layers 2 and 3: A = H, B = streamed blocks
    for (int l = 0; l < 2 && ok; ++l) {
      if (warp == 0 && !*fail && !ring_layer(g0 + 1 + 4 * l, 4, false) && lane == 0) *fail = 1;
      if (!(ok = layer_done())) break;
      hidden_epilogue(sbias + 256 * (l + 1));
    }
    if (!ok) break;
    // layer 4 (N = 64, resident weights) into the output accumulator
    if (warp == 0 && !*fail) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (lane == 0) {
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
          const uint32_t a0 = smem_u32(Hs + kb * (kTM * 128)), w0 = smem_u32(W4s + kb * 64 * 128);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_bf16(tmem_out, make_desc(a0 + 32 * kk, 16, 1024, kSwizzle128B),
                     make_desc(w0 + 32 * kk, 16, 1024, kSwizzle128B), make_idesc(kTM, 64),
                     (kb | kk) ? 1u : 0u);
        }
        mma_commit(bar_mma);
      }
      __syncwarp();
    }
    if (!(ok = layer_done())) break;
    // the next tile's layer 1 (hidden accumulator) runs under this epilogue
    if (warp == 0 && i + 1 < my_tiles && !issue_layer1(i + 1) && lane == 0) *fail = 1;
    {
      // the thread's row, columns [32 half, 32 half + 32) of the output
      float *yrow = Y + ((size_t)tile * kTM + row) * 64 + 32 * half;
      const float *bo = sbias + 768 + 32 * half;
      uint32_t r[32];
      tmem_ld16_nowait(tmem_out + lane_off + (uint32_t)(32 * half), r);
      tmem_ld16_nowait(tmem_out + lane_off + (uint32_t)(32 * half + 16), r + 16);
      tmem_wait();
      float4 *o = reinterpret_cast<float4 *>(yrow);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float4 bb = *reinterpret_cast<const float4 *>(bo + 4 * j);
        o[j] = make_float4(__uint_as_float(r[4 * j]) + bb.x, __uint_as_float(r[4 * j + 1]) + bb.y,
                           __uint_as_float(r[4 * j + 2]) + bb.z, __uint_as_float(r[4 * j + 3]) + bb.w);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // the output accumulator is read before the next tile's layer 4
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
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
