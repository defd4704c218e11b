// BF16 tensor-core GEMM for the learned warm start, written for sm_103a's
// fifth-generation tensor cores (tcgen05): C = act(A B^T + bias).
//
//   A: [M][K] bf16 row-major (K contiguous), B: [N][K] bf16 row-major,
//   bias: [N] fp32 (or NULL), C: [M][N] bf16 or fp32 row-major.
//   M % 128 == 0, K % 64 == 0, 16 <= N <= 256, N % 16 == 0.
//
// One CTA of 128 threads computes a 128 x N tile.  Operand tiles (128 x 64
// and N x 64) are staged in shared memory in the tensor core's canonical
// K-major layout without swizzle (8-row x 16-byte core matrices), a single
// elected thread issues tcgen05.mma (M = 128, K = 16 per instruction) with
// the fp32 accumulator in tensor memory, tcgen05.commit signals an mbarrier,
// and the four warps read their 32 accumulator lanes back with tcgen05.ld
// for the epilogue (bias, ReLU, conversion).  Two shared-memory stages let
// the next K block load (cp.async) while the tensor core works on the current one.
// Every mbarrier wait is bounded: on timeout the kernel records an error
// flag, skips the rest and frees its tensor memory.
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "dm_internal.h"
#include "dm_tc.cuh"

namespace dm {

namespace {

constexpr int kBM = 128, kBK = 64, kThreads = 128;
using tc::make_desc;
using tc::make_idesc;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_bf16;
using tc::mma_commit;
using tc::smem_u32;

// Copies a rows x 64 bf16 tile (row-major source with leading dimension ld
// elements) into the canonical no-swizzle K-major layout: core matrix
// (r/8, k/8) at ((r/8) * 8 + k/8) * 128 bytes, row r%8 at 16-byte stride.
// Asynchronous 16-byte copies (cp.async), so that every thread's loads are
// in flight together; the caller commits the group and waits on it.
__device__ __forceinline__ void stage_tile(char *dst, const uint16_t *src, int rows, int ld,
                                           int k0, int tid) {
  const int chunks = rows * (kBK / 8);  // 16-byte chunks
  for (int c = tid; c < chunks; c += kThreads) {
    const int r = c >> 3, kc = c & 7;
    const uint16_t *g = src + (size_t)r * ld + k0 + kc * 8;
    const uint32_t d = smem_u32(dst + ((r >> 3) * 8 + kc) * 128 + (r & 7) * 16);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(g) : "memory");
  }
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace

// Split K (gridDim.y > 1): CTA (x, z) reduces K columns [z kchunk, (z+1) kchunk)
// and writes its fp32 partial tile to C + z M N (k_sum_splits adds them).
__global__ void __launch_bounds__(kThreads) k_gemm_bf16(const uint16_t *__restrict__ A,
                                                        const uint16_t *__restrict__ B,
                                                        const float *__restrict__ bias, void *C,
                                                        int M, int N, int K, int relu,
                                                        int out_f32, int *err, int kchunk) {
  extern __shared__ __align__(1024) char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM;
  const int kz = blockIdx.y * kchunk;  // first K column of this CTA
  if (gridDim.y > 1) C = reinterpret_cast<float *>(C) + (size_t)blockIdx.y * M * N;
  const int a_bytes = kBM * kBK * 2, b_bytes = N * kBK * 2;
  // stage s: A tile at s * (a_bytes + b_bytes), B tile right after it
  auto sA = [&](int st) { return smem + st * (a_bytes + b_bytes); };
  auto sB = [&](int st) { return smem + a_bytes + st * (a_bytes + b_bytes); };
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * (a_bytes + b_bytes));
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2);
  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = make_idesc(kBM, N);
  const int nk = kchunk / kBK;
  bool ok = true;
  uint32_t phase[2] = {0, 0};

  // two-stage pipeline: the copies of block kb + 1 are in flight while the
  // tensor core multiplies block kb
  stage_tile(sA(0), A + (size_t)m0 * K, kBM, K, kz, tid);
  stage_tile(sB(0), B, N, K, kz, tid);
  cp_commit();
  for (int kb = 0; kb < nk && ok; ++kb) {
    const int s = kb & 1;
    if (kb + 1 < nk) {
      // stage s^1 was last read by the MMAs of block kb - 1
      if (kb >= 1) {
        const bool w = mbar_wait(&bar[s ^ 1], phase[s ^ 1]);
        phase[s ^ 1] ^= 1u;
        ok = __syncthreads_and(w) != 0;  // uniform decision: no thread is left behind
        if (!ok) break;
      }
      stage_tile(sA(s ^ 1), A + (size_t)m0 * K, kBM, K, kz + (kb + 1) * kBK, tid);
      stage_tile(sB(s ^ 1), B, N, K, kz + (kb + 1) * kBK, tid);
      cp_commit();
      cp_wait<1>();  // block kb has landed (block kb + 1 may still be in flight)
    } else {
      cp_wait<0>();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(sA(s)), b0 = smem_u32(sB(s));
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        // K = 16 per instruction = two 8-element core matrices (256 bytes)
        const uint64_t ad = make_desc(a0 + kk * 256, 128, 1024);
        const uint64_t bd = make_desc(b0 + kk * 256, 128, 1024);
        mma_bf16(tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&bar[s]);
    }
    __syncthreads();
  }
  // the last commit covers every MMA issued before it
  {
    const int sl = (nk - 1) & 1;
    const bool w = ok ? mbar_wait(&bar[sl], phase[sl]) : false;
    ok = __syncthreads_and(w) != 0;
  }
  cp_wait<0>();  // nothing left in flight on an early exit
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok) {
    if (lane == 0) atomicExch(err, 1);
  } else {
    // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w + 31
    // (16 columns per tcgen05.ld: N is a multiple of 16)
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
          "%10, %11, %12, %13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
            "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
            "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        v[j] = __uint_as_float(r[j]) + (bias ? bias[c0 + j] : 0.0f);
        if (relu) v[j] = fmaxf(v[j], 0.0f);
      }
      if (row < M) {
        if (out_f32) {
          float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(C) + (size_t)row * N + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
          uint32_t w[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            w[j] = *reinterpret_cast<const uint32_t *>(&b);
          }
          uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(C) + (size_t)row * N + c0);
          o[0] = make_uint4(w[0], w[1], w[2], w[3]);
          o[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// out[i] = sum over z < nsplit of part[z n + i] (fixed order: deterministic).
__global__ void k_sum_splits(int64_t n, int nsplit, const float *part, float *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.0f;
  for (int z = 0; z < nsplit; ++z) acc += part[(size_t)z * n + i];
  out[i] = acc;
}

size_t gemm_smem_bytes(int N) { return 2 * (size_t)(kBM * kBK * 2 + N * kBK * 2) + 64; }

// Launches k_gemm_bf16; err: device int (set to 1 on a barrier timeout).
// ksplit > 1: fp32 output only, the partial tiles go to `work` (ksplit M N
// floats) and are summed into C; K / ksplit must be a multiple of 64.
cudaError_t launch_gemm_bf16(int M, int N, int K, const void *A, const void *B, const float *bias,
                             void *C, int relu, int out_f32, int *err, cudaStream_t st,
                             int ksplit, float *work) {
  static bool attr_set = false;
  const size_t smem = gemm_smem_bytes(256);
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (ksplit > 1) {
    if (!out_f32 || relu || bias || !work || K % (ksplit * kBK)) return cudaErrorInvalidValue;
    k_gemm_bf16<<<dim3(M / kBM, ksplit), kThreads, gemm_smem_bytes(N), st>>>(
        (const uint16_t *)A, (const uint16_t *)B, nullptr, work, M, N, K, 0, 1, err, K / ksplit);
    const int64_t n = (int64_t)M * N;
    k_sum_splits<<<(int)((n + 255) / 256), 256, 0, st>>>(n, ksplit, work, (float *)C);
    return cudaGetLastError();
  }
  k_gemm_bf16<<<M / kBM, kThreads, gemm_smem_bytes(N), st>>>(
      (const uint16_t *)A, (const uint16_t *)B, bias, C, M, N, K, relu, out_f32, err, K);
  return cudaGetLastError();
}

bool check_gemm_shape(int M, int N, int K) {
  return M > 0 && M % kBM == 0 && K > 0 && K % kBK == 0 && N >= 16 && N <= 256 && N % 16 == 0;
}

}  // namespace dm

extern "C" dm_status dm_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *A, const void *B,
                                  const float *bias, void *C, int32_t relu, int32_t out_f32,
                                  void *stream) {
  using namespace dm;
  if (!A || !B || !C || !check_gemm_shape(M, N, K) ||
      (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 15)) {
    set_error("dm_gemm_bf16: need M % 128 == 0, K % 64 == 0, N in [16, 256] with N % 16 == 0 "
              "and 16-byte aligned A, B, C");
    return DM_ERR_INVALID_ARG;
  }
  int *err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    set_error("dm_gemm_bf16: cudaMalloc");
    return DM_ERR_OOM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = launch_gemm_bf16(M, N, K, A, B, bias, C, relu, out_f32, err, st, 1, nullptr);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(err);
  if (e != cudaSuccess) {
    set_error(std::string("dm_gemm_bf16: ") + cudaGetErrorString(e));
    return DM_ERR_CUDA;
  }
  if (h) {
    set_error("dm_gemm_bf16: tensor-core completion barrier timed out");
    return DM_ERR_CUDA;
  }
  return DM_OK;
}
