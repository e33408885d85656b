// Arithmetic-throughput probes: the denominators of the roofline fractions the
// library's kernels are measured against.  Each probe keeps one pipe busy with
// independent work that never leaves registers (or, for the tensor cores,
// shared memory and tensor memory) and is timed with CUDA events:
//
//   GBC_PEAK_FFMA    FP32 fused multiply-add, one per instruction
//   GBC_PEAK_FFMA2   FP32 paired fused multiply-add (two per instruction)
//   GBC_PEAK_DFMA    FP64 fused multiply-add
//   GBC_PEAK_TF32    tcgen05.mma kind::tf32, M = 128, N = 256, K = 8
//   GBC_PEAK_BF16    tcgen05.mma kind::f16 with BF16 operands, M = 128, N = 256, K = 16
//
// The tensor-core probes issue back-to-back MMAs from one elected thread per
// SM onto operands that stay resident in shared memory, alternating between two
// accumulators in tensor memory; completion is awaited with a bounded wait.
#include <algorithm>

#include "gbc_internal.h"
#include "tc.cuh"

namespace {

__device__ int g_peak_err;
__device__ float g_peak_sink;

constexpr int kChains = 16;

template <int ITERS>
__global__ void __launch_bounds__(256) k_ffma(float seed, int flag) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = seed + threadIdx.x * 1e-7f + i;
  const float m = 0.999999f, c = 1e-7f;
#pragma unroll 4
  for (int it = 0; it < ITERS; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, c);
  float s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (flag == 12345 && s == 0.123f) g_peak_sink = s;   // keeps the chains alive
}

template <int ITERS>
__global__ void __launch_bounds__(256) k_ffma2(float seed, int flag) {
  float2 a[kChains / 2 + kChains / 2];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = make_float2(seed + threadIdx.x * 1e-7f + i, seed - i);
  const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
#pragma unroll 4
  for (int it = 0; it < ITERS; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], m, c);
  float s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
  if (flag == 12345 && s == 0.123f) g_peak_sink = s;
}

template <int ITERS>
__global__ void __launch_bounds__(256) k_dfma(double seed, int flag) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = seed + threadIdx.x * 1e-9 + i;
  const double m = 0.9999999, c = 1e-9;
#pragma unroll 4
  for (int it = 0; it < ITERS; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);
  double s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (flag == 12345 && s == 0.123) g_peak_sink = (float)s;
}

// instruction descriptor: kind::f16 with BF16 A and B, F32 accumulate, K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// A: 128 rows x 128 B, B: 256 rows x 128 B (K-major, 128-byte swizzle), zero-filled
template <bool BF16>
__global__ void __launch_bounds__(128) k_mma_loop(int nmma) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023;
  float4* A = reinterpret_cast<float4*>(base);
  float4* B = A + 128 * 8;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(B + 256 * 8);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x;
  for (int i = tid; i < (128 + 256) * 8; i += blockDim.x) A[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid < 32) {
    tc::tmem_alloc(tc::smem_u32(tslot), 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(mbar), 1);
    tc::fence_mbar_init();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    const uint64_t ad = tc::sdesc_sw128(tc::smem_u32(A)), bd = tc::sdesc_sw128(tc::smem_u32(B));
    for (int i = 0; i < nmma; ++i) {
      const uint32_t d = tmem + (uint32_t)((i & 1) * 256);
      if (BF16)
        mma_bf16(d, ad, bd, idesc_bf16(128, 256), i > 1 ? 1u : 0u);
      else
        tc::mma_tf32(d, ad, bd, tc::idesc_tf32(128, 256), i > 1 ? 1u : 0u);
    }
    tc::mma_commit(tc::smem_u32(mbar));
  }
  __syncwarp();
  const bool ok = tc::mbar_wait_bounded(tc::smem_u32(mbar), 0);
  if (!ok && tid == 0) atomicExch(&g_peak_err, 1);
  tc::fence_after_sync();
  __syncthreads();
  if (tid < 32) tc::tmem_dealloc(tmem, 512);
}

}  // namespace

extern "C" gbc_status gbc_alu_peak(int which, double* flops_per_s, double* seconds, void* stream) {
  if (!flops_per_s || which < 0 || which > 4) return GBC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GBC_ECUDA;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return GBC_ECUDA;
  int zero = 0;
  cudaMemcpyToSymbolAsync(g_peak_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
  constexpr int kIters = 8192;
  double flops = 0;
  cudaError_t e = cudaSuccess;
  const int nmma = 16384;
  const size_t tc_smem = 1024 + sizeof(float4) * 8 * (128 + 256) + 64 + 96 * 1024;  // 1 CTA/SM
  auto launch = [&]() -> cudaError_t {
    switch (which) {
      case 0: k_ffma<kIters><<<nsm * 8, 256, 0, s>>>(1.0f, 0); break;
      case 1: k_ffma2<kIters><<<nsm * 8, 256, 0, s>>>(1.0f, 0); break;
      case 2: k_dfma<kIters / 16><<<nsm * 8, 256, 0, s>>>(1.0, 0); break;
      case 3: k_mma_loop<false><<<nsm, 128, tc_smem, s>>>(nmma); break;
      case 4: k_mma_loop<true><<<nsm, 128, tc_smem, s>>>(nmma); break;
    }
    return cudaGetLastError();
  };
  if (which >= 3) {
    e = cudaFuncSetAttribute(which == 3 ? k_mma_loop<false> : k_mma_loop<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem);
    if (e != cudaSuccess) return GBC_ECUDA;
  }
  switch (which) {
    case 0: flops = 2.0 * kChains * kIters * 256.0 * nsm * 8; break;
    case 1: flops = 4.0 * kChains * kIters * 256.0 * nsm * 8; break;
    case 2: flops = 2.0 * kChains * (kIters / 16) * 256.0 * nsm * 8; break;
    case 3: flops = 2.0 * 128 * 256 * 8 * (double)nmma * nsm; break;
    case 4: flops = 2.0 * 128 * 256 * 16 * (double)nmma * nsm; break;
  }
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first launch is the warm-up
    cudaEventRecord(a, s);
    e = launch();
    cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    if (rep > 0) best = std::min(best, ms);
  }
  int err = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyFromSymbol(&err, g_peak_err, sizeof(int));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return GBC_ECUDA;
  if (err) return GBC_ETIMEOUT;
  *flops_per_s = flops / (best * 1e-3);
  if (seconds) *seconds = best * 1e-3;
  return GBC_OK;
}
