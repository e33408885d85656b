// 3xTF32 NT GEMM on the tcgen05 tensor cores: D[M][N] = A[M][K] B[N][K]^T, FP32
// in and out, row-major.  One CTA (4 warps) owns 128 rows of D and all N
// columns (16 <= N <= 256, a multiple of 16); K advances in tiles of 32.  Each
// tile of A and B is split into TF32 hi and lo parts in 128B-swizzled K-major
// shared memory and accumulated in TMEM with hi*hi + hi*lo + lo*hi.  This is
// the building block of the nonlocal projector contractions and is exported
// (gbc_tc_gemm_nt) so its layouts are tested on their own.
#include "gbc_internal.h"
#include "tc.cuh"

namespace {

__device__ int g_tc_err;   // set when a bounded wait expired

template <int N>
__global__ void __launch_bounds__(128) k_tc_gemm_nt(const float* __restrict__ A,
                                                    const float* __restrict__ B, float* D, int M,
                                                    int K) {
  static_assert(N >= 16 && N <= 256 && N % 16 == 0, "N");
  constexpr int NCOL = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023;
  float4* Ahi = reinterpret_cast<float4*>(base);   // 128 rows x 8 chunks
  float4* Alo = Ahi + 128 * 8;
  float4* Bhi = Alo + 128 * 8;                     // N rows x 8 chunks
  float4* Blo = Bhi + N * 8;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + N * 8);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * 128;

  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(tslot), NCOL);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(mbar), 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::idesc_tf32(128, N);
  bool ok = true;
  uint32_t phase = 0;
  for (int k0 = 0; k0 < K && ok; k0 += 32) {
    {   // A: thread = row
      const int m = m0 + tid;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = k0 + 4 * c + j;
          const float x = (m < M && k < K) ? A[(size_t)m * K + k] : 0.f;
          tc::split_tf32(x, h[j], l[j]);
        }
        Ahi[tc::sw128(tid, c)] = make_float4(h[0], h[1], h[2], h[3]);
        Alo[tc::sw128(tid, c)] = make_float4(l[0], l[1], l[2], l[3]);
      }
    }
    for (int n = tid; n < N; n += 128) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = k0 + 4 * c + j;
          const float x = k < K ? B[(size_t)n * K + k] : 0.f;
          tc::split_tf32(x, h[j], l[j]);
        }
        Bhi[tc::sw128(n, c)] = make_float4(h[0], h[1], h[2], h[3]);
        Blo[tc::sw128(n, c)] = make_float4(l[0], l[1], l[2], l[3]);
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo);
      const uint32_t bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t o = kk * 32;
        const uint32_t acc = (k0 > 0 || kk > 0) ? 1u : 0u;
        tc::mma_tf32(tmem, tc::sdesc_sw128(ah + o), tc::sdesc_sw128(bh + o), idesc, acc);
        tc::mma_tf32(tmem, tc::sdesc_sw128(ah + o), tc::sdesc_sw128(bl + o), idesc, 1u);
        tc::mma_tf32(tmem, tc::sdesc_sw128(al + o), tc::sdesc_sw128(bh + o), idesc, 1u);
      }
      tc::mma_commit(tc::smem_u32(mbar));
    }
    ok = tc::mbar_wait_bounded(tc::smem_u32(mbar), phase);
    phase ^= 1u;
    tc::fence_after_sync();
    __syncthreads();
  }
  if (!ok && (tid & 31) == 0) atomicExch(&g_tc_err, 1);
  if (ok) {
    const int row = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < M)
#pragma unroll
        for (int j = 0; j < 16; ++j) D[(size_t)row * N + c0 + j] = v[j];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, NCOL);
}

template <int N>
cudaError_t run_gemm(const float* A, const float* B, float* D, int M, int K, cudaStream_t s) {
  const size_t smem = 1024 + sizeof(float4) * 8 * (2 * 128 + 2 * N) + 64;
  auto k = k_tc_gemm_nt<N>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<(M + 127) / 128, 128, smem, s>>>(A, B, D, M, K);
  return cudaGetLastError();
}

}  // namespace

extern "C" gbc_status gbc_tc_gemm_nt(const float* A, const float* B, float* D, int M, int N, int K,
                                     void* stream) {
  if (!A || !B || !D || M < 1 || K < 1) return GBC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int zero = 0;
  if (cudaMemcpyToSymbolAsync(g_tc_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return GBC_ECUDA;
  cudaError_t e;
  switch (N) {
    case 16: e = run_gemm<16>(A, B, D, M, K, s); break;
    case 32: e = run_gemm<32>(A, B, D, M, K, s); break;
    case 48: e = run_gemm<48>(A, B, D, M, K, s); break;
    case 64: e = run_gemm<64>(A, B, D, M, K, s); break;
    case 128: e = run_gemm<128>(A, B, D, M, K, s); break;
    case 256: e = run_gemm<256>(A, B, D, M, K, s); break;
    default: return GBC_EUNSUPPORTED;
  }
  if (e != cudaSuccess) return GBC_ECUDA;
  int err = 0;
  if (cudaMemcpyFromSymbolAsync(&err, g_tc_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GBC_ECUDA;
  return err ? GBC_ETIMEOUT : GBC_OK;
}
