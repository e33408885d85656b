// Tensor-core form of the cell-level local apply: the TF32 and BF16x3 precision
// paths of the FP32 block path.
//
// Paper: Sec. IV.B.1-2 -- the cell operator of Eq. FEHlocEl (plus the k-terms of
// Eq. FEHloc) applied as dense products of reference-cell matrices.  On a
// uniform mesh every cell shares those matrices, so the local apply of all
// cells is three plain products over the gathered cell blocks X^(e):
//
//   U      = N3 X^(e)                                  interpolation to the Gauss points
//   W      = w_q J [(V + |k|^2/2) I + B . sigma] U       pointwise 2x2 spin operator (SIMT)
//   Y^(e)  = N3^T W + K_r X^(e) + K_i (i X^(e))          testing, kinetic / k part
//
// N3 = N (x) N (x) N (n_q^3 x n_p^3), K = K_r + i K_i = sum_d G_d (x) B (x) B the
// n_p^3 x n_p^3 kinetic/k matrix.  Each product is one tcgen05 GEMM (D = A B^T,
// both operands K-major, FP32 accumulation in tensor memory) over "rows" =
// (cell, spin, vector, re|im) of a chunk of cells:
//
//   A2 [rows][QP | NPP | NPP] = [W | X | i X] (per row: the real or imaginary part)
//   GEMM 1:  U [rows][QP]  = A2[:, QP : QP + NPP] . N3^T
//   GEMM 2:  D [rows][NPP] = A2 . [N3^T | K_r | K_i]^T
//
// and the scatter-add of D into the block is SIMT with FP32 atomics.  TF32: one
// kind::tf32 pass on FP32 operands (10-bit mantissas); BF16x3: every operand
// split into BF16 hi + lo, products hi*hi + hi*lo + lo*hi with kind::f16.
//
// The sum-factorised SIMT kernel (hx_cell.cuh) does ~1.2k flop per node-vector
// at p = 6; these dense products do ~19k, so this path trades 16x the
// arithmetic for tensor-core throughput; the library reports both.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "gbc_internal.h"
#include "tc.cuh"

namespace {

__device__ int g_tcl_err;   // set when a bounded wait of the GEMM expired

constexpr int kBM = 128;    // rows of D per CTA

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(tmap), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

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

template <int MODE, int BN> struct GemmCfg {
  static constexpr int PL = MODE ? 2 : 1;               // planes (hi, lo) per operand
  static constexpr int ABYTES = kBM * 128;              // one 128-byte K slice of A
  static constexpr int BBYTES = BN * 128;
  static constexpr int STAGE = PL * (ABYTES + BBYTES);
  static constexpr int STAGES = STAGE <= 32 * 1024 ? 3 : 2;
  static constexpr int TCOLS = BN <= 128 ? 128 : 256;
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256;
};

// D[m][n0 + j] = sum_k A[m][ax0 + k] B[n0 + j][k], m in this CTA's 128 rows, j < BN,
// k over nkt tiles of 128 bytes.  Warp 0: TMA producer; warp 1: MMA issue;
// warps 2..5: epilogue (warp w reads TMEM lanes 32 (w % 4) ..).
template <int MODE, int BN>
__global__ void __launch_bounds__(192)
k_tcl_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap ta_lo,
           const __grid_constant__ CUtensorMap tb, const __grid_constant__ CUtensorMap tb_lo,
           int ax0, int nkt, float* __restrict__ D, long long ldd, long long M) {
  using G = GemmCfg<MODE, BN>;
  constexpr int KE = MODE ? 64 : 32;   // elements per 128-byte K slice
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023;
  unsigned char* st = reinterpret_cast<unsigned char*>(base);
  uint64_t* full = reinterpret_cast<uint64_t*>(st + G::STAGES * G::STAGE);
  uint64_t* empty = full + G::STAGES;
  uint64_t* accb = empty + G::STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accb + 1);
  int* fail = reinterpret_cast<int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long m0 = (long long)blockIdx.x * kBM;
  const int n0 = blockIdx.y * BN;
  auto A = [&](int s, int pl) { return tc::smem_u32(st + s * G::STAGE + pl * G::ABYTES); };
  auto B = [&](int s, int pl) {
    return tc::smem_u32(st + s * G::STAGE + G::PL * G::ABYTES + pl * G::BBYTES);
  };

  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(tslot), G::TCOLS);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < G::STAGES; ++s) {
      tc::mbar_init(tc::smem_u32(&full[s]), 1);
      tc::mbar_init(tc::smem_u32(&empty[s]), 1);
    }
    tc::mbar_init(tc::smem_u32(accb), 1);
    *fail = 0;
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // producer: stage s is reused once the MMAs that read it have completed
    int kt = 0;
    for (; kt < nkt; ++kt) {
      const int s = kt % G::STAGES;
      if (kt >= G::STAGES &&
          !tc::mbar_wait_bounded(tc::smem_u32(&empty[s]), ((kt / G::STAGES) - 1) & 1)) {
        atomicExch(fail, 1);
        break;
      }
      if (*reinterpret_cast<volatile int*>(fail)) break;
      const uint32_t fb = tc::smem_u32(&full[s]);
      tc::mbar_arrive_expect_tx(fb, G::STAGE);
      tma_load_2d(A(s, 0), &ta, ax0 + kt * KE, (int)m0, fb);
      tma_load_2d(B(s, 0), &tb, kt * KE, n0, fb);
      if (MODE) {
        tma_load_2d(A(s, 1), &ta_lo, ax0 + kt * KE, (int)m0, fb);
        tma_load_2d(B(s, 1), &tb_lo, kt * KE, n0, fb);
      }
    }
    if (*reinterpret_cast<volatile int*>(fail))   // let the copies in flight land first
      for (int j = kt > G::STAGES ? kt - G::STAGES : 0; j < kt; ++j)
        tc::mbar_wait_bounded(tc::smem_u32(&full[j % G::STAGES]), (j / G::STAGES) & 1);
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = MODE ? idesc_bf16(kBM, BN) : tc::idesc_tf32(kBM, BN);
    int kt = 0;
    for (; kt < nkt; ++kt) {
      const int s = kt % G::STAGES;
      if (!tc::mbar_wait_bounded(tc::smem_u32(&full[s]), (kt / G::STAGES) & 1)) {
        atomicExch(fail, 1);
        break;
      }
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t o = kk * 32;
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        if (MODE) {
          mma_bf16(tmem, tc::sdesc_sw128(A(s, 0) + o), tc::sdesc_sw128(B(s, 0) + o), idesc, acc);
          mma_bf16(tmem, tc::sdesc_sw128(A(s, 0) + o), tc::sdesc_sw128(B(s, 1) + o), idesc, 1u);
          mma_bf16(tmem, tc::sdesc_sw128(A(s, 1) + o), tc::sdesc_sw128(B(s, 0) + o), idesc, 1u);
        } else {
          tc::mma_tf32(tmem, tc::sdesc_sw128(A(s, 0) + o), tc::sdesc_sw128(B(s, 0) + o), idesc, acc);
        }
      }
      tc::mma_commit(tc::smem_u32(&empty[s]));
    }
    tc::mma_commit(tc::smem_u32(accb));   // also after a failure: drains the issued MMAs
  } else if (warp >= 2) {
    const int g = warp & 3;
    const bool ok = tc::mbar_wait_bounded(tc::smem_u32(accb), 0);
    if (!ok) atomicExch(fail, 1);
    tc::fence_after_sync();
    const long long row = m0 + g * 32 + lane;
    if (ok && !*reinterpret_cast<volatile int*>(fail)) {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(g * 32) << 16) + (uint32_t)c0, v);
        if (row < M) {
          float4* dst = reinterpret_cast<float4*>(D + row * ldd + n0 + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(fail) && threadIdx.x == 0) atomicExch(&g_tcl_err, 1);
  if (warp == 0) tc::tmem_dealloc(tmem, G::TCOLS);
}

// hi = bf16(x), lo = bf16(x - hi)
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

template <int MODE>
__device__ __forceinline__ void put(void* p0, void* p1, long long i, float x) {
  if (MODE) {
    __nv_bfloat16 h, l;
    split_bf16(x, h, l);
    reinterpret_cast<__nv_bfloat16*>(p0)[i] = h;
    reinterpret_cast<__nv_bfloat16*>(p1)[i] = l;
  } else {
    reinterpret_cast<float*>(p0)[i] = x;
  }
}

// one CTA per (cell of the chunk, 8 vectors): node rows staged through shared
// memory, then written as the X and i X segments of 32 rows (spin, vector, part)
constexpr int kGV = 8;
template <int MODE>
__global__ void __launch_bounds__(256)
k_tcl_gather(const float2* __restrict__ X, int ldx, int nvec, MeshDev mesh, int cell0, void* A0,
             void* A1, int KT, int QP, int NPP, int np) {
  extern __shared__ float2 xs[];   // [np^3][2][kGV]
  const int c = blockIdx.x, e = cell0 + c, v0 = blockIdx.y * kGV;
  const int np3 = np * np * np;
  const int cx = e % mesh.ncell[0], cy = (e / mesh.ncell[0]) % mesh.ncell[1],
            cz = e / (mesh.ncell[0] * mesh.ncell[1]);
  for (int i = threadIdx.x; i < np3 * 2 * kGV; i += blockDim.x) {
    const int v = i % kGV, s = (i / kGV) & 1, n = i / (2 * kGV);
    const long long I = gbc_node(mesh, cx, cy, cz, n % np, (n / np) % np, n / (np * np));
    float2 val = make_float2(0.f, 0.f);
    if (I >= 0 && v0 + v < nvec) val = X[(I * 2 + s) * ldx + v0 + v];
    xs[i] = val;
  }
  __syncthreads();
  // rows r = ((c * 2 + s) * nvec + v) * 2 + part for v < nvec
  for (int i = threadIdx.x; i < 2 * kGV * 2 * NPP; i += blockDim.x) {
    const int n = i % NPP, rr = i / NPP;
    const int part = rr & 1, v = (rr >> 1) % kGV, s = rr / (2 * kGV);
    if (v0 + v >= nvec) continue;
    const long long r = (((long long)c * 2 + s) * nvec + v0 + v) * 2 + part;
    float x = 0.f, xi = 0.f;
    if (n < np3) {
      const float2 val = xs[(n * 2 + s) * kGV + v];
      x = part ? val.y : val.x;
      xi = part ? val.x : -val.y;   // i X: (-Im, Re)
    }
    put<MODE>(A0, A1, r * KT + QP + n, x);
    put<MODE>(A0, A1, r * KT + QP + NPP + n, xi);
  }
}

// W = w_q J [(V + |k|^2/2) I + B . sigma] U at every Gauss point, written as
// the first segment of A2 (zero in the padding q >= nq^3)
template <int MODE>
__global__ void k_tcl_point(const float* __restrict__ U, const float* __restrict__ fields,
                            int nvec, int ncell, int cell0, int nq3, int QP, int KT, void* A0,
                            void* A1) {
  const long long n = (long long)ncell * nvec * QP;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i % QP);
    const long long cv = i / QP;
    const int v = (int)(cv % nvec);
    const long long c = cv / nvec;
    const long long r_u = ((c * 2 + 0) * nvec + v) * 2, r_d = ((c * 2 + 1) * nvec + v) * 2;
    float ou_r = 0.f, ou_i = 0.f, od_r = 0.f, od_i = 0.f;
    if (q < nq3) {
      const float* f = fields + (size_t)(cell0 + c) * 4 * nq3;
      const float V = f[4 * q], bx = f[4 * q + 1], by = f[4 * q + 2], bz = f[4 * q + 3];
      const float ur = U[r_u * QP + q], ui = U[(r_u + 1) * QP + q];
      const float dr = U[r_d * QP + q], di = U[(r_d + 1) * QP + q];
      // [(V + bz) u + (bx - i by) d ; (bx + i by) u + (V - bz) d]
      ou_r = (V + bz) * ur + bx * dr + by * di;
      ou_i = (V + bz) * ui + bx * di - by * dr;
      od_r = bx * ur - by * ui + (V - bz) * dr;
      od_i = bx * ui + by * ur + (V - bz) * di;
    }
    put<MODE>(A0, A1, r_u * KT + q, ou_r);
    put<MODE>(A0, A1, (r_u + 1) * KT + q, ou_i);
    put<MODE>(A0, A1, r_d * KT + q, od_r);
    put<MODE>(A0, A1, (r_d + 1) * KT + q, od_i);
  }
}

// Y[node][s][v] += D rows of the chunk (staged through shared memory per
// (cell, 8 vectors) so both the D reads and the atomics are contiguous)
__global__ void __launch_bounds__(256)
k_tcl_scatter(const float* __restrict__ D, int NPP, float2* Y, int ldx, int nvec, MeshDev mesh,
              int cell0, int np) {
  extern __shared__ float ds[];   // [2 s][kGV][2 part][NPP]
  const int c = blockIdx.x, e = cell0 + c, v0 = blockIdx.y * kGV;
  const int np3 = np * np * np;
  for (int i = threadIdx.x; i < 2 * kGV * 2 * NPP; i += blockDim.x) {
    const int n = i % NPP, rr = i / NPP;
    const int part = rr & 1, v = (rr >> 1) % kGV, s = rr / (2 * kGV);
    float val = 0.f;
    if (v0 + v < nvec) val = D[((((long long)c * 2 + s) * nvec + v0 + v) * 2 + part) * NPP + n];
    ds[i] = val;
  }
  __syncthreads();
  const int cx = e % mesh.ncell[0], cy = (e / mesh.ncell[0]) % mesh.ncell[1],
            cz = e / (mesh.ncell[0] * mesh.ncell[1]);
  for (int i = threadIdx.x; i < np3 * 2 * kGV; i += blockDim.x) {
    const int v = i % kGV, s = (i / kGV) & 1, n = i / (2 * kGV);
    if (v0 + v >= nvec) continue;
    const long long I = gbc_node(mesh, cx, cy, cz, n % np, (n / np) % np, n / (np * np));
    if (I < 0) continue;
    const int rr = (s * kGV + v) * 2;
    atomicAdd(&Y[(I * 2 + s) * ldx + v0 + v], make_float2(ds[rr * NPP + n], ds[(rr + 1) * NPP + n]));
  }
}

using EncodeTiledFn = PFN_cuTensorMapEncodeTiled_v12000;
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// row-major [rows][cols] array of FP32 (MODE 0) or BF16 (MODE 1) with a box of
// one 128-byte K slice x box_rows rows, 128-byte swizzle
bool make_map(CUtensorMap* m, const void* p, long long rows, int cols, int box_rows, int mode) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !p) return false;
  const int es = mode ? 2 : 4;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * es};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, mode ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
            const_cast<void*>(p), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE, int BN>
cudaError_t run_gemm_t(const CUtensorMap& ta, const CUtensorMap& ta_lo, const CUtensorMap& tb,
                       const CUtensorMap& tb_lo, int ax0, int K, int N, float* D, long long ldd,
                       long long M, cudaStream_t s) {
  using G = GemmCfg<MODE, BN>;
  auto k = k_tcl_gemm<MODE, BN>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  if (e != cudaSuccess) return e;
  const int KE = MODE ? 64 : 32;
  dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)(N / BN));
  k<<<grid, 192, G::SMEM, s>>>(ta, ta_lo, tb, tb_lo, ax0, K / KE, D, ldd, M);
  return cudaGetLastError();
}

// N-tile width: the widest of 256, 128, 64 that divides N (N is a multiple of 64)
inline int pick_bn(int N) { return N % 256 == 0 ? 256 : N % 128 == 0 ? 128 : 64; }

cudaError_t run_gemm(int mode, const CUtensorMap& ta, const CUtensorMap& ta_lo,
                     const CUtensorMap& tb, const CUtensorMap& tb_lo, int ax0, int K, int N,
                     float* D, long long ldd, long long M, cudaStream_t s) {
  const int bn = pick_bn(N);
#define GBC_TCL_GEMM(MD, BNV) \
  if (mode == MD && bn == BNV) return run_gemm_t<MD, BNV>(ta, ta_lo, tb, tb_lo, ax0, K, N, D, ldd, M, s)
  GBC_TCL_GEMM(0, 64);
  GBC_TCL_GEMM(0, 128);
  GBC_TCL_GEMM(0, 256);
  GBC_TCL_GEMM(1, 64);
  GBC_TCL_GEMM(1, 128);
  GBC_TCL_GEMM(1, 256);
#undef GBC_TCL_GEMM
  return cudaErrorInvalidValue;
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

// ---------------------------------------------------------------------------
// host side: dense reference-cell operators, scratch, and the chunked apply
// ---------------------------------------------------------------------------
struct TclState {
  int mode = -1, p = 0, QP = 0, NPP = 0, KT = 0;
  double h[3] = {0, 0, 0}, k[3] = {0, 0, 0};
  void* n3[2] = {nullptr, nullptr};    // [QP][NPP]  (hi, lo planes for BF16x3)
  void* b2[2] = {nullptr, nullptr};    // [NPP][KT]
  void* a2[2] = {nullptr, nullptr};    // [rows][KT]
  float* u = nullptr;                  // [rows][QP]
  float* d = nullptr;                  // [rows][NPP]
  long long rows_cap = 0;
  int a2_mode = -1, a2_kt = 0;         // mode and row width the scratch was sized for
};

void tcl_free(TclState* t) {
  if (!t) return;
  for (int i = 0; i < 2; ++i) {
    cudaFree(t->n3[i]);
    cudaFree(t->b2[i]);
    cudaFree(t->a2[i]);
  }
  cudaFree(t->u);
  cudaFree(t->d);
  delete t;
}

namespace {

// upload a row-major FP64 matrix as FP32 (mode 0) or BF16 hi/lo planes (mode 1)
gbc_status upload_op(gbc_ctx* c, const std::vector<double>& m, void** planes, int mode) {
  const size_t n = m.size();
  if (mode == 0) {
    std::vector<float> f(n);
    for (size_t i = 0; i < n; ++i) f[i] = (float)m[i];
    GBC_CU(c, cudaMalloc(&planes[0], n * sizeof(float)));
    GBC_CU(c, cudaMemcpy(planes[0], f.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    return GBC_OK;
  }
  std::vector<__nv_bfloat16> hi(n), lo(n);
  for (size_t i = 0; i < n; ++i) {
    const float x = (float)m[i];
    hi[i] = __float2bfloat16_rn(x);
    lo[i] = __float2bfloat16_rn(x - __bfloat162float(hi[i]));
  }
  for (int pl = 0; pl < 2; ++pl) {
    GBC_CU(c, cudaMalloc(&planes[pl], n * sizeof(__nv_bfloat16)));
    GBC_CU(c, cudaMemcpy(planes[pl], pl ? lo.data() : hi.data(), n * sizeof(__nv_bfloat16),
                         cudaMemcpyHostToDevice));
  }
  return GBC_OK;
}

// dense N3 and [N3^T | K_r | K_i] for the context's p, cell edges and k-point
gbc_status tcl_tables(gbc_ctx* c, TclState* t, int mode) {
  const HostTables& h = c->tab;
  const int np = c->mesh.p + 1, nq = c->nq, np3 = np * np * np, nq3 = nq * nq * nq;
  t->QP = round_up(nq3, 64);
  t->NPP = round_up(np3, 64);
  t->KT = t->QP + 2 * t->NPP;
  std::vector<double> B[3], Gr[3], Gi[3];
  for (int d = 0; d < 3; ++d) {
    B[d].resize(np * np);
    Gr[d].resize(np * np);
    Gi[d].resize(np * np);
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) {
        B[d][i * np + j] = 0.5 * c->h[d] * h.Bh[i * np + j];
        Gr[d][i * np + j] = 0.5 * (2.0 / c->h[d]) * h.Ah[i * np + j];
        Gi[d][i * np + j] = -0.5 * c->k[d] * (h.Ch[i * np + j] - h.Ch[j * np + i]);
      }
  }
  std::vector<double> n3((size_t)t->QP * t->NPP, 0.0), b2((size_t)t->NPP * t->KT, 0.0);
  for (int q = 0; q < nq3; ++q) {
    const int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
    for (int n = 0; n < np3; ++n) {
      const int ix = n % np, iy = (n / np) % np, iz = n / (np * np);
      const double v = h.N1[ix * nq + qx] * h.N1[iy * nq + qy] * h.N1[iz * nq + qz];
      n3[(size_t)q * t->NPP + n] = v;
      b2[(size_t)n * t->KT + q] = v;   // N3^T
    }
  }
  for (int m = 0; m < np3; ++m) {
    const int mx = m % np, my = (m / np) % np, mz = m / (np * np);
    for (int n = 0; n < np3; ++n) {
      const int nx = n % np, ny = (n / np) % np, nz = n / (np * np);
      const double bx = B[0][mx * np + nx], by = B[1][my * np + ny], bz = B[2][mz * np + nz];
      const double kr = Gr[0][mx * np + nx] * by * bz + bx * Gr[1][my * np + ny] * bz +
                        bx * by * Gr[2][mz * np + nz];
      const double ki = Gi[0][mx * np + nx] * by * bz + bx * Gi[1][my * np + ny] * bz +
                        bx * by * Gi[2][mz * np + nz];
      b2[(size_t)m * t->KT + t->QP + n] = kr;
      b2[(size_t)m * t->KT + t->QP + t->NPP + n] = ki;
    }
  }
  for (int i = 0; i < 2; ++i) {
    cudaFree(t->n3[i]);
    cudaFree(t->b2[i]);
    t->n3[i] = t->b2[i] = nullptr;
  }
  GBC_TRY(upload_op(c, n3, t->n3, mode));
  GBC_TRY(upload_op(c, b2, t->b2, mode));
  t->mode = mode;
  t->p = c->mesh.p;
  for (int d = 0; d < 3; ++d) {
    t->h[d] = c->h[d];
    t->k[d] = c->k[d];
  }
  return GBC_OK;
}

}  // namespace

// Y += H^loc X for an FP32 block with the local products on the tensor cores
// (mode 0: TF32, mode 1: BF16x3).  Cells are processed in chunks whose scratch
// stays under ~4 GB.
gbc_status tcl_apply(gbc_ctx* c, const float2* X, float2* Y, int nvec, int ldx, int mode,
                     cudaStream_t s) {
  if (nvec == 0) return GBC_OK;
  if (!c->tcl) c->tcl = new TclState();
  TclState* t = c->tcl;
  bool stale = t->mode != mode || t->p != c->mesh.p;
  for (int d = 0; d < 3; ++d) stale = stale || t->h[d] != c->h[d] || t->k[d] != c->k[d];
  if (stale) GBC_TRY(tcl_tables(c, t, mode));
  const int np = c->mesh.p + 1, nq3 = c->nq * c->nq * c->nq;
  const int es = mode ? 2 : 4;
  const long long per_cell = 4LL * nvec;   // rows per cell
  // per row: A2 (FP32, or two BF16 planes) + U + D, 4 bytes per column each
  const size_t row_bytes = sizeof(float) * (size_t)(t->KT + t->QP + t->NPP);
  long long ec = std::max<long long>(1, (4LL << 30) / ((long long)row_bytes * per_cell));
  ec = std::min<long long>(ec, c->mesh.E);
  const long long rows = ec * per_cell;
  // A2 holds FP32 (TF32) or two BF16 planes (BF16x3): reallocate when the mode changes
  if (rows > t->rows_cap || t->a2_mode != mode || t->a2_kt != t->KT) {
    for (int i = 0; i < 2; ++i) {
      cudaFree(t->a2[i]);
      t->a2[i] = nullptr;
    }
    cudaFree(t->u);
    cudaFree(t->d);
    t->u = t->d = nullptr;
    t->rows_cap = 0;
    for (int i = 0; i < (mode ? 2 : 1); ++i) GBC_CU(c, cudaMalloc(&t->a2[i], (size_t)rows * t->KT * es));
    GBC_CU(c, cudaMalloc(&t->u, sizeof(float) * (size_t)rows * t->QP));
    GBC_CU(c, cudaMalloc(&t->d, sizeof(float) * (size_t)rows * t->NPP));
    t->rows_cap = rows;
    t->a2_mode = mode;
    t->a2_kt = t->KT;
  }
  CUtensorMap ma, ma_lo, mn3, mn3_lo, mb2, mb2_lo;
  bool ok = make_map(&ma, t->a2[0], t->rows_cap, t->KT, kBM, mode) &&
            make_map(&mn3, t->n3[0], t->QP, t->NPP, pick_bn(t->QP), mode) &&
            make_map(&mb2, t->b2[0], t->NPP, t->KT, pick_bn(t->NPP), mode);
  if (mode) {
    ok = ok && make_map(&ma_lo, t->a2[1], t->rows_cap, t->KT, kBM, mode) &&
         make_map(&mn3_lo, t->n3[1], t->QP, t->NPP, pick_bn(t->QP), mode) &&
         make_map(&mb2_lo, t->b2[1], t->NPP, t->KT, pick_bn(t->NPP), mode);
  } else {
    ma_lo = ma;
    mn3_lo = mn3;
    mb2_lo = mb2;
  }
  if (!ok) return gbc_fail(c, GBC_ECUDA, "tensor map encoding failed (tensor-core cell apply)");
  const size_t gsm = sizeof(float2) * (size_t)np * np * np * 2 * kGV;
  const size_t ssm = sizeof(float) * 2 * kGV * 2 * (size_t)t->NPP;
  GBC_CU(c, cudaFuncSetAttribute(k_tcl_gather<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
  GBC_CU(c, cudaFuncSetAttribute(k_tcl_gather<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
  GBC_CU(c, cudaFuncSetAttribute(k_tcl_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm));
  for (long long c0 = 0; c0 < c->mesh.E; c0 += ec) {
    const int nc = (int)std::min<long long>(ec, c->mesh.E - c0);
    const long long m = (long long)nc * per_cell;
    dim3 gg((unsigned)nc, (unsigned)((nvec + kGV - 1) / kGV));
    if (mode)
      k_tcl_gather<1><<<gg, 256, gsm, s>>>(X, ldx, nvec, c->mesh, (int)c0, t->a2[0], t->a2[1], t->KT,
                                           t->QP, t->NPP, np);
    else
      k_tcl_gather<0><<<gg, 256, gsm, s>>>(X, ldx, nvec, c->mesh, (int)c0, t->a2[0], t->a2[1], t->KT,
                                           t->QP, t->NPP, np);
    GBC_CU(c, cudaGetLastError());
    GBC_CU(c, run_gemm(mode, ma, ma_lo, mn3, mn3_lo, t->QP, t->NPP, t->QP, t->u, t->QP, m, s));
    const long long npt = (long long)nc * nvec * t->QP;
    const unsigned pg = (unsigned)std::max<long long>(
        1, std::min<long long>((npt + 255) / 256, 64LL * gbc_sm_count()));
    if (mode)
      k_tcl_point<1><<<pg, 256, 0, s>>>(t->u, c->d_fields32, nvec, nc, (int)c0, nq3, t->QP, t->KT,
                                        t->a2[0], t->a2[1]);
    else
      k_tcl_point<0><<<pg, 256, 0, s>>>(t->u, c->d_fields32, nvec, nc, (int)c0, nq3, t->QP, t->KT,
                                        t->a2[0], t->a2[1]);
    GBC_CU(c, cudaGetLastError());
    GBC_CU(c, run_gemm(mode, ma, ma_lo, mb2, mb2_lo, 0, t->KT, t->NPP, t->d, t->NPP, m, s));
    k_tcl_scatter<<<gg, 256, ssm, s>>>(t->d, t->NPP, Y, ldx, nvec, c->mesh, (int)c0, np);
    GBC_CU(c, cudaGetLastError());
  }
  return GBC_OK;
}

// bounded-wait flag of the tensor-core cell apply (cleared on read)
cudaError_t tcl_error(int* err, cudaStream_t s) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(err, g_tcl_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_tcl_err, &zero, sizeof(int));
}
