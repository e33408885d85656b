// Nonlocal spin-orbit step of H.X on the tcgen05 tensor cores (FP32 path).
//
// Paper: Eq. FEHnloc and step 3 of Sec. IV.B.2, C = P_a^H X, C' = Delta_a C,
// Y += P_a C'.  The two large contractions are real GEMMs over real and
// imaginary parts, computed in 3xTF32 (hi*hi + hi*lo + lo*hi, FP32-level
// accuracy) with TMEM accumulators; the 2npj x 2npj coupling stays on the SIMT
// cores.  A "real column" is one float of a node row [2][ldx] complex, i.e.
// col = 2*(s*ldx + v) + part.
//
//  projection  (per atom, 32 support nodes per K tile)
//              D[m][n] = sum_nodes X(node, col0 + m) Q_n(node), Q_2chi = Re P_chi,
//              Q_2chi+1 = Im P_chi.  Neighbouring lanes hold the real and the
//              imaginary column of one complex column, and C = sum conj(P) X is
//              Re C = D[re][2chi] + D[im][2chi+1], Im C = D[im][2chi] - D[re][2chi+1].
//  expansion   (per chunk of <= 128 owned nodes, K over the chunk's atom slots)
//              D[m][n] = sum_k A[m][k] B[n][k] with A[m] = (Re P_b, Im P_b)(node m)
//              for every slot atom b holding node m (zero otherwise), and
//              B[re col] = (Re C'_b, -Im C'_b), B[im col] = (Im C'_b, Re C'_b):
//              D is the real / imaginary part of sum_b P_b C'_b, added to Y once.
#include <algorithm>
#include <type_traits>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>

#include "gbc_internal.h"
#include "tc.cuh"

namespace {

__device__ int g_nltc_err;   // set when a bounded wait expired

constexpr int kMT = 128;     // rows of D per CTA (one per thread)
constexpr int kCT = 128;     // real columns per CTA
constexpr int kMaxGridY = 65535;   // chunks per launch (grid y limit)

struct TcCtx {
  uint32_t tmem;
  uint32_t mbar;
};

template <int NCOL>
__device__ __forceinline__ TcCtx tc_begin(uint64_t* mbar, uint32_t* tslot) {
  if ((threadIdx.x >> 5) == 0) {
    tc::tmem_alloc(tc::smem_u32(tslot), NCOL);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(mbar), 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  return TcCtx{*tslot, tc::smem_u32(mbar)};
}

template <int NCOL>
__device__ __forceinline__ void tc_end(const TcCtx& t) {
  tc::fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(t.tmem, NCOL);
}

// make the staged tile visible to the tensor core and issue its 3 x 4 MMAs
// (thread 0), completion signalled on the mbarrier.  The tensor core's FP32
// accumulator truncates toward zero at every accumulating MMA, a bias that
// grows with the chain length, so the main products hi*hi go to their own
// accumulator D0 (4 accumulations per tile) and the small cross terms
// hi*lo + lo*hi (relative size 2^-11, their truncation is negligible) to D1 =
// D0 + d1col; callers keep D0 chains short and add D0 + D1 in FP32.  Without
// SPLIT all three products accumulate into D0.
template <int N, bool SPLIT = true>
__device__ __forceinline__ void tc_issue(const TcCtx& t, uint32_t d1col, const float4* Ahi,
                                         const float4* Alo, const float4* Bhi, const float4* Blo,
                                         bool first) {
  tc::fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc::fence_after_sync();
    constexpr uint32_t idesc = tc::idesc_tf32(kMT, N);
    const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo);
    const uint32_t bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
    const uint32_t d0 = t.tmem, d1 = SPLIT ? t.tmem + d1col : t.tmem;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint32_t o = kk * 32;
      const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
      tc::mma_tf32(d0, tc::sdesc_sw128(ah + o), tc::sdesc_sw128(bh + o), idesc, acc);
      tc::mma_tf32(d1, tc::sdesc_sw128(ah + o), tc::sdesc_sw128(bl + o), idesc, SPLIT ? acc : 1u);
      tc::mma_tf32(d1, tc::sdesc_sw128(al + o), tc::sdesc_sw128(bh + o), idesc, 1u);
    }
    tc::mma_commit(t.mbar);
  }
}

// all threads: wait (bounded) for the issued MMAs; the tile buffers are free after
__device__ __forceinline__ bool tc_wait(const TcCtx& t, uint32_t& phase) {
  const bool ok = tc::mbar_wait_bounded(t.mbar, phase);
  phase ^= 1u;
  tc::fence_after_sync();
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

// after an expired wait: flag it and give the MMAs in flight a second bounded
// wait before the TMEM is freed
__device__ __forceinline__ void tc_fail(const TcCtx& t, uint32_t phase) {
  if (threadIdx.x == 0) atomicExch(&g_nltc_err, 1);
  tc::mbar_wait_bounded(t.mbar, phase ^ 1u);
}

__device__ __forceinline__ void put_split(float4* hi, float4* lo, int row, int chunk, float a,
                                          float b, float c, float d) {
  float h0, h1, h2, h3, l0, l1, l2, l3;
  tc::split_tf32(a, h0, l0);
  tc::split_tf32(b, h1, l1);
  tc::split_tf32(c, h2, l2);
  tc::split_tf32(d, h3, l3);
  hi[tc::sw128(row, chunk)] = make_float4(h0, h1, h2, h3);
  lo[tc::sw128(row, chunk)] = make_float4(l0, l1, l2, l3);
}

// ---- projection ------------------------------------------------------------------
constexpr int kPrjChunk = 1024;   // support nodes per projection chunk (setup table)
constexpr int kSeg = 8;           // K tiles per accumulation segment (256 nodes)

template <int NB>
constexpr size_t project_smem() {
  return 1024 + sizeof(float4) * 8 * (2 * kMT + 2 * NB) + sizeof(long long) * kPrjChunk + 64;
}

template <int NB>
__global__ void __launch_bounds__(128, 4)
k_tc_project(const float* __restrict__ Xr, int ldx, int nvec, const int4* __restrict__ chunks,
             const long long* __restrict__ nodes, const float2* __restrict__ P,
             const int* __restrict__ atom_npj, const int* __restrict__ atom_pv_off,
             const int* __restrict__ atom_c_off, float2* __restrict__ Cbuf, int chunk0, long long M) {
  static_assert(NB % 16 == 0 && NB >= 16 && NB <= 128, "NB");
  constexpr int NCOL = NB <= 32 ? 32 : NB <= 64 ? 64 : 128;   // per accumulator (D0, D1)
  constexpr int NBC = NB / 16;   // B float4 chunks per thread (NB rows x 8 chunks / 128)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023;
  float4* Ahi = reinterpret_cast<float4*>(base);
  float4* Alo = Ahi + kMT * 8;
  float4* Bhi = Alo + kMT * 8;
  float4* Blo = Bhi + NB * 8;
  long long* Ns = reinterpret_cast<long long*>(Blo + NB * 8);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Ns + kPrjChunk);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

  // an earlier CTA gave up (read once, the same decision in every thread)
  if (__syncthreads_or(*reinterpret_cast<volatile int*>(&g_nltc_err))) return;
  const int4 ch = chunks[chunk0 + blockIdx.y];   // (atom, first position, count, node offset)
  const int atom = ch.x, j0 = ch.y, cnt = min(ch.z, kPrjChunk), noff = ch.w;
  const int npj = atom_npj[atom];
  const float2* Pa = P + atom_pv_off[atom] + (size_t)j0 * npj;
  const int ncols = 4 * ldx;
  const int tid = threadIdx.x;
  const int col = blockIdx.x * kCT + tid;
  const bool cok = col < ncols && ((col >> 1) % ldx) < nvec;
  for (int t = tid; t < cnt; t += 128) Ns[t] = nodes[noff + j0 + t];
  const TcCtx t = tc_begin<2 * NCOL>(mbar, tslot);   // includes a __syncthreads

  // kind::tf32 takes K-major operands only (an MN-major tf32 operand reads as
  // zero on sm_103a), so A row m = column col0 + m is gathered column-wise: 32
  // scalar loads per thread and tile, coalesced across the warp.  Two register
  // buffers: the loads of tile i + 2 are issued while tile i is multiplied.
  float xa0[32], xa1[32];
  float xb0[NBC][4], xb1[NBC][4];
  auto load = [&](float (&xa)[32], float (&xb)[NBC][4], int k0) {
#pragma unroll
    for (int k = 0; k < 32; ++k)
      xa[k] = (cok && k0 + k < cnt && GBC_IN_RANGE(GBC_SITE_NL_NODE, Ns[k0 + k], M))
                  ? __ldg(&Xr[Ns[k0 + k] * (long long)ncols + col]) : 0.f;
#pragma unroll
    for (int i = 0; i < NBC; ++i) {
      const int q = tid + 128 * i, n = q >> 3, c = q & 7;
      const int chi = n >> 1, im = n & 1;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = k0 + 4 * c + j;
        float val = 0.f;
        if (chi < npj && k < cnt) {
          const float2 p = __ldg(&Pa[(size_t)k * npj + chi]);
          val = im ? p.y : p.x;
        }
        xb[i][j] = val;
      }
    }
  };
  auto stage = [&](const float (&xa)[32], const float (&xb)[NBC][4]) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
      put_split(Ahi, Alo, tid, c, xa[4 * c], xa[4 * c + 1], xa[4 * c + 2], xa[4 * c + 3]);
#pragma unroll
    for (int i = 0; i < NBC; ++i) {
      const int q = tid + 128 * i;
      put_split(Bhi, Blo, q >> 3, q & 7, xb[i][0], xb[i][1], xb[i][2], xb[i][3]);
    }
  };
  // C += D0 + D1 for this CTA's columns (round-to-nearest FP32 atomics); lane
  // pairs hold the real / imaginary column of one complex column
  const int warp = tid >> 5;
  const int ci = col >> 1, s = ci / ldx, v = ci % ldx;
  const bool store = (tid & 1) == 0 && cok;
  const int r0 = atom_c_off[atom];
  auto flush = [&]() {
#pragma unroll 1
    for (int c0 = 0; c0 < NB; c0 += 8) {
      uint32_t a0[8], a1[8];
      const uint32_t ta = t.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      tc::tmem_ld8_nowait(ta, a0);
      tc::tmem_ld8_nowait(ta + NCOL, a1);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        const float dr = __uint_as_float(a0[j]) + __uint_as_float(a1[j]);
        const float di = __uint_as_float(a0[j + 1]) + __uint_as_float(a1[j + 1]);
        const float pr = __shfl_xor_sync(0xffffffffu, dr, 1);   // D[im][2chi]
        const float pi = __shfl_xor_sync(0xffffffffu, di, 1);   // D[im][2chi+1]
        const int chi = (c0 + j) >> 1;
        if (store && chi < npj)
          atomicAdd(&Cbuf[(size_t)(r0 + 2 * chi + s) * nvec + v], make_float2(dr + pi, pr - di));
      }
    }
    tc::fence_before_sync();   // the next tile's MMAs overwrite D0 / D1
  };
  uint32_t phase = 0;
  bool ok = true;
  if (cnt > 0) load(xa0, xb0, 0);
  if (cnt > 32) load(xa1, xb1, 32);
  for (int k0 = 0; k0 < cnt && ok; k0 += 64) {
    stage(xa0, xb0);
    tc_issue<NB>(t, NCOL, Ahi, Alo, Bhi, Blo, k0 % (32 * kSeg) == 0);
    if (k0 + 64 < cnt) load(xa0, xb0, k0 + 64);
    ok = tc_wait(t, phase);
    if (!ok || k0 + 32 >= cnt) break;
    stage(xa1, xb1);
    tc_issue<NB>(t, NCOL, Ahi, Alo, Bhi, Blo, false);
    if (k0 + 96 < cnt) load(xa1, xb1, k0 + 96);
    ok = tc_wait(t, phase);
    if (ok && (k0 + 64) % (32 * kSeg) == 0 && k0 + 64 < cnt) flush();
  }
  if (!ok)
    tc_fail(t, phase);
  else if (cnt > 0)
    flush();
  tc_end<2 * NCOL>(t);
}

// ---- projection, TMA-fed pipeline -------------------------------------------------
// The same product with the X rows brought in by TMA and A kept in tensor
// memory.  Warp roles:
//   warp 0        producer: per tile of 32 support nodes, eight tile::gather4
//                 copies (4 rows x 128 columns each) and one bulk copy of the
//                 tile's P rows into a ring of kStages raw stages (completion:
//                 mbarrier transaction bytes);
//   warp 1        MMA issue (A from tensor memory, B from shared memory);
//   warps 2..17   converters: warp w owns TMEM lanes 32 (w % 4) .. + 31 (A rows =
//                 real columns) and the K quarter 8 q .. 8 q + 7, q = (w - 2) / 4;
//                 they split a raw stage into TF32 hi / lo, store A into tensor
//                 memory (tcgen05.st) and the K-major B tile into shared memory,
//                 kAB buffers each, so that kAB tiles of MMAs can be in flight;
//   warps 18..21  epilogue: flush each finished 256-node segment's accumulators
//                 through round-to-nearest FP32 atomics while the next segment
//                 is multiplied into the other accumulator set.
// Accumulators: two sets (segment parity, 128 TMEM columns apart): one N = 2 NB
// MMA per K step multiplies A_hi by the stacked [B_lo; B_hi] tile (hi*lo in
// columns 0..NB-1, hi*hi in NB..2NB-1) and one N = NB MMA adds lo*hi to the
// cross-term columns: 8 MMAs per tile instead of 12 (the tensor core's time per
// MMA at these shapes is mostly fixed), and the truncating hi*hi chain stays 4
// MMAs per tile, 32 per segment.  No CTA-wide
// barrier sits between a load and its use.  Requires ldx == nvec, 4 ldx >= 128,
// 16-byte aligned X and even P offsets.
constexpr int kStages = 6;
constexpr int kAB = 4;                           // A / B buffers
constexpr int kConvWarps = 16;
constexpr int kConv = 32 * kConvWarps;           // converter threads
constexpr int kEpiWarp0 = 2 + kConvWarps;        // first epilogue warp
constexpr int kPrjThreads = 32 * (kEpiWarp0 + 4);

__device__ __forceinline__ bool wait_uniform(uint32_t mbar, uint32_t parity, volatile int* abort_flag) {
  bool ok = false;
  for (uint32_t i = 0; i < (1u << 22); ++i) {
    if (tc::mbar_try_wait(mbar, parity)) {
      ok = true;
      break;
    }
    if ((i & 255u) == 255u && *abort_flag) break;
  }
  ok = __all_sync(0xffffffffu, ok);
  if (!ok && (threadIdx.x & 31) == 0) {
    *abort_flag = 1;
    atomicExch(&g_nltc_err, 1);
  }
  return ok;
}

template <int NB>
constexpr size_t project_tma_smem() {
  return 1024 + 2 * kAB * (size_t)NB * 128     // B hi / lo, kAB buffers
         + (size_t)kStages * 16384             // raw X stages
         + (size_t)kStages * NB * 128          // raw P stages
         + 4 * kPrjChunk                       // node rows of the chunk
         + 8 * (2 * kStages + 2 * kAB + 4) + 32;   // barriers, TMEM slot, flags
}

template <int NB>
__global__ void __launch_bounds__(kPrjThreads, 1)
k_tc_project_tma(const __grid_constant__ CUtensorMap xmap, int ldx, int nvec,
                 const int4* __restrict__ chunks, const long long* __restrict__ nodes,
                 const float2* __restrict__ P, const int* __restrict__ atom_npj,
                 const int* __restrict__ atom_pv_off, const int* __restrict__ atom_c_off,
                 float2* __restrict__ Cbuf, int chunk0) {
  static_assert(NB % 16 == 0 && NB >= 16 && NB <= 64, "NB");
  constexpr int ACOL = 256;                    // A buffers (hi 32 + lo 32 columns) after the two sets
  constexpr int TCOLS = 512;
  static_assert(ACOL + 64 * kAB <= TCOLS, "TMEM");
  constexpr uint32_t kBT = NB * 128;           // bytes of one B tile (hi or lo)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr uint32_t kBB = 2 * kAB * kBT;     // all B buffers
  float* rawX = reinterpret_cast<float*>(base + kBB);                         // [S][32][128]
  float2* rawP = reinterpret_cast<float2*>(base + kBB + kStages * 16384);      // [S][NB * 16]
  int* rows = reinterpret_cast<int*>(base + kBB + kStages * 16384 + kStages * kBT);
  uint64_t* bars = reinterpret_cast<uint64_t*>(rows + kPrjChunk);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 2 * kAB + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* prog = reinterpret_cast<volatile int*>(tslot + 2);   // issued / waited / MMA'd tiles
  auto Bl = [&](int b) { return reinterpret_cast<float4*>(base + 2 * b * kBT); };
  auto Bh = [&](int b) { return reinterpret_cast<float4*>(base + (2 * b + 1) * kBT); };
  auto full = [&](int s) { return tc::smem_u32(bars + s); };
  auto empty = [&](int s) { return tc::smem_u32(bars + kStages + s); };
  auto afull = [&](int b) { return tc::smem_u32(bars + 2 * kStages + b); };
  auto aempty = [&](int b) { return tc::smem_u32(bars + 2 * kStages + kAB + b); };
  auto segdone = [&](int p) { return tc::smem_u32(bars + 2 * kStages + 2 * kAB + p); };
  auto setfree = [&](int p) { return tc::smem_u32(bars + 2 * kStages + 2 * kAB + 2 + p); };

  // an earlier CTA gave up (read once, the same decision in every thread)
  if (__syncthreads_or(*reinterpret_cast<volatile int*>(&g_nltc_err))) return;
  const int4 ch = chunks[chunk0 + blockIdx.y];   // (atom, first position, count, node offset)
  const int atom = ch.x, j0 = ch.y, cnt = min(ch.z, kPrjChunk), noff = ch.w;
  const int npj = atom_npj[atom];
  const float2* Pa = P + atom_pv_off[atom] + (size_t)j0 * npj;
  const int col0 = blockIdx.x * kCT;
  const int ncols = 4 * ldx;
  const int T = (cnt + 31) / 32;
  const int nseg = (T + kSeg - 1) / kSeg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int i = threadIdx.x; i < 32 * T; i += blockDim.x)
    rows[i] = i < cnt ? (int)nodes[noff + j0 + i] : -1;   // -1: rows read as zero
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(tslot), TCOLS);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < kStages; ++i) {
      tc::mbar_init(full(i), 1);
      tc::mbar_init(empty(i), kConv);
    }
    for (int b = 0; b < kAB; ++b) {
      tc::mbar_init(afull(b), kConv);
      tc::mbar_init(aempty(b), 1);
    }
    for (int p = 0; p < 2; ++p) {
      tc::mbar_init(segdone(p), 1);
      tc::mbar_init(setfree(p), 128);
    }
    *abort_flag = 0;
    prog[0] = prog[1] = prog[2] = 0;
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ---- producer
    for (int t = 0; t < T; ++t) {
      const int s = t % kStages;
      if (t >= kStages && !wait_uniform(empty(s), ((t / kStages) - 1) & 1, abort_flag)) break;
      const int nval = min(32, cnt - t * 32);
      const uint32_t pbytes = ((uint32_t)(nval * npj * 8) + 15u) & ~15u;
      if (lane == 0) tc::mbar_arrive_expect_tx(full(s), 16384u + pbytes);
      __syncwarp();
      if (lane < 8) {
        const int* r = rows + t * 32 + 4 * lane;
        tc::tma_gather4(tc::smem_u32(rawX + s * 4096 + lane * 512), &xmap, col0, r[0], r[1], r[2],
                        r[3], full(s));
      }
      if (lane == 0) {
        tc::bulk_g2s(tc::smem_u32(rawP + s * (kBT / 8)), Pa + (size_t)t * 32 * npj, pbytes, full(s));
        prog[0] = t + 1;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue
    constexpr uint32_t idesc2 = tc::idesc_tf32(kMT, 2 * NB);   // A_hi x [B_lo; B_hi]
    constexpr uint32_t idesc = tc::idesc_tf32(kMT, NB);        // A_lo x B_hi
    for (int t = 0; t < T; ++t) {
      const int b = t % kAB, sg = t / kSeg, p = sg & 1;
      const bool first = t % kSeg == 0;
      if (first && sg >= 2 && !wait_uniform(setfree(p), ((sg >> 1) - 1) & 1, abort_flag)) break;
      if (!wait_uniform(afull(b), (t / kAB) & 1, abort_flag)) break;
      tc::fence_after_sync();
      if (lane == 0) {
        const uint32_t ah = tmem + (uint32_t)(ACOL + 64 * b), al = ah + 32;
        const uint32_t bh = tc::smem_u32(Bh(b)), bl = tc::smem_u32(Bl(b));
        const uint32_t d = tmem + (uint32_t)(128 * p);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t o = kk * 32;
          const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
          // B_hi follows B_lo: the N = 2 NB descriptor at B_lo covers both
          tc::mma_tf32_ts(d, ah + 8 * kk, tc::sdesc_sw128(bl + o), idesc2, acc);
          tc::mma_tf32_ts(d, al + 8 * kk, tc::sdesc_sw128(bh + o), idesc, 1u);
        }
        tc::mma_commit(aempty(b));
        if (t % kSeg == kSeg - 1 || t == T - 1) tc::mma_commit(segdone(p));
        prog[2] = t + 1;
      }
      __syncwarp();
    }
  } else if (warp < kEpiWarp0) {
    // ---- converters
    const int m = 32 * (warp & 3) + lane;      // A row = TMEM lane = real column col0 + m
    const int q = (warp - 2) >> 2;             // K quarter
    const int ct = threadIdx.x - 64;           // converter thread 0 .. kConv - 1
    const int col = col0 + m;
    const bool cok = col < ncols && ((col >> 1) % ldx) < nvec;
    for (int t = 0; t < T; ++t) {
      const int s = t % kStages, b = t % kAB;
      if (!wait_uniform(full(s), (t / kStages) & 1, abort_flag)) break;
      if (ct == 0) prog[1] = t + 1;
      if (t >= kAB && !wait_uniform(aempty(b), ((t / kAB) - 1) & 1, abort_flag)) break;
      tc::fence_after_sync();   // the MMAs that read A / B buffer b have completed
      {
        const float* rx = rawX + s * 4096 + 8 * q * 128;
        float hi[8], lo[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) tc::split_tf32(cok ? rx[k * 128 + m] : 0.f, hi[k], lo[k]);
        const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(ACOL + 64 * b + 8 * q);
        tc::tmem_st8(ta, hi);
        tc::tmem_st8(ta + 32, lo);
      }
      // B: chunk (row n, K chunk c), n fastest across the lanes (conflict-free)
      const float2* rp = rawP + s * (kBT / 8);
      const int nval = min(32, cnt - t * 32);
      for (int qq = ct; qq < NB * 8; qq += kConv) {
        const int n = qq % NB, c = qq / NB;
        const int chi = n >> 1, im = n & 1;
        float y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = 4 * c + j;
          float val = 0.f;
          if (chi < npj && k < nval) {
            const float2 pv = rp[k * npj + chi];
            val = im ? pv.y : pv.x;
          }
          y[j] = val;
        }
        put_split(Bh(b), Bl(b), n, c, y[0], y[1], y[2], y[3]);
      }
      tc::tmem_wait_st();
      tc::fence_proxy_async();
      tc::fence_before_sync();
      tc::mbar_arrive(empty(s));
      tc::mbar_arrive(afull(b));
    }
  } else {
    // ---- epilogue: C += sum of the segment's three accumulators
    const int m = 32 * (warp & 3) + lane;
    const int col = col0 + m;
    const bool cok = col < ncols && ((col >> 1) % ldx) < nvec;
    const int ci = col >> 1, sp = ci / ldx, v = ci % ldx;
    const bool store = (lane & 1) == 0 && cok;
    const int r0c = atom_c_off[atom];
    for (int sg = 0; sg < nseg; ++sg) {
      const int p = sg & 1;
      if (!wait_uniform(segdone(p), (sg >> 1) & 1, abort_flag)) break;
      tc::fence_after_sync();
#pragma unroll 1
      for (int c0 = 0; c0 < NB; c0 += 8) {
        const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(128 * p + c0);
        uint32_t a0[8], a1[8];
        tc::tmem_ld8_nowait(ta + NB, a0);   // hi*hi
        tc::tmem_ld8_nowait(ta, a1);        // cross terms
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          const float dr = __uint_as_float(a0[j]) + __uint_as_float(a1[j]);
          const float di = __uint_as_float(a0[j + 1]) + __uint_as_float(a1[j + 1]);
          const float pr = __shfl_xor_sync(0xffffffffu, dr, 1);   // D[im][2chi]
          const float pi = __shfl_xor_sync(0xffffffffu, di, 1);   // D[im][2chi+1]
          const int chi = (c0 + j) >> 1;
          if (store && chi < npj)
            atomicAdd(&Cbuf[(size_t)(r0c + 2 * chi + sp) * nvec + v], make_float2(dr + pi, pr - di));
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(setfree(p));
    }
  }
  // ---- teardown: after an expired wait, give the copies and MMAs in flight a
  // bounded wait of their own before the TMEM is freed
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) {
    for (int t = prog[1]; t < prog[0]; ++t) tc::mbar_wait_bounded(full(t % kStages), (t / kStages) & 1);
    if (prog[2] > 0) tc::mbar_wait_bounded(aempty((prog[2] - 1) % kAB), ((prog[2] - 1) / kAB) & 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

// ---- expansion -------------------------------------------------------------------
constexpr int kDsStride = 68;     // staged D half-tile row stride (floats), conflict-free

constexpr size_t expand_smem() {
  return 1024 + sizeof(float4) * 8 * 4 * 128                 // A, B hi / lo tiles
         + sizeof(int) * 128 * GBC_TC_MAX_SLOTS              // row position per slot
         + sizeof(int) * 4 * GBC_TC_MAX_SLOTS                // slot metadata
         + sizeof(long long) * 128 + 64;                     // row nodes, barrier
}

__global__ void __launch_bounds__(128)
k_tc_expand(float* __restrict__ Yr, int ldx, int nvec, int ks, const int4* __restrict__ chunks,
            const int* __restrict__ slots, const long long* __restrict__ own_node,
            const int* __restrict__ own_pos, const int* __restrict__ own_xptr,
            const int2* __restrict__ own_xinc, const float2* __restrict__ P,
            const int* __restrict__ atom_npj, const int* __restrict__ atom_pv_off,
            const int* __restrict__ atom_c_off, const float2* __restrict__ Cp, int chunk0,
            int overwrite, long long M) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023;
  float4* Ahi = reinterpret_cast<float4*>(base);
  float4* Alo = Ahi + 128 * 8;
  float4* Bhi = Alo + 128 * 8;
  float4* Blo = Bhi + 128 * 8;
  float* Ds = reinterpret_cast<float*>(base);     // epilogue staging over the free tiles
  int* rowpos = reinterpret_cast<int*>(Blo + 128 * 8);   // [slot][row]
  int* s_npj = rowpos + 128 * GBC_TC_MAX_SLOTS;
  int* s_pv = s_npj + GBC_TC_MAX_SLOTS;
  int* s_c = s_pv + GBC_TC_MAX_SLOTS;
  int* s_atom = s_c + GBC_TC_MAX_SLOTS;
  long long* s_node = reinterpret_cast<long long*>(s_atom + GBC_TC_MAX_SLOTS);   // [128]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(s_node + 128);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

  // an earlier CTA gave up (read once, the same decision in every thread)
  if (__syncthreads_or(*reinterpret_cast<volatile int*>(&g_nltc_err))) return;
  const int4 ch = chunks[chunk0 + blockIdx.y];   // (first owned index, count, slot offset, slots)
  const int u0 = ch.x, cnt = min(ch.y, 128), nsl = min(ch.w, GBC_TC_MAX_SLOTS);
  const int tid = threadIdx.x;
  const int ncols = 4 * ldx;
  const int col0 = blockIdx.x * kCT;
  if (tid < nsl) {
    const int b = slots[ch.z + tid];
    s_atom[tid] = b;
    s_npj[tid] = atom_npj[b];
    s_pv[tid] = atom_pv_off[b];
    s_c[tid] = atom_c_off[b];
  }
  for (int i = tid; i < 128 * GBC_TC_MAX_SLOTS; i += 128) rowpos[i] = -1;
  // one accumulator: the chain is short (K = slots x 2 npj, about 4 tiles), and
  // 128 TMEM columns keep 3 CTAs per SM
  const TcCtx t = tc_begin<128>(mbar, tslot);   // includes a __syncthreads
  if (tid < cnt) {   // slot 0 is the owner of every row of the chunk
    const int u = u0 + tid;
    s_node[tid] = own_node[u];
    if (!GBC_IN_RANGE(GBC_SITE_NL_NODE, s_node[tid], M)) s_node[tid] = -1;   // checked build: skipped
    rowpos[tid] = own_pos[u];
    for (int k = own_xptr[u]; k < own_xptr[u + 1]; ++k) {
      const int2 inc = own_xinc[k];
      for (int sl = 1; sl < nsl; ++sl)
        if (s_atom[sl] == inc.x) rowpos[sl * 128 + tid] = inc.y;
    }
  }
  __syncthreads();

  // B row n = real column col0 + n
  const int col = col0 + tid;
  const int ci = col >> 1, cs = ci / ldx, cv = ci % ldx;
  const bool cok = col < ncols && cv < nvec;
  const bool cim = (col & 1) != 0;
  const int ktot = nsl * ks;
  float xa[32], xb[32];
  auto load = [&](int k0) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {   // pairs (2chi, 2chi + 1) of one slot
      const int kg = k0 + 2 * j;
      const int sl = kg / ks, chi = (kg - sl * ks) >> 1;
      float2 p = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
      if (kg < ktot && chi < s_npj[sl]) {
        const int pos = rowpos[sl * 128 + tid];
        if (pos >= 0) p = __ldg(&P[s_pv[sl] + (size_t)pos * s_npj[sl] + chi]);
        if (cok) c = __ldg(&Cp[(size_t)(s_c[sl] + 2 * chi + cs) * nvec + cv]);
      }
      xa[2 * j] = p.x;
      xa[2 * j + 1] = p.y;
      xb[2 * j] = cim ? c.y : c.x;
      xb[2 * j + 1] = cim ? c.x : -c.y;
    }
  };
  uint32_t phase = 0;
  bool ok = true;
  load(0);
  for (int k0 = 0; k0 < ktot && ok; k0 += 32) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      put_split(Ahi, Alo, tid, c, xa[4 * c], xa[4 * c + 1], xa[4 * c + 2], xa[4 * c + 3]);
      put_split(Bhi, Blo, tid, c, xb[4 * c], xb[4 * c + 1], xb[4 * c + 2], xb[4 * c + 3]);
    }
    tc_issue<128, false>(t, 0, Ahi, Alo, Bhi, Blo, k0 == 0);
    if (k0 + 32 < ktot) load(k0 + 32);
    ok = tc_wait(t, phase);
  }
  if (!ok) {
    tc_fail(t, phase);
  } else if (ktot > 0) {
    // epilogue in two 64-column halves: TMEM -> shared (row per thread) ->
    // coalesced read-modify-write of 256 contiguous bytes of each node row
    const int warp = tid >> 5, lane = tid & 31;
    const bool full = ldx == nvec;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
#pragma unroll 1
      for (int c0 = 0; c0 < 64; c0 += 16) {
        float d[16];
        tc::tmem_ld16(t.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(64 * h + c0), d);
        float4* dst = reinterpret_cast<float4*>(Ds + tid * kDsStride + c0);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          dst[j] = make_float4(d[4 * j], d[4 * j + 1], d[4 * j + 2], d[4 * j + 3]);
      }
      __syncthreads();
      const int cc = 64 * h + 4 * (lane & 15);   // this lane's 4 columns of the half
      const int gc = col0 + cc;
      const int rbase = warp * 2 + (lane >> 4);    // rows rbase + 8 i
      if (full && gc + 4 <= ncols) {
        // all 16 row loads in flight before the first add
        float4 yv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int r = rbase + 8 * i;
          yv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (r < cnt && !overwrite && (!GBC_CHECKED_BUILD || s_node[r] >= 0))
            yv[i] = *reinterpret_cast<const float4*>(Yr + s_node[r] * (long long)ncols + gc);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int r = rbase + 8 * i;
          if (r < cnt && (!GBC_CHECKED_BUILD || s_node[r] >= 0)) {
            const float4 dv = *reinterpret_cast<const float4*>(Ds + r * kDsStride + 4 * (lane & 15));
            yv[i].x += dv.x;
            yv[i].y += dv.y;
            yv[i].z += dv.z;
            yv[i].w += dv.w;
            *reinterpret_cast<float4*>(Yr + s_node[r] * (long long)ncols + gc) = yv[i];
          }
        }
      } else {
#pragma unroll 1
        for (int r = rbase; r < cnt; r += 8) {
          if (GBC_CHECKED_BUILD && s_node[r] < 0) continue;
          const float* dv = Ds + r * kDsStride + 4 * (lane & 15);
          float* y = Yr + s_node[r] * (long long)ncols + gc;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int c = gc + j;
            if (c < ncols && ((c >> 1) % ldx) < nvec) y[j] = overwrite ? dv[j] : y[j] + dv[j];
          }
        }
      }
      __syncthreads();
    }
  }
  tc_end<128>(t);
}

// ---- expansion from packed operands -----------------------------------------------
// The same product D = A B^T per (chunk, column tile) with both operands prepared
// ahead in the MMA's shared-memory layout, so the kernel only copies, multiplies and
// stores:
//   A (P values): per slot instance of a chunk (setup, k_xpack_a), K = 40 (2 n_pj <= 40
//       zero-padded), 128 rows; rows of nodes outside the slot atom's support are zero.
//   B (C' values): per (atom, column tile) after the coupling step (k_xpack_b).
// Each operand of one slot is [hi: 5 K steps][lo: 5 K steps], a K step being 128 rows
// x 8 values in the 32-byte swizzled layout (4 KB): 40 KB, one bulk copy.
constexpr int kXSteps = 5;                        // K steps of 8 per slot
constexpr int kXK = 8 * kXSteps;                  // K per slot (>= 2 n_pj)
constexpr uint32_t kXBlk = 128u * 32u;            // one K step, bytes
constexpr uint32_t kXHalf = kXSteps * kXBlk;      // hi or lo part of one operand
constexpr uint32_t kXOp = 2 * kXHalf;             // one operand (40 KB)
constexpr uint32_t kXStage = 2 * kXOp;            // A and B of one slot (80 KB)
constexpr int kXRow = 128 * 4 + 16;               // epilogue row: one tile row + pad, bytes
constexpr int kXThreads = 192;                    // producer, MMA, 4 epilogue warps

// 256-byte alignment (the 32-byte swizzle atom), two stages, 128 staging rows, barriers
// and the chunk-index ring
constexpr size_t xexp_smem() { return 256 + 2 * (size_t)kXStage + 128 * (size_t)kXRow + 256; }

// store the hi / lo split of K values v[0..kXK) of row r into an operand block
__device__ __forceinline__ void xpack_row(float* blk, int r, const float (&v)[kXK]) {
#pragma unroll
  for (int ks = 0; ks < kXSteps; ++ks) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float hi[4], lo[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) tc::split_tf32(v[8 * ks + 4 * h + e], hi[e], lo[e]);
      const int off = ks * 1024 + tc::sw32(r, h);
      *reinterpret_cast<float4*>(blk + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<float4*>(blk + kXHalf / 4 + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

// A blocks: one CTA per chunk, thread r = row (owned node u0 + r); slot sl of the
// chunk at block (slot offset + sl).  A[r][2chi] = Re P_b(node, chi), [2chi+1] = Im.
__global__ void __launch_bounds__(128)
k_xpack_a(float* __restrict__ Apre, const int4* __restrict__ chunks, const int* __restrict__ slots,
          const int* __restrict__ own_pos, const int* __restrict__ own_xptr,
          const int2* __restrict__ own_xinc, const float2* __restrict__ P,
          const int* __restrict__ atom_npj, const int* __restrict__ atom_pv_off) {
  const int4 ch = chunks[blockIdx.x];
  const int r = threadIdx.x;
  const int u = ch.x + r;
  for (int sl = 0; sl < ch.w; ++sl) {
    const int b = slots[ch.z + sl];
    int pos = -1;
    if (r < ch.y) {
      if (sl == 0) {
        pos = own_pos[u];
      } else {
        for (int k = own_xptr[u]; k < own_xptr[u + 1]; ++k)
          if (own_xinc[k].x == b) pos = own_xinc[k].y;
      }
    }
    const int npj = atom_npj[b];
    float v[kXK];
#pragma unroll
    for (int k = 0; k < kXK; k += 2) {
      float2 p = make_float2(0.f, 0.f);
      if (pos >= 0 && k / 2 < npj) p = P[atom_pv_off[b] + (size_t)pos * npj + k / 2];
      v[k] = p.x;
      v[k + 1] = p.y;
    }
    xpack_row(Apre + (size_t)(ch.z + sl) * (kXOp / 4), r, v);
  }
}

// B blocks: one CTA per (atom b, column tile j), thread n = real column 128 j + n of
// the [2][ldx] complex node row.  B[re col][2chi] = Re C', [2chi+1] = -Im C';
// B[im col][2chi] = Im C', [2chi+1] = Re C' (so D = Re / Im of sum_chi P C').
__global__ void __launch_bounds__(128)
k_xpack_b(float* __restrict__ Bpre, const float2* __restrict__ Cp, int ldx, int nvec,
          const int* __restrict__ atom_npj, const int* __restrict__ atom_c_off) {
  const int b = blockIdx.x, j = blockIdx.y, n = threadIdx.x;
  const int col = j * 128 + n;
  const int ci = col >> 1, s = ci / ldx, v = ci % ldx;
  const bool ok = col < 4 * ldx && v < nvec;
  const bool im = (col & 1) != 0;
  const int npj = atom_npj[b], r0 = atom_c_off[b];
  float x[kXK];
#pragma unroll
  for (int k = 0; k < kXK; k += 2) {
    float2 c = make_float2(0.f, 0.f);
    if (ok && k / 2 < npj) c = Cp[(size_t)(r0 + k + s) * nvec + v];
    x[k] = im ? c.y : c.x;
    x[k + 1] = im ? c.x : -c.y;
  }
  xpack_row(Bpre + ((size_t)b * gridDim.y + j) * (kXOp / 4), n, x);
}

// single-thread bounded wait that also gives up once another role has flagged a failure
__device__ __forceinline__ bool wait_one(uint32_t mbar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t i = 0; i < (1u << 22); ++i) {
    if (tc::mbar_try_wait(mbar, parity)) return true;
    if ((i & 255u) == 255u && *abort_flag) break;
  }
  *abort_flag = 1;
  atomicExch(&g_nltc_err, 1);
  return false;
}

// Y rows of the owned nodes = P C' (overwrite), persistent: the CTAs take chunks from the
// zeroed counter *ctr (one thread fetches, a four-entry ring in shared memory hands each
// index to the MMA thread and the epilogue warps), and every column tile of each in turn:
//   warp 0    one thread: bulk copies of each slot's A and B blocks into a two-stage ring;
//             an A block already held by the stage (chunks of one or two atoms, from the
//             previous tile) is not copied again
//   warp 1    TMEM owner; one thread issues 5 K steps x 3 products (3xTF32) per slot
//             into one of two 128-column accumulators
//   warps 2-5 epilogue: TMEM -> registers -> the thread's own staging row -> one bulk
//             copy of the tile's 512 contiguous bytes of its node row; lane quadrant = warp % 4
__global__ void __launch_bounds__(kXThreads, 1)
k_tc_expand_ws(float* __restrict__ Yr, long long M, int ncols, int ntiles, int nchunks,
               const int4* __restrict__ chunks, const int* __restrict__ slots,
               const long long* __restrict__ own_node, const float* __restrict__ Apre,
               const float* __restrict__ Bpre, unsigned long long* __restrict__ ctr) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 255) & ~(uintptr_t)255;
  unsigned char* stage0 = reinterpret_cast<unsigned char*>(base);
  unsigned char* rows = stage0 + 2 * kXStage;
  // full[2] empty[2] tfull[2] tempty[2] cfull[4] cempty[4]
  uint64_t* bars = reinterpret_cast<uint64_t*>(rows + 128 * kXRow);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 16);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  int* prog = reinterpret_cast<int*>(tslot + 2);   // [0] stage uses issued, [1] consumed, [2] commits
  volatile int* s_chunk = reinterpret_cast<volatile int*>(prog + 3);   // [4] chunk-index ring
  auto full = [&](int s) { return tc::smem_u32(bars + s); };
  auto empty = [&](int s) { return tc::smem_u32(bars + 2 + s); };
  auto tfull = [&](int a) { return tc::smem_u32(bars + 4 + a); };
  auto tempty = [&](int a) { return tc::smem_u32(bars + 6 + a); };
  auto cfull = [&](int k) { return tc::smem_u32(bars + 8 + k); };
  auto cempty = [&](int k) { return tc::smem_u32(bars + 12 + k); };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // an earlier CTA gave up (read once, the same decision in every thread)
  if (__syncthreads_or(*reinterpret_cast<volatile int*>(&g_nltc_err))) return;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 6; ++i) tc::mbar_init(tc::smem_u32(bars + i), 1);
    for (int i = 6; i < 8; ++i) tc::mbar_init(tc::smem_u32(bars + i), 4);   // one per epilogue warp
    for (int i = 8; i < 12; ++i) tc::mbar_init(tc::smem_u32(bars + i), 1);  // producer
    for (int i = 12; i < 16; ++i) tc::mbar_init(tc::smem_u32(bars + i), 5); // MMA + 4 epilogue warps
    *abort_flag = 0;
    prog[0] = prog[1] = prog[2] = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tc::smem_u32(tslot), 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      int use = 0;
      int held0 = -1, held1 = -1;   // slot instance whose A block each stage holds
      bool ok = true;
      int chn = (int)atomicAdd(ctr, 1ULL);
      for (int kk = 0; ok && !*abort_flag; ++kk) {
        // hand the chunk index to the other roles (nchunks or more: the end)
        const int rs = kk & 3;
        if (kk >= 4 && !wait_one(cempty(rs), ((kk >> 2) - 1) & 1, abort_flag)) break;
        s_chunk[rs] = chn;
        tc::mbar_arrive(cfull(rs));
        if (chn >= nchunks) break;
        const int4 ch = chunks[chn];
        chn = (int)atomicAdd(ctr, 1ULL);   // the next index, fetched while this chunk runs
        for (int j = 0; j < ntiles && ok; ++j) {
          for (int sl = 0; sl < ch.w; ++sl, ++use) {
            const int st = use & 1;
            if (use >= 2 && !wait_one(empty(st), ((use >> 1) - 1) & 1, abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t dst = tc::smem_u32(stage0 + st * kXStage);
            const bool loadA = (st ? held1 : held0) != ch.z + sl;
            tc::mbar_arrive_expect_tx(full(st), loadA ? kXStage : kXOp);
            if (loadA) tc::bulk_g2s(dst, Apre + (size_t)(ch.z + sl) * (kXOp / 4), kXOp, full(st));
            tc::bulk_g2s(dst + kXOp, Bpre + ((size_t)slots[ch.z + sl] * ntiles + j) * (kXOp / 4),
                         kXOp, full(st));
            if (st) held1 = ch.z + sl;
            else held0 = ch.z + sl;
            prog[0] = use + 1;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_tf32(128, 128);
      int use = 0, n = 0;
      bool ok = true;
      for (int kk = 0; ok && !*abort_flag; ++kk) {
        const int rs = kk & 3;
        if (!wait_one(cfull(rs), (kk >> 2) & 1, abort_flag)) break;
        const int chn = s_chunk[rs];
        tc::mbar_arrive(cempty(rs));
        if (chn >= nchunks) break;
        const int4 ch = chunks[chn];
      for (int j = 0; j < ntiles && ok; ++j, ++n) {
        const int acc = n & 1;
        if (n >= 2 && !wait_one(tempty(acc), ((n >> 1) - 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(128 * acc);
        for (int sl = 0; sl < ch.w; ++sl, ++use) {
          const int st = use & 1;
          if (!wait_one(full(st), (use >> 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          prog[1] = use + 1;
          tc::fence_after_sync();
          const uint32_t a = tc::smem_u32(stage0 + st * kXStage), b = a + kXOp;
#pragma unroll
          for (int ks = 0; ks < kXSteps; ++ks) {
            const uint32_t o = ks * kXBlk;
            tc::mma_tf32(d, tc::sdesc_sw32(a + o), tc::sdesc_sw32(b + o), idesc,
                         (sl > 0 || ks > 0) ? 1u : 0u);
            tc::mma_tf32(d, tc::sdesc_sw32(a + o), tc::sdesc_sw32(b + kXHalf + o), idesc, 1u);
            tc::mma_tf32(d, tc::sdesc_sw32(a + kXHalf + o), tc::sdesc_sw32(b + o), idesc, 1u);
          }
          tc::mma_commit(empty(st));   // the stage is free once these MMAs complete
        }
        if (!ok) break;
        tc::mma_commit(tfull(acc));
        prog[2] = n + 1;
      }
      }
    }
  } else {
    // epilogue: thread -> row r of the accumulator (TMEM lane r)
    const int q = warp & 3;
    const int r = 32 * q + lane;
    unsigned char* myrow = rows + r * kXRow;
    const uint32_t myrow_s = tc::smem_u32(myrow);
    int n = 0;
    bool ok = true;
    for (int kk = 0; ok; ++kk) {
      const int rs = kk & 3;
      if (!wait_uniform(cfull(rs), (kk >> 2) & 1, abort_flag)) break;
      const int chn = s_chunk[rs];
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(cempty(rs));
      if (chn >= nchunks) break;
      const int4 ch = chunks[chn];
      long long node = r < ch.y ? own_node[ch.x + r] : -1;
      if (node >= 0 && !GBC_IN_RANGE(GBC_SITE_NL_NODE, node, M)) node = -1;   // checked build
      for (int j = 0; j < ntiles; ++j, ++n) {
        const int acc = n & 1;
        if (!wait_uniform(tfull(acc), (n >> 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const int col0 = 128 * j;
        const int nb = min(128, ncols - col0);
        if (node >= 0) tc::bulk_wait_read0();   // the previous copy out of this row has read it
        float4* dst = reinterpret_cast<float4*>(myrow);
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          uint32_t v[64];   // both loads in flight, one wait
          const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(128 * acc + 64 * h);
          tc::tmem_ld32_nowait(ta, v);
          tc::tmem_ld32_nowait(ta + 32, v + 32);
          tc::tmem_wait_ld();
          if (h == 1) {   // accumulator read: hand it back to the MMA thread
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tempty(acc));
          }
          if (node >= 0) {
#pragma unroll
            for (int e = 0; e < 16; ++e)
              dst[16 * h + e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                            __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
          }
        }
        if (node >= 0) {
          tc::fence_proxy_async();
          tc::bulk_s2g(Yr + node * (long long)ncols + col0, myrow_s, (uint32_t)nb * 4u);
          tc::bulk_commit();
        }
      }
    }
    tc::bulk_wait0();
  }
  // ---- teardown: after an expired wait, bounded waits for the copies and MMAs
  // still in flight before the TMEM is freed and the CTA exits
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) {
    for (int u = prog[1]; u < prog[0]; ++u) tc::mbar_wait_bounded(full(u & 1), (u >> 1) & 1);
    if (prog[1] > 0) tc::mbar_wait_bounded(empty((prog[1] - 1) & 1), ((prog[1] - 1) >> 1) & 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, 256);
}

template <int NB>
cudaError_t run_tc_project(const ProjDev& pj, const float2* X, int nvec, int ldx, float2* Cbuf,
                           cudaStream_t s, long long M) {
  auto k = k_tc_project<NB>;
  constexpr size_t smem = project_smem<NB>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned ntile = (unsigned)((4 * ldx + kCT - 1) / kCT);
  for (int c0 = 0; c0 < pj.nchunks; c0 += kMaxGridY) {
    dim3 grid(ntile, (unsigned)std::min(kMaxGridY, pj.nchunks - c0));
    k<<<grid, 128, smem, s>>>(reinterpret_cast<const float*>(X), ldx, nvec, pj.d_chunks,
                              pj.d_nodes, pj.d_P32, pj.d_atom_npj, pj.d_atom_pv_off,
                              pj.d_atom_c_off, Cbuf, c0, M);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

using EncodeTiledFn = PFN_cuTensorMapEncodeTiled_v12000;
EncodeTiledFn encode_tiled() {
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

// X viewed as a 2-D tensor [M rows][4 ldx floats]; box = 128 floats x 1 row
bool make_x_map(CUtensorMap* map, const float2* X, long long M, int ldx) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(4 * (long long)ldx), (cuuint64_t)M};
  const cuuint64_t strides[1] = {(cuuint64_t)(4 * (long long)ldx) * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kCT, 1};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(X), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NB>
cudaError_t run_tc_project_tma(const ProjDev& pj, const CUtensorMap& map, int nvec, int ldx,
                               float2* Cbuf, cudaStream_t s) {
  auto k = k_tc_project_tma<NB>;
  constexpr size_t smem = project_tma_smem<NB>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned ntile = (unsigned)((4 * ldx + kCT - 1) / kCT);
  for (int c0 = 0; c0 < pj.nchunks; c0 += kMaxGridY) {
    dim3 grid(ntile, (unsigned)std::min(kMaxGridY, pj.nchunks - c0));
    k<<<grid, kPrjThreads, smem, s>>>(map, ldx, nvec, pj.d_chunks, pj.d_nodes, pj.d_P32, pj.d_atom_npj,
                              pj.d_atom_pv_off, pj.d_atom_c_off, Cbuf, c0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

bool tc_nonlocal_supported(const ProjDev& pj) {
  return pj.natoms > 0 && pj.max_npj <= 64 && pj.ntc_exp > 0 &&
         pj.tc_max_slots <= GBC_TC_MAX_SLOTS;
}

cudaError_t launch_tc_project(const ProjDev& pj, long long M, const float2* X, int nvec, int ldx,
                              float2* Cbuf, cudaStream_t s) {
  const int nb = 16 * ((2 * pj.max_npj + 15) / 16);
  // TMA-fed pipeline where the block layout allows it
  if (ldx == nvec && 4 * ldx >= kCT && nb <= 64 && M < (1LL << 31) &&
      (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
    CUtensorMap map;
    if (make_x_map(&map, X, M, ldx)) {
      switch (nb) {
        case 16: return run_tc_project_tma<16>(pj, map, nvec, ldx, Cbuf, s);
        case 32: return run_tc_project_tma<32>(pj, map, nvec, ldx, Cbuf, s);
        case 48: return run_tc_project_tma<48>(pj, map, nvec, ldx, Cbuf, s);
        case 64: return run_tc_project_tma<64>(pj, map, nvec, ldx, Cbuf, s);
        default: break;
      }
    }
  }
  switch (nb) {
    case 16: return run_tc_project<16>(pj, X, nvec, ldx, Cbuf, s, M);
    case 32: return run_tc_project<32>(pj, X, nvec, ldx, Cbuf, s, M);
    case 48: return run_tc_project<48>(pj, X, nvec, ldx, Cbuf, s, M);
    case 64: return run_tc_project<64>(pj, X, nvec, ldx, Cbuf, s, M);
    case 80: return run_tc_project<80>(pj, X, nvec, ldx, Cbuf, s, M);
    case 96: return run_tc_project<96>(pj, X, nvec, ldx, Cbuf, s, M);
    case 112: return run_tc_project<112>(pj, X, nvec, ldx, Cbuf, s, M);
    case 128: return run_tc_project<128>(pj, X, nvec, ldx, Cbuf, s, M);
    default: return cudaErrorInvalidValue;
  }
}

size_t tc_expand_bpre_bytes(const ProjDev& pj, int nvec, int ldx) {
  if (!pj.d_xA || ldx != nvec || nvec <= 0) return 0;
  const size_t ntiles = (size_t)(4 * ldx + 127) / 128;
  return (size_t)pj.natoms * ntiles * kXOp;
}

cudaError_t tc_expand_prepare(ProjDev& pj, cudaStream_t s) {
  if (!tc_nonlocal_supported(pj) || 2 * pj.max_npj > kXK || pj.ntc_slots <= 0) return cudaSuccess;
  if (!pj.d_xA && cudaMalloc(&pj.d_xA, (size_t)pj.ntc_slots * kXOp) != cudaSuccess) {
    cudaGetLastError();   // no room: the expansion keeps staging its operands itself
    pj.d_xA = nullptr;
    return cudaSuccess;
  }
  k_xpack_a<<<(unsigned)pj.ntc_exp, 128, 0, s>>>(pj.d_xA, pj.d_tcexp_chunks, pj.d_tcexp_slots,
                                                 pj.d_own_pos, pj.d_own_xptr, pj.d_own_xinc,
                                                 pj.d_P32, pj.d_atom_npj, pj.d_atom_pv_off);
  return cudaGetLastError();
}

cudaError_t launch_tc_expand(const ProjDev& pj, float2* Y, int nvec, int ldx, const float2* Cp,
                             cudaStream_t s, bool overwrite, void* bpre, unsigned long long* ctr) {
  if (overwrite && bpre && ctr && tc_expand_bpre_bytes(pj, nvec, ldx) > 0) {
    const int ntiles = (4 * ldx + 127) / 128;
    k_xpack_b<<<dim3((unsigned)pj.natoms, (unsigned)ntiles), 128, 0, s>>>(
        reinterpret_cast<float*>(bpre), Cp, ldx, nvec, pj.d_atom_npj, pj.d_atom_c_off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    constexpr size_t smem = xexp_smem();
    e = cudaFuncSetAttribute(k_tc_expand_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min(pj.ntc_exp, gbc_sm_count());
    e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_tc_expand_ws<<<grid, kXThreads, smem, s>>>(reinterpret_cast<float*>(Y), pj.M, 4 * ldx, ntiles, pj.ntc_exp,
                                                 pj.d_tcexp_chunks, pj.d_tcexp_slots, pj.d_own_node,
                                                 pj.d_xA, reinterpret_cast<const float*>(bpre), ctr);
    return cudaGetLastError();
  }
  constexpr size_t smem = expand_smem();
  cudaError_t e =
      cudaFuncSetAttribute(k_tc_expand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned ntile = (unsigned)((4 * ldx + kCT - 1) / kCT);
  for (int c0 = 0; c0 < pj.ntc_exp; c0 += kMaxGridY) {
    dim3 grid(ntile, (unsigned)std::min(kMaxGridY, pj.ntc_exp - c0));
    k_tc_expand<<<grid, 128, smem, s>>>(reinterpret_cast<float*>(Y), ldx, nvec, 2 * pj.max_npj,
                                        pj.d_tcexp_chunks, pj.d_tcexp_slots, pj.d_own_node,
                                        pj.d_own_pos, pj.d_own_xptr, pj.d_own_xinc, pj.d_P32,
                                        pj.d_atom_npj, pj.d_atom_pv_off, pj.d_atom_c_off, Cp, c0,
                                        overwrite ? 1 : 0, pj.M);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {
// one warp waits on an mbarrier that nothing arrives at, with the caller's
// iteration cap, and reports the expiry exactly as the nonlocal kernels do
__global__ void k_wait_selftest(uint32_t max_iter) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar), 1);
    tc::fence_mbar_init();
  }
  __syncwarp();
  const bool ok = tc::mbar_wait_bounded(tc::smem_u32(&bar), 0, max_iter);
  if (!ok && threadIdx.x == 0) atomicExch(&g_nltc_err, 1);
}
}  // namespace

extern "C" gbc_status gbc_tc_wait_selftest(int max_iter, void* stream) {
  if (max_iter < 1 || max_iter > (1 << 20)) return GBC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  k_wait_selftest<<<1, 32, 0, s>>>((uint32_t)max_iter);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return GBC_ECUDA;
  return GBC_OK;
}

// reset / read the bounded-wait flag of the tensor-core nonlocal kernels
cudaError_t tc_nonlocal_reset(cudaStream_t s) {
  static const int zero = 0;
  return cudaMemcpyToSymbolAsync(g_nltc_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
}
cudaError_t tc_nonlocal_error(int* err, cudaStream_t s) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(err, g_nltc_err, sizeof(int), 0,
                                            cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

GBC_CHECK_WORD_ACCESSOR(gbc_check_word_nltc)
