// Cell-level apply of the local spinor Hamiltonian for FP32 blocks, with an
// optional fused Chebyshev recurrence epilogue.
//
// Paper: Sec. IV.B.2 (extract X^(e) = R^(e) X, cell products, assemble
// Y = sum_e R^(e)T Y^(e)) for the cell operator of Eq. FEHlocEl plus the k-terms
// of Eq. FEHloc (per-cell Hermitian form), and Eq. chebfilt for the recurrence.
// The arithmetic is the sum factorisation of the FP64 kernel (hx_local.cuh):
// kinetic/k part K = G_x B_y B_z + B_x G_y B_z + B_x B_y G_z, potential part
// N^T diag(w_q J [(V + |k|^2/2) I + B . sigma]) N, every 1-D operator in even-odd
// form.  What differs is how it maps to the SM:
//
//  * complex values are float2 (re, im) and every real-matrix x complex-vector
//    product is a paired FP32 multiply-add (one instruction for both parts);
//  * per vector only three shared buffers: A (the gathered X^(e), n_p^3 nodes),
//    T2 (n_p^3) and T1 (n_q^3 points), reused in place through the stages
//      gather  X -> A
//      Kz      A  -> T1 = B_z X, T2 = G_z X                     (z pencils)
//      Ky      T1, T2 -> U1 = B_y T1, U2 = G_y T1 + B_y T2      (y pencils, in place)
//      Kx+Ix   U1, U2, A -> T2 = G_x U1 + B_x U2 (kinetic result),
//              T1 = N_x X                                       (x pencils, in place)
//      Iy      T1 -> N_y T1                                     (y pencils, in place)
//      Iz+W+Tz T1 -> N_z^T W N_z T1 with the 2x2 spin operator W at each point
//              (z pencils; the two spins of a pencil on neighbouring lanes)
//      Ty      T1 -> N_y^T T1                                   (y pencils, in place)
//      Tx+out  T1 -> N_x^T T1 + T2, assembled                   (x pencils)
//  * VB vectors per CTA, the vector index fastest across threads, so the gather
//    and the scatter touch VB consecutive complex values of each node row; the
//    gather of the next work item is issued (cp.async) as soon as A is free, so
//    its latency hides behind the last four stages of the current item.
//
// Assembly modes (per system):
//  * accumulate: Y += H^loc X with FP32 atomics on every node;
//  * recurrence: for nodes interior to the cell (owned by it alone) the cell
//    holds the complete local row, so the Chebyshev update is applied here:
//      X_out = a (M_D^-1 (Y + y_loc) - c X) - b X_prev
//    (Y holds the nonlocal term P C' of that row, written before this kernel,
//    or zero); nodes on cell faces are accumulated into Y with atomics and
//    finished by a separate row pass (launch_cheb_rows).
#pragma once

#include "hx_local.cuh"

namespace gbc {

// 1-D operator in even-odd form with every entry duplicated into a float2, the
// multiplier of a paired multiply-add on (re, im)
template <int NO, int NI> struct EO2 {
  static constexpr int HO = (NO + 1) / 2;
  static constexpr int HI = NI / 2 > 0 ? NI / 2 : 1;
  float2 E[HO][HI];
  float2 O[HO][HI];
  float2 Mid[HO];
};

// PACKED: entries duplicated for paired multiply-adds; otherwise plain FP32
// entries for two scalar multiply-adds (re, im) that take the entry straight
// from the constant bank
template <int NP, int NQ, bool PACKED> struct CellTables {
  template <int NO, int NI>
  using M = typename std::conditional<PACKED, EO2<NO, NI>, EO<float, NO, NI>>::type;
  M<NP, NP> B[3];    // 1-D Gauss mass
  M<NP, NP> Gr[3];   // 1/2 A_d
  M<NP, NP> Gi[3];   // -1/2 k_d (C^ - C^T)
  M<NQ, NP> Ni;      // interpolation to the Gauss points
  M<NP, NQ> Nt;      // testing back to the nodes
};

// One system of a launch.
struct CellSys {
  const float2* X;      // block applied to
  float2* Y;            // accumulator
  const float* fields;  // [E][NQ^3][4] w_q J (V + |k|^2/2), w_q J B_x, B_y, B_z
  float2* Xout;         // recurrence mode: X_{k+1} (may alias Xprev)
  const float2* Xprev;  // recurrence mode: X_{k-1}, or null on the first step
  const float* invmd;   // recurrence mode: 1 / M_D per node
  float ca, cc, cb;     // recurrence mode: X_{k+1} = ca (M_D^-1 Y - cc X) - cb X_{k-1}
  int ldx, nvec, vchunks, cheb;
  long long item0;      // work items [item0, item0 + E * vchunks)
  MeshDev mesh;
};

struct CellArgs {
  CellSys sys[GBC_MAX_SYS];
  int nsys;
  long long nitems;
};

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, exactly (the fused product -1 * b is exact)
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) {
  return __ffma2_rn(make_float2(-1.f, -1.f), b, a);
}
__device__ __forceinline__ float2 p_mul(float2 m, float2 x) { return __fmul2_rn(m, x); }
__device__ __forceinline__ float2 p_fma(float2 m, float2 x, float2 acc) {
  return __ffma2_rn(m, x, acc);
}
__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

// 8-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// y = M x for a centro-symmetric (S = 1) or centro-antisymmetric (S = -1) M
template <int S, int NO, int NI>
__device__ __forceinline__ void eo2_apply(const EO2<NO, NI>& M, const float2 (&x)[NI],
                                          float2 (&y)[NO]) {
  constexpr int HI = NI / 2, HO = (NO + 1) / 2;
  static_assert(HI >= 1, "NI >= 2");
  float2 e[HI], o[HI];
#pragma unroll
  for (int j = 0; j < HI; ++j) {
    e[j] = p_add(x[j], x[NI - 1 - j]);
    o[j] = p_sub(x[j], x[NI - 1 - j]);
  }
#pragma unroll
  for (int i = 0; i < HO; ++i) {
    float2 ae = p_mul(M.E[i][0], e[0]);
    float2 ao = p_mul(M.O[i][0], o[0]);
#pragma unroll
    for (int j = 1; j < HI; ++j) {
      ae = p_fma(M.E[i][j], e[j], ae);
      ao = p_fma(M.O[i][j], o[j], ao);
    }
    if (NI & 1) ae = p_fma(M.Mid[i], x[HI], ae);
    y[i] = p_add(ae, ao);
    if (NO - 1 - i != i) y[NO - 1 - i] = S > 0 ? p_sub(ae, ao) : p_sub(ao, ae);
  }
}

// the same with plain FP32 entries: two scalar multiply-adds per complex product
template <int S, int NO, int NI>
__device__ __forceinline__ void eo2_apply(const EO<float, NO, NI>& M, const float2 (&x)[NI],
                                          float2 (&y)[NO]) {
  constexpr int HI = NI / 2, HO = (NO + 1) / 2;
  static_assert(HI >= 1, "NI >= 2");
  float2 e[HI], o[HI];
#pragma unroll
  for (int j = 0; j < HI; ++j) {
    e[j] = make_float2(x[j].x + x[NI - 1 - j].x, x[j].y + x[NI - 1 - j].y);
    o[j] = make_float2(x[j].x - x[NI - 1 - j].x, x[j].y - x[NI - 1 - j].y);
  }
#pragma unroll
  for (int i = 0; i < HO; ++i) {
    float er = M.E[i][0] * e[0].x, ei = M.E[i][0] * e[0].y;
    float orr = M.O[i][0] * o[0].x, oi = M.O[i][0] * o[0].y;
#pragma unroll
    for (int j = 1; j < HI; ++j) {
      er = fmaf(M.E[i][j], e[j].x, er);
      ei = fmaf(M.E[i][j], e[j].y, ei);
      orr = fmaf(M.O[i][j], o[j].x, orr);
      oi = fmaf(M.O[i][j], o[j].y, oi);
    }
    if (NI & 1) {
      er = fmaf(M.Mid[i], x[HI].x, er);
      ei = fmaf(M.Mid[i], x[HI].y, ei);
    }
    y[i] = make_float2(er + orr, ei + oi);
    if (NO - 1 - i != i)
      y[NO - 1 - i] = S > 0 ? make_float2(er - orr, ei - oi) : make_float2(orr - er, oi - ei);
  }
}

// y = (Gr + i Gi) x, Gr symmetric, Gi antisymmetric (Gi only at k != 0)
template <bool KPT, int N, typename MT>
__device__ __forceinline__ void g2_apply(const MT& Gr, const MT& Gi, const float2 (&x)[N],
                                         float2 (&y)[N]) {
  eo2_apply<1>(Gr, x, y);
  if (KPT) {
    float2 t[N];
    eo2_apply<-1>(Gi, x, t);
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = make_float2(y[i].x - t[i].y, y[i].y + t[i].x);
  }
}

// Point strides (y, z) of the n_p^3 buffers (A, T2) and of the n_q^3 buffer (T1).
// With the unit order of the stages (vector fastest, then spin, then pencil) a
// half-warp touches 4 pencils x 2 spins x 2 vectors; these strides put those 16
// 8-byte accesses in 16 distinct bank pairs for every stage's pencil direction
// (found by enumerating strides against a model of the 64-bit shared-memory
// wavefronts); the n_p^3 buffers are dense for odd n_p.
template <int NP> struct CellLayout;
template <> struct CellLayout<3> { static constexpr int AY = 3, AZ = 9, QY = 5, QZ = 23; };
template <> struct CellLayout<4> { static constexpr int AY = 5, AZ = 21, QY = 5, QZ = 25; };
template <> struct CellLayout<5> { static constexpr int AY = 5, AZ = 25, QY = 9, QZ = 57; };
template <> struct CellLayout<6> { static constexpr int AY = 7, AZ = 43, QY = 7, QZ = 51; };
template <> struct CellLayout<7> { static constexpr int AY = 7, AZ = 49, QY = 9, QZ = 75; };
template <> struct CellLayout<8> { static constexpr int AY = 9, AZ = 73, QY = 9, QZ = 81; };
template <int NP> __host__ __device__ constexpr int cell_bufa() {   // points of A / T2
  return (NP - 1) * (1 + CellLayout<NP>::AY + CellLayout<NP>::AZ) + 1;
}
template <int NP> __host__ __device__ constexpr int cell_bufq() {   // points of T1
  return NP * (1 + CellLayout<NP>::QY + CellLayout<NP>::QZ) + 1;
}

template <int NP, int NQ, int VB> __host__ __device__ constexpr int cell_vstride() {
  // float2 elements per vector: [A | T2 | T1], two spins per point, padded so that the
  // VB vectors of a lane group start in distinct quarters (VB = 4: 4 mod 16) or halves
  // (VB = 2: 8 mod 16) of a 128-byte bank row (the same wavefront model as the strides)
  static_assert(VB == 2 || VB == 4, "VB");
  constexpr int n = 2 * (2 * cell_bufa<NP>() + cell_bufq<NP>());
  constexpr int r = VB == 4 ? 4 : 8;
  return n + ((16 + r - n % 16) % 16);
}
// vector buffers, then the node-offset tables of the current and the next work item
template <int NP, int NQ, int VB> constexpr size_t hx_cell_smem() {
  return sizeof(float2) * (size_t)VB * cell_vstride<NP, NQ, VB>() + sizeof(int) * 2 * 3 * NP + 16;
}
constexpr int kNoNode = -(1 << 29);   // offset of a direction with no free node (Dirichlet face)

// The work items [0, nitems) of the systems sys[0 .. nsys) (item0 ascending), taken
// from the counter *ctr (zero at launch) one atomic increment at a time, so CTAs
// that finish early take more and the items in flight stay close to each other in
// the order (cell-major, vector chunks of a cell adjacent).
template <int NP, int NQ, bool KPT, int VB, int NT, bool PACKED>
__device__ __forceinline__ void cell_body(const CellSys* __restrict__ sys, int nsys,
                                          long long nitems, const CellTables<NP, NQ, PACKED>& tb,
                                          unsigned long long* __restrict__ ctr) {
  constexpr int BA = cell_bufa<NP>();
  constexpr int NQ3 = NQ * NQ * NQ;
  constexpr int VS = cell_vstride<NP, NQ, VB>();
  using L = CellLayout<NP>;
  extern __shared__ __align__(16) float2 sm[];
  // spin s of point pidx of vector v: Buf(v)[2 * pidx + s]
  auto Ab = [&](int v) { return sm + v * VS; };
  auto T2b = [&](int v) { return sm + v * VS + 2 * BA; };
  auto T1b = [&](int v) { return sm + v * VS + 4 * BA; };
  auto pa = [](int x, int y, int z) { return x + y * L::AY + z * L::AZ; };
  auto pq = [](int x, int y, int z) { return x + y * L::QY + z * L::QZ; };
  const int tid = threadIdx.x;
  auto locate = [&](long long it) {
    int q = 0;
    if (nsys == 1) return q;   // one system: skip the scan over the descriptor slots
#pragma unroll
    for (int r = 1; r < GBC_MAX_SYS; ++r)
      if (r < nsys && it >= sys[r].item0) q = r;
    return q;
  };

  // node index of local node (ix, iy, iz) of a work item's cell:
  // noff[b][0][ix] + noff[b][1][iy] + noff[b][2][iz], negative where the node is
  // on a Dirichlet face; b alternates between the current and the next item
  int* noff = reinterpret_cast<int*>(sm + VB * VS);
  auto offsets = [&](long long it, int b) {
    if (tid < 3 * NP) {
      const CellSys& g = sys[locate(it)];
      const int e = (int)((it - g.item0) / g.vchunks);
      const int dd = tid / NP, i = tid % NP;
      const int c = dd == 0 ? e % g.mesh.ncell[0]
                  : dd == 1 ? (e / g.mesh.ncell[0]) % g.mesh.ncell[1]
                            : e / (g.mesh.ncell[0] * g.mesh.ncell[1]);
      const int gc = c * g.mesh.p + i;
      int f;
      if (g.mesh.periodic[dd]) {
        f = gc >= g.mesh.period[dd] ? gc - g.mesh.period[dd] : gc;
      } else {
        f = (gc == 0 || gc == g.mesh.period[dd]) ? -1 : gc - 1;
      }
      const int scale = dd == 0 ? 1 : dd == 1 ? g.mesh.nfree[0] : g.mesh.nfree[0] * g.mesh.nfree[1];
      noff[b * 3 * NP + tid] = f < 0 ? kNoNode : f * scale;
    }
  };
  // asynchronous gather of X^(e) of work item ``it`` into A: thread -> (vector,
  // spin, node), vector fastest; absent nodes (Dirichlet faces) and vectors
  // beyond nvec are zero-filled
  auto gather = [&](long long it, int b) {
    const CellSys& g = sys[locate(it)];
    const int vb0 = (int)((it - g.item0) % g.vchunks) * VB;
    const int* no = noff + b * 3 * NP;
    for (int i = tid; i < VB * 2 * NP * NP * NP; i += NT) {
      const int v = i % VB, r = i / VB, s = r & 1, n = r >> 1;
      const int ix = n % NP, iy = (n / NP) % NP, iz = n / (NP * NP);
      const int I = no[ix] + no[NP + iy] + no[2 * NP + iz];
      const bool ok = I >= 0 && vb0 + v < g.nvec && GBC_IN_RANGE(GBC_SITE_CELL_GATHER, I, g.mesh.M);
      cp_async8(&Ab(v)[2 * pa(ix, iy, iz) + s],
                ok ? &g.X[((long long)I * 2 + s) * g.ldx + vb0 + v] : g.X, ok ? 8 : 0);
    }
    cp_async_commit();
  };

  // the next item's index; tid 0 writes it before a barrier that every thread
  // passes after its last read of the previous value (the stage barriers below)
  long long* s_next = reinterpret_cast<long long*>(noff + 2 * 3 * NP);
  if (tid == 0) *s_next = (long long)atomicAdd(ctr, 1ULL);
  __syncthreads();
  const long long first = *s_next;
  __syncthreads();
  if (first < nitems) {
    offsets(first, 0);
    __syncthreads();
    gather(first, 0);
  }
  int buf = 0;
  long long next = first;
  for (long long item = first; item < nitems; item = next, buf ^= 1) {
    const CellSys& d = sys[locate(item)];
    const long long li = item - d.item0;
    const int e = (int)(li / d.vchunks);
    const int vbase = (int)(li % d.vchunks) * VB;
    const int* no = noff + buf * 3 * NP;
    if (tid == 0) *s_next = (long long)atomicAdd(ctr, 1ULL);
    cp_async_wait_all();
    __syncthreads();
    next = *s_next;
    if (next < nitems) offsets(next, buf ^ 1);   // read after the next two barriers

    // ---- Kz: T1 = B_z X, T2 = G_z X
    for (int u = tid; u < VB * 2 * NP * NP; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int x = pen % NP, y = pen / NP;
      float2 in[NP], t1[NP], t2[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = Ab(v)[2 * pa(x, y, j) + s];
      eo2_apply<1>(tb.B[2], in, t1);
      g2_apply<KPT>(tb.Gr[2], tb.Gi[2], in, t2);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T1b(v)[2 * pq(x, y, i) + s] = t1[i];
        T2b(v)[2 * pa(x, y, i) + s] = t2[i];
      }
    }
    __syncthreads();

    // ---- Ky (in place): U1 = B_y T1, U2 = G_y T1 + B_y T2
    for (int u = tid; u < VB * 2 * NP * NP; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int x = pen % NP, z = pen / NP;
      float2 t1[NP], t2[NP], u1[NP], u2[NP], w2[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        t1[j] = T1b(v)[2 * pq(x, j, z) + s];
        t2[j] = T2b(v)[2 * pa(x, j, z) + s];
      }
      eo2_apply<1>(tb.B[1], t1, u1);
      g2_apply<KPT>(tb.Gr[1], tb.Gi[1], t1, u2);
      eo2_apply<1>(tb.B[1], t2, w2);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T1b(v)[2 * pq(x, i, z) + s] = u1[i];
        T2b(v)[2 * pa(x, i, z) + s] = p_add(u2[i], w2[i]);
      }
    }
    __syncthreads();

    // ---- Kx + Ix (in place, x pencils): T2 = G_x U1 + B_x U2, T1 = N_x X
    for (int u = tid; u < VB * 2 * NP * NP; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int y = pen % NP, z = pen / NP;
      {
        float2 u1[NP], u2[NP], yk[NP], w2[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          u1[j] = T1b(v)[2 * pq(j, y, z) + s];
          u2[j] = T2b(v)[2 * pa(j, y, z) + s];
        }
        g2_apply<KPT>(tb.Gr[0], tb.Gi[0], u1, yk);
        eo2_apply<1>(tb.B[0], u2, w2);
#pragma unroll
        for (int i = 0; i < NP; ++i) T2b(v)[2 * pa(i, y, z) + s] = p_add(yk[i], w2[i]);
      }
      {
        float2 in[NP], out[NQ];
#pragma unroll
        for (int j = 0; j < NP; ++j) in[j] = Ab(v)[2 * pa(j, y, z) + s];
        eo2_apply<1>(tb.Ni, in, out);
#pragma unroll
        for (int q = 0; q < NQ; ++q) T1b(v)[2 * pq(q, y, z) + s] = out[q];
      }
    }
    __syncthreads();
    // A is free from here on: start the next item's gather behind the remaining stages
    if (next < nitems) gather(next, buf ^ 1);

    // ---- Iy (in place): T1 (nq, np, np) -> (nq, nq, np)
    for (int u = tid; u < VB * 2 * NQ * NP; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int x = pen % NQ, z = pen / NQ;
      float2 in[NP], out[NQ];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = T1b(v)[2 * pq(x, j, z) + s];
      eo2_apply<1>(tb.Ni, in, out);
#pragma unroll
      for (int q = 0; q < NQ; ++q) T1b(v)[2 * pq(x, q, z) + s] = out[q];
    }
    __syncthreads();

    // ---- Iz + spin operator + Tz (z pencils, in place); spin fastest, so the
    // two spins of a pencil sit on neighbouring lanes and swap values by shuffle
    {
      const float* __restrict__ fld = d.fields + (size_t)e * 4 * NQ3;
      constexpr int UNITS = VB * 2 * NQ * NQ;
      constexpr int ROUNDS = (UNITS + NT - 1) / NT;
#pragma unroll 1
      for (int r = 0; r < ROUNDS; ++r) {
        const int uu = tid + r * NT;
        const bool act = uu < UNITS;
        const int u = act ? uu : (uu & 1);
        const int s = u & 1, v = (u >> 1) % VB, pen = (u >> 1) / VB;
        const int x = pen % NQ, y = pen / NQ;
        float2 in[NP], own[NQ];
#pragma unroll
        for (int j = 0; j < NP; ++j) in[j] = T1b(v)[2 * pq(x, y, j) + s];
        eo2_apply<1>(tb.Ni, in, own);
        const float sg = s ? -1.f : 1.f;
        float2 w[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          float2 oth;
          oth.x = __shfl_xor_sync(0xffffffffu, own[q].x, 1);
          oth.y = __shfl_xor_sync(0xffffffffu, own[q].y, 1);
          const int qq = (q * NQ + y) * NQ + x;
          const float4 F = __ldg(reinterpret_cast<const float4*>(fld) + qq);
          const float V = F.x, bx = F.y, by = F.z, bz = F.w;
          // up:   (V + bz) u + bx d + by (d.y, -d.x)
          // down: (V - bz) d + bx u - by (u.y, -u.x)
          float2 o = p_mul(dup(V + sg * bz), own[q]);
          o = p_fma(dup(bx), oth, o);
          w[q] = p_fma(make_float2(sg * by, -sg * by), make_float2(oth.y, oth.x), o);
        }
        float2 out[NP];
        eo2_apply<1>(tb.Nt, w, out);
        if (act) {
#pragma unroll
          for (int i = 0; i < NP; ++i) T1b(v)[2 * pq(x, y, i) + s] = out[i];
        }
      }
    }
    __syncthreads();

    // ---- Ty (in place): T1 (nq, nq, np) -> (nq, np, np)
    for (int u = tid; u < VB * 2 * NQ * NP; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int x = pen % NQ, z = pen / NQ;
      float2 in[NQ], out[NP];
#pragma unroll
      for (int q = 0; q < NQ; ++q) in[q] = T1b(v)[2 * pq(x, q, z) + s];
      eo2_apply<1>(tb.Nt, in, out);
#pragma unroll
      for (int i = 0; i < NP; ++i) T1b(v)[2 * pq(x, i, z) + s] = out[i];
    }
    __syncthreads();

    // ---- Tx, add the kinetic part, assemble (vector fastest across threads)
    for (int u = tid; u < VB * 2 * NP * NP; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int y = pen % NP, z = pen / NP;
      const int vec = vbase + v;
      float2 in[NQ], out[NP];
#pragma unroll
      for (int q = 0; q < NQ; ++q) in[q] = T1b(v)[2 * pq(q, y, z) + s];
      eo2_apply<1>(tb.Nt, in, out);
      if (vec >= d.nvec) continue;
      const bool yz_in = y > 0 && y < NP - 1 && z > 0 && z < NP - 1;
      const int Iyz = no[NP + y] + no[2 * NP + z];
#pragma unroll
      for (int i = 0; i < NP; ++i) out[i] = p_add(out[i], T2b(v)[2 * pa(i, y, z) + s]);
      if (d.cheb && yz_in) {
        // nodes x = 1 .. NP-2 of this pencil are interior to the cell: every load is
        // issued before the first update (X_out may alias X_prev), so their latencies
        // overlap
        constexpr int NIN = NP - 2;
        float2 yv[NIN], xv[NIN], pv[NIN];
        float wv[NIN];
#pragma unroll
        for (int j = 0; j < NIN; ++j) {
          const int I = Iyz + no[1 + j];
          const long long o = ((long long)I * 2 + s) * d.ldx + vec;
          if (GBC_IN_RANGE(GBC_SITE_CELL_STORE, I, d.mesh.M)) {
            yv[j] = d.Y[o];
            xv[j] = __ldg(&d.X[o]);
            wv[j] = __ldg(d.invmd + I);
            pv[j] = d.Xprev ? d.Xprev[o] : make_float2(0.f, 0.f);
          } else {
            yv[j] = xv[j] = pv[j] = make_float2(0.f, 0.f);
            wv[j] = 0.f;
          }
        }
#pragma unroll
        for (int j = 0; j < NIN; ++j) {
          const int I = Iyz + no[1 + j];
          const long long o = ((long long)I * 2 + s) * d.ldx + vec;
          const float2 yt = p_add(yv[j], out[1 + j]);
          const float2 xn = p_fma(dup(-d.cb), pv[j],
                                  p_mul(dup(d.ca), p_fma(dup(-d.cc), xv[j], p_mul(dup(wv[j]), yt))));
          if (GBC_IN_RANGE(GBC_SITE_CELL_STORE, I, d.mesh.M)) d.Xout[o] = xn;
        }
#pragma unroll
        for (int i = 0; i < NP; i += NP - 1) {   // the pencil's two face nodes
          const int I = Iyz + no[i];
          if (I >= 0 && GBC_IN_RANGE(GBC_SITE_CELL_STORE, I, d.mesh.M))
            atomicAdd(&d.Y[((long long)I * 2 + s) * d.ldx + vec], out[i]);
        }
      } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          const int I = Iyz + no[i];
          if (I >= 0 && GBC_IN_RANGE(GBC_SITE_CELL_STORE, I, d.mesh.M))
            atomicAdd(&d.Y[((long long)I * 2 + s) * d.ldx + vec], out[i]);
        }
      }
    }
  }
}

// One persistent launch over systems that share p, the cell edges and the k-point;
// the CTAs take their work items from the zeroed counter *ctr in ascending order.
template <int NP, int NQ, bool KPT, int VB, int NT, int MINB, bool PACKED>
__global__ void __launch_bounds__(NT, MINB)
hx_cell_kernel(const __grid_constant__ CellArgs a,
               const __grid_constant__ CellTables<NP, NQ, PACKED> tb,
               unsigned long long* __restrict__ ctr) {
  cell_body<NP, NQ, KPT, VB, NT, PACKED>(a.sys, a.nsys, a.nitems, tb, ctr);
}

template <int NO, int NI>
inline void cvt_table(const EO<float, NO, NI>& src, EO<float, NO, NI>& dst) { dst = src; }
template <int NO, int NI>
inline void cvt_table(const EO<float, NO, NI>& src, EO2<NO, NI>& dst) {
  for (int i = 0; i < EO2<NO, NI>::HO; ++i) {
    for (int j = 0; j < EO2<NO, NI>::HI; ++j) {
      dst.E[i][j] = make_float2(src.E[i][j], src.E[i][j]);
      dst.O[i][j] = make_float2(src.O[i][j], src.O[i][j]);
    }
    dst.Mid[i] = make_float2(src.Mid[i], src.Mid[i]);
  }
}

template <int NP, int NQ, bool PACKED>
inline bool make_cell_tables(const gbc_ctx* c, CellTables<NP, NQ, PACKED>* t) {
  TablesEO<float, NP, NQ> f;
  if (!make_tables_eo<float, NP, NQ>(c, &f)) return false;
  for (int d = 0; d < 3; ++d) {
    cvt_table(f.B[d], t->B[d]);
    cvt_table(f.Gr[d], t->Gr[d]);
    cvt_table(f.Gi[d], t->Gi[d]);
  }
  cvt_table(f.Ni, t->Ni);
  cvt_table(f.Nt, t->Nt);
  return true;
}

// descriptor of one system (items numbered from item0)
inline void fill_sys(CellSys& d, const CellJob& j, int vb, long long item0) {
    const gbc_ctx* c = j.c;
    d.X = (const float2*)j.X;
    d.Y = (float2*)j.Y;
    d.fields = c->d_fields32;
    d.Xout = (float2*)j.Xout;
    d.Xprev = (const float2*)j.Xprev;
    d.invmd = c->d_invmd32;
    d.ca = (float)j.a;
    d.cc = (float)j.cshift;
    d.cb = (float)j.b;
    d.cheb = j.Xout != nullptr;
    d.ldx = j.ldx;
    d.nvec = j.nvec;
    d.vchunks = (j.nvec + vb - 1) / vb;
    d.item0 = item0;
    d.mesh = c->mesh;
}

// One launch over up to GBC_MAX_SYS systems sharing p, the cell edges and the
// k-point.
template <int NP, int VB, int NT, int MINB, bool PACKED>
cudaError_t launch_cell_group_p(const CellJob* jobs, int n, cudaStream_t s) {
  constexpr int NQ = NP + 1;   // nq = p + 2
  if (n < 1 || n > GBC_MAX_SYS) return cudaErrorInvalidValue;
  CellArgs a;
  long long item = 0;
  for (int i = 0; i < GBC_MAX_SYS; ++i) {
    CellSys& d = a.sys[i];
    if (i >= n) {
      d = a.sys[0];
      d.item0 = 0x7fffffffffffffffLL;
      continue;
    }
    fill_sys(d, jobs[i], VB, item);
    item += (long long)jobs[i].c->mesh.E * d.vchunks;
  }
  a.nsys = n;
  a.nitems = item;
  if (item <= 0) return cudaSuccess;
  const gbc_ctx* c0 = jobs[0].c;
  CellTables<NP, NQ, PACKED> tb;
  if (!make_cell_tables<NP, NQ, PACKED>(c0, &tb)) return cudaErrorInvalidValue;
  const bool kpt = (c0->k[0] != 0.0 || c0->k[1] != 0.0 || c0->k[2] != 0.0);
  constexpr size_t smem = hx_cell_smem<NP, NQ, VB>();
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  unsigned long long* ctr = c0->d_cell_ctr;   // the first system's work counter
  if (!ctr) return cudaErrorInvalidValue;
  auto run = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long nblk = std::min<long long>(item, (long long)nsm * per_sm);
    e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nblk, NT, smem, s>>>(a, tb, ctr);
    return cudaGetLastError();
  };
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (kpt) return run(hx_cell_kernel<NP, NQ, true, VB, NT, MINB, PACKED>);
  return run(hx_cell_kernel<NP, NQ, false, VB, NT, MINB, PACKED>);
}

template <int VB, int NT, int MINB, bool PACKED>
cudaError_t launch_cell_group(const CellJob* jobs, int n, cudaStream_t s) {
  for (int i = 0; i < n; ++i)   // node offsets are 32-bit
    if (jobs[i].c->mesh.M >= (1LL << 29)) return cudaErrorInvalidValue;
  switch (jobs[0].c->mesh.p) {
    case 2: return launch_cell_group_p<3, VB, NT, MINB, PACKED>(jobs, n, s);
    case 3: return launch_cell_group_p<4, VB, NT, MINB, PACKED>(jobs, n, s);
    case 4: return launch_cell_group_p<5, VB, NT, MINB, PACKED>(jobs, n, s);
    case 5: return launch_cell_group_p<6, VB, NT, MINB, PACKED>(jobs, n, s);
    case 6: return launch_cell_group_p<7, VB, NT, MINB, PACKED>(jobs, n, s);
    case 7: return launch_cell_group_p<8, VB, NT, MINB, PACKED>(jobs, n, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gbc
