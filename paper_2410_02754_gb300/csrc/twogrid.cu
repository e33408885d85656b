// Two-grid transfer of a spinor block from FE order p_c to p_f (p_f = p_c or
// p_c + 1) on the same mesh (Sec. IV.A, Eq. FEWfnsCMesh: the first SCF
// iterations use N^{h,p-1}, the later ones N^{h,p}).  The order-p_c space lies
// in the order-p_f space, so the coarse FE function is carried over exactly by
// nodal interpolation at the fine GLL nodes:
//
//   X_f[J] = sum_I N^{p_c}_I(r_J) X_c[I],
//
// per cell a tensor product of the 1-D matrix T[j][i] = l^{p_c}_i(x^{p_f}_j),
// applied in three sum-factorised stages.
//
// One CTA per (cell, tile of VT vectors), 128 threads = VT vector lanes x G
// pencil groups, so every global access of a node row is one contiguous
// VT-vector segment (64 bytes: two full 32-byte sectors; the tile is kept this
// small so that six CTAs fit an SM's shared memory and their gathers overlap).
// Per spin: stage the coarse cell in shared memory with asynchronous copies
// (every load of the cell in flight at once, zero-fill for absent nodes),
// x stage -> B, y stage -> A, z stage -> global.  A cell writes only
// the fine nodes it owns (local index < p_f in every direction); with the
// periodic wrap and the Dirichlet faces this writes every free fine node
// exactly once, with no atomics.  HBM-bound: the coarse block is read and the
// fine block written once (shared coarse nodes are re-read from L2).
#include "gbc_internal.h"

namespace {

template <typename T, int NC, int NF> struct TwoGridTab {
  T t[NF][NC];   // l^{p_c}_i(x^{p_f}_j)
};

// asynchronous global -> shared copy of one complex value (8 or 16 bytes);
// src_bytes = 0 writes zeros
template <int N>
__device__ __forceinline__ void cp_async_n(void* dst, const void* src, int src_bytes) {
  static_assert(N == 8 || N == 16, "8- or 16-byte copies");
  if (N == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

template <typename T, int NC, int NF, int VT>
__global__ void __launch_bounds__(128)
k_prolongate(const MeshDev mc, const MeshDev mf, const cplx<T>* __restrict__ Xc, int ldxc,
             cplx<T>* __restrict__ Xf, int ldxf, int nvec, const TwoGridTab<T, NC, NF> tb) {
  using C = cplx<T>;
  constexpr int G = 128 / VT;                          // pencil groups
  constexpr int ASZ = (NC * NC * NC > NF * NF * NC ? NC * NC * NC : NF * NF * NC);
  constexpr int BSZ = NF * NC * NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);               // [ASZ][VT]
  C* B = A + ASZ * VT;                                 // [BSZ][VT]
  const int v = threadIdx.x % VT, grp = threadIdx.x / VT;
  const int e = blockIdx.x;
  const int vec = blockIdx.y * VT + v;
  const bool vok = vec < nvec;
  const int cx = e % mc.ncell[0], cy = (e / mc.ncell[0]) % mc.ncell[1];
  const int cz = e / (mc.ncell[0] * mc.ncell[1]);
  for (int s = 0; s < 2; ++s) {
    // coarse cell nodes (ix fastest) -> A
    for (int i = grp; i < NC * NC * NC; i += G) {
      const int ix = i % NC, iy = (i / NC) % NC, iz = i / (NC * NC);
      const long long I = gbc_node(mc, cx, cy, cz, ix, iy, iz);
      const bool ok = I >= 0 && vok;
      cp_async_n<sizeof(C)>(&A[i * VT + v], ok ? &Xc[(I * 2 + s) * ldxc + vec] : Xc,
                            ok ? (int)sizeof(C) : 0);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;" ::: "memory");
    __syncthreads();
    // x: A [z][y][x] (NC^3) -> B [z][y][xq] (NC^2 NF)
    for (int pid = grp; pid < NC * NC; pid += G) {
      C in[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) in[j] = A[(pid * NC + j) * VT + v];
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        T r = 0, im = 0;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          r += tb.t[q][j] * in[j].x;
          im += tb.t[q][j] * in[j].y;
        }
        B[(pid * NF + q) * VT + v] = cmake<C>(r, im);
      }
    }
    __syncthreads();
    // y: B [z][y][xq] -> A [z][yq][xq] (NC NF^2)
    for (int pid = grp; pid < NF * NC; pid += G) {
      const int xq = pid % NF, z = pid / NF;
      C in[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) in[j] = B[((z * NC + j) * NF + xq) * VT + v];
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        T r = 0, im = 0;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          r += tb.t[q][j] * in[j].x;
          im += tb.t[q][j] * in[j].y;
        }
        A[((z * NF + q) * NF + xq) * VT + v] = cmake<C>(r, im);
      }
    }
    __syncthreads();
    // z: A [z][yq][xq] -> owned fine nodes (xq, yq, zq < p_f)
    for (int pid = grp; pid < (NF - 1) * (NF - 1); pid += G) {
      const int xq = pid % (NF - 1), yq = pid / (NF - 1);
      C in[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) in[j] = A[((j * NF + yq) * NF + xq) * VT + v];
#pragma unroll
      for (int q = 0; q < NF - 1; ++q) {
        T r = 0, im = 0;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          r += tb.t[q][j] * in[j].x;
          im += tb.t[q][j] * in[j].y;
        }
        const long long J = gbc_node(mf, cx, cy, cz, xq, yq, q);
        if (J >= 0 && vok) Xf[(J * 2 + s) * ldxf + vec] = cmake<C>(r, im);
      }
    }
    __syncthreads();   // A is restaged by the next spin
  }
}

template <typename T, int NC, int NF> constexpr int vt_of() { return sizeof(T) == 4 ? 8 : 4; }

template <typename T, int NC, int NF> constexpr size_t prolongate_smem() {
  constexpr int VT = vt_of<T, NC, NF>();
  constexpr int ASZ = (NC * NC * NC > NF * NF * NC ? NC * NC * NC : NF * NF * NC);
  return sizeof(cplx<T>) * (size_t)VT * (ASZ + NF * NC * NC);
}

template <typename T, int NC, int NF>
cudaError_t launch_prolongate_t(const gbc_ctx* cc, const gbc_ctx* cf, const cplx<T>* Xc, int ldxc,
                                cplx<T>* Xf, int ldxf, int nvec, cudaStream_t s) {
  constexpr int VT = vt_of<T, NC, NF>();
  TwoGridTab<T, NC, NF> tb;   // coarse Lagrange basis at the fine GLL nodes
  const std::vector<double>& xc = cc->tab.gll_x;
  const std::vector<double>& xf = cf->tab.gll_x;
  for (int j = 0; j < NF; ++j)
    for (int i = 0; i < NC; ++i) {
      double l = 1.0;
      for (int k = 0; k < NC; ++k)
        if (k != i) l *= (xf[j] - xc[k]) / (xc[i] - xc[k]);
      tb.t[j][i] = (T)l;
    }
  constexpr size_t smem = prolongate_smem<T, NC, NF>();
  auto k = k_prolongate<T, NC, NF, VT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(cf->mesh.E, (nvec + VT - 1) / VT);
  k<<<grid, 128, smem, s>>>(cc->mesh, cf->mesh, Xc, ldxc, Xf, ldxf, nvec, tb);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolongate(const gbc_ctx* cc, const gbc_ctx* cf, const void* Xc, int ldxc,
                              void* Xf, int ldxf, int nvec, cudaStream_t s) {
  const int pc = cc->mesh.p, pf = cf->mesh.p;
  const cplx<T>* xc = (const cplx<T>*)Xc;
  cplx<T>* xf = (cplx<T>*)Xf;
#define GBC_TG(PC, PF) \
  if (pc == PC && pf == PF) return launch_prolongate_t<T, PC + 1, PF + 1>(cc, cf, xc, ldxc, xf, ldxf, nvec, s);
  GBC_TG(2, 2) GBC_TG(2, 3) GBC_TG(3, 3) GBC_TG(3, 4) GBC_TG(4, 4) GBC_TG(4, 5)
  GBC_TG(5, 5) GBC_TG(5, 6) GBC_TG(6, 6) GBC_TG(6, 7) GBC_TG(7, 7)
#undef GBC_TG
  return cudaErrorInvalidValue;
}

}  // namespace

extern "C" gbc_status gbc_prolongate(gbc_ctx* coarse, gbc_ctx* fine, const void* Xc, int ldxc,
                                     void* Xf, int ldxf, int nvec, void* stream) {
  if (!coarse || !fine) return GBC_EINVAL;
  if (!Xc || !Xf) return gbc_fail(fine, GBC_EINVAL, "null block pointer");
  if (Xc == Xf) return gbc_fail(fine, GBC_EINVAL, "Xc and Xf must be distinct");
  if (!gbc_is_device_ptr(Xc) || !gbc_is_device_ptr(Xf))
    return gbc_fail(fine, GBC_EINVAL, "Xc and Xf must be device memory");
  if (nvec < 1 || ldxc < nvec || ldxf < nvec)
    return gbc_fail(fine, GBC_EINVAL, "need 1 <= nvec <= ldxc, ldxf");
  if (!coarse->mesh_set || !fine->mesh_set) return gbc_fail(fine, GBC_ESTATE, "mesh not set");
  if (coarse->dev != fine->dev) return gbc_fail(fine, GBC_EINVAL, "contexts on different devices");
  if (coarse->prec != fine->prec) return gbc_fail(fine, GBC_EINVAL, "precisions differ");
  for (int d = 0; d < 3; ++d)
    if (coarse->mesh.ncell[d] != fine->mesh.ncell[d] || coarse->h[d] != fine->h[d] ||
        coarse->mesh.periodic[d] != fine->mesh.periodic[d])
      return gbc_fail(fine, GBC_EINVAL, "coarse and fine contexts must share the mesh");
  const int pc = coarse->mesh.p, pf = fine->mesh.p;
  if (pf != pc && pf != pc + 1)
    return gbc_fail(fine, GBC_EUNSUPPORTED, "this build transfers p -> p or p -> p + 1");
  if (coarse->tab.gll_x.size() != (size_t)pc + 1 || fine->tab.gll_x.size() != (size_t)pf + 1)
    return gbc_fail(fine, GBC_ESTATE, "GLL tables not built");
  GBC_CU(fine, cudaSetDevice(fine->dev));
  cudaStream_t s = (cudaStream_t)stream;
  if (fine->prec == GBC_FP64)
    GBC_CU(fine, launch_prolongate<double>(coarse, fine, Xc, ldxc, Xf, ldxf, nvec, s));
  else
    GBC_CU(fine, launch_prolongate<float>(coarse, fine, Xc, ldxc, Xf, ldxf, nvec, s));
  return GBC_OK;
}
