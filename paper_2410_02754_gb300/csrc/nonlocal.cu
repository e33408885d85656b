// Nonlocal spin-orbit part of H.X over compact projector supports.
//
// Paper: Eq. FEHnloc and the cell-level step 3 of Sec. IV.B.2,
//   Y += sum_a P_a Delta_a sum P_a^H X,
// done as three batched small contractions on the atom-support node lists:
//   C   = P_a^H X        (per atom: npj x 2 x nvec, reduction over the support)
//   C'  = Delta_a C      (2npj x 2npj times 2npj x nvec)
//   Y  += P_a C'         (node-centric: every support node sums its atoms' terms,
//                         a plain read-modify-write of Y, no atomics)
// P_a is the node-based projector table (one row per distinct free node of the
// support, so nodes shared by several support cells are stored once).
#include <algorithm>
#include <type_traits>

#include "gbc_internal.h"

namespace {

template <typename C> __device__ __forceinline__ void cmac_conj(C& acc, C p, C x) {
  // acc += conj(p) * x
  acc.x += p.x * x.x + p.y * x.y;
  acc.y += p.x * x.y - p.y * x.x;
}
template <typename C> __device__ __forceinline__ void cmac(C& acc, C p, C x) {
  acc.x += p.x * x.x - p.y * x.y;
  acc.y += p.x * x.y + p.y * x.x;
}
__device__ __forceinline__ void catomic(float2* p, float2 v) { atomicAdd(p, v); }
__device__ __forceinline__ void catomic(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

constexpr int kStage = 64;      // support nodes staged in shared memory at a time
constexpr int kCols = 128;      // threads (columns) per block

// C[(c_off + 2chi + s) * nvec + v] += sum_j conj(P[j][chi]) X[node_j][s][v]
template <typename T, int MAXPJ>
__global__ void __launch_bounds__(kCols)
nl_project(const cplx<T>* __restrict__ X, int ldx, int nvec, const int4* __restrict__ chunks,
           const long long* __restrict__ nodes, const cplx<T>* __restrict__ P,
           const int* __restrict__ atom_npj, const int* __restrict__ atom_pv_off,
           const int* __restrict__ atom_c_off, cplx<T>* __restrict__ Cbuf, long long M,
           cplx<T>* __restrict__ Cpart) {
  using C = cplx<T>;
  __shared__ C Ps[kStage][MAXPJ];
  __shared__ long long Ns[kStage];
  const int4 ch = chunks[blockIdx.x];      // (atom, first position, count, node offset of atom)
  const int atom = ch.x, j0 = ch.y, cnt = ch.z, noff = ch.w;
  const int npj = atom_npj[atom];
  const C* Pa = P + atom_pv_off[atom];
  const int col = blockIdx.y * kCols + threadIdx.x;
  const bool ok = col < 2 * nvec;
  const int s = ok ? col / nvec : 0, v = ok ? col % nvec : 0;
  C acc[MAXPJ];
#pragma unroll
  for (int c = 0; c < MAXPJ; ++c) acc[c] = cmake<C>(0, 0);
  for (int jb = 0; jb < cnt; jb += kStage) {
    const int nb = min(kStage, cnt - jb);
    for (int t = threadIdx.x; t < nb * npj; t += kCols) {
      const int jj = t / npj, c = t % npj;
      Ps[jj][c] = Pa[(size_t)(j0 + jb + jj) * npj + c];
    }
    for (int t = threadIdx.x; t < nb; t += kCols) Ns[t] = nodes[noff + j0 + jb + t];
    __syncthreads();
    if (ok) {
      for (int t = 0; t < nb; t += 4) {
        C x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          x[u] = (t + u < nb && GBC_IN_RANGE(GBC_SITE_NL_NODE, Ns[t + u], M))
                     ? X[(Ns[t + u] * 2 + s) * ldx + v] : cmake<C>(0, 0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (t + u >= nb) break;
#pragma unroll
          for (int c = 0; c < MAXPJ; ++c)
            if (c < npj) cmac_conj(acc[c], Ps[t + u][c], x[u]);
        }
      }
    }
    __syncthreads();
  }
  if (ok && Cpart) {   // this chunk's sums, rows 2chi + s (k_nl_chunk_sum adds them in order)
#pragma unroll
    for (int c = 0; c < MAXPJ; ++c)
      if (c < npj) Cpart[((size_t)blockIdx.x * 2 * MAXPJ + 2 * c + s) * nvec + v] = acc[c];
  } else if (ok) {
    const int r0 = atom_c_off[atom];
#pragma unroll
    for (int c = 0; c < MAXPJ; ++c)
      if (c < npj) catomic(&Cbuf[(size_t)(r0 + 2 * c + s) * nvec + v], acc[c]);
  }
}

// C[(c_off + r) * nvec + v] = sum over the atom's chunks k, in order, of Cpart[k][r][v]
template <typename T, int MAXPJ>
__global__ void k_nl_chunk_sum(const cplx<T>* __restrict__ Cpart, cplx<T>* __restrict__ Cbuf,
                               const int* __restrict__ chunk_off, const int* __restrict__ atom_npj,
                               const int* __restrict__ atom_c_off, int nvec) {
  const int atom = blockIdx.x, r = blockIdx.y;
  const int v = blockIdx.z * blockDim.x + threadIdx.x;
  if (r >= 2 * atom_npj[atom] || v >= nvec) return;
  cplx<T> acc = cmake<cplx<T>>(0, 0);
  for (int k = chunk_off[atom]; k < chunk_off[atom + 1]; ++k) {
    const cplx<T> p = Cpart[((size_t)k * 2 * MAXPJ + r) * nvec + v];
    acc.x += p.x;
    acc.y += p.y;
  }
  Cbuf[(size_t)(atom_c_off[atom] + r) * nvec + v] = acc;
}

// Cp[(c_off + r) * nvec + v] = sum_c Delta[r][c] C[(c_off + c) * nvec + v]
template <typename T>
__global__ void nl_couple(const cplx<T>* __restrict__ Cbuf, cplx<T>* __restrict__ Cp,
                          const cplx<T>* __restrict__ delta, const int* __restrict__ atom_npj,
                          const int* __restrict__ atom_delta_off, const int* __restrict__ atom_c_off,
                          int nvec) {
  using C = cplx<T>;
  const int atom = blockIdx.x, r = blockIdx.y;
  const int n2 = 2 * atom_npj[atom];
  if (r >= n2) return;
  const int v = blockIdx.z * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  const C* D = delta + atom_delta_off[atom] + (size_t)r * n2;
  const size_t base = (size_t)atom_c_off[atom] * nvec + v;
  C acc = cmake<C>(0, 0);
  for (int c = 0; c < n2; ++c) cmac(acc, D[c], Cbuf[base + (size_t)c * nvec]);
  Cp[base + (size_t)r * nvec] = acc;
}

// Y[node][s][v] += sum over atoms whose support holds node of sum_chi P[pos][chi] Cp[2chi+s][v].
// Every distinct support node is owned by the lowest-index atom whose support
// holds it; the owner's block writes it once (plain read-modify-write, no
// atomics) and adds the other atoms' terms from their incidence list.  The
// owner's C' column stays in registers, the staged P rows in shared memory.
constexpr int kExpStage = 32;
template <typename T, int MAXPJ>
__global__ void __launch_bounds__(kCols)
nl_expand(cplx<T>* __restrict__ Y, int ldx, int nvec, const int4* __restrict__ chunks,
          const long long* __restrict__ own_node, const int* __restrict__ own_pos,
          const int* __restrict__ own_xptr, const int2* __restrict__ own_xinc,
          const cplx<T>* __restrict__ P, const int* __restrict__ atom_npj,
          const int* __restrict__ atom_pv_off, const int* __restrict__ atom_c_off,
          const cplx<T>* __restrict__ Cp, int overwrite, long long M) {
  using C = cplx<T>;
  __shared__ C Ps[kExpStage][MAXPJ];
  const int4 ch = chunks[blockIdx.x];       // (atom, first owned index, count, -)
  const int atom = ch.x, u0 = ch.y, cnt = ch.z;
  const int npj = atom_npj[atom];
  const C* Pa = P + atom_pv_off[atom];
  const int col = blockIdx.y * kCols + threadIdx.x;
  const bool ok = col < 2 * nvec;
  const int s = ok ? col / nvec : 0, v = ok ? col % nvec : 0;
  C cp[MAXPJ];
  const C* Ca = Cp + (size_t)(atom_c_off[atom] + s) * nvec + v;
#pragma unroll
  for (int c = 0; c < MAXPJ; ++c) cp[c] = (ok && c < npj) ? Ca[(size_t)(2 * c) * nvec] : cmake<C>(0, 0);
  for (int jb = 0; jb < cnt; jb += kExpStage) {
    const int nb = min(kExpStage, cnt - jb);
    for (int t = threadIdx.x; t < nb * npj; t += kCols) {
      const int jj = t / npj, c = t % npj;
      Ps[jj][c] = Pa[(size_t)own_pos[u0 + jb + jj] * npj + c];
    }
    __syncthreads();
    if (ok) {
      for (int t = 0; t < nb; ++t) {
        const int u = u0 + jb + t;
        C acc = cmake<C>(0, 0);
#pragma unroll
        for (int c = 0; c < MAXPJ; ++c)
          if (c < npj) cmac(acc, Ps[t][c], cp[c]);
        for (int k = own_xptr[u]; k < own_xptr[u + 1]; ++k) {
          const int2 inc = own_xinc[k];
          const int nb2 = atom_npj[inc.x];
          const C* Pr = P + atom_pv_off[inc.x] + (size_t)inc.y * nb2;
          const C* Cr = Cp + (size_t)(atom_c_off[inc.x] + s) * nvec + v;
          for (int c = 0; c < nb2; ++c) cmac(acc, Pr[c], Cr[(size_t)(2 * c) * nvec]);
        }
        if (!GBC_IN_RANGE(GBC_SITE_NL_NODE, own_node[u], M)) continue;
        C* y = &Y[(own_node[u] * 2 + s) * ldx + v];
        if (overwrite) {
          *y = acc;
        } else {
          C o = *y;
          o.x += acc.x;
          o.y += acc.y;
          *y = o;
        }
      }
    }
    __syncthreads();
  }
}

template <typename T, int MAXPJ>
cudaError_t run_project(gbc_ctx* c, const cplx<T>* X, int nvec, int ldx, cplx<T>* Cbuf,
                        cudaStream_t s) {
  const ProjDev& pj = c->proj;
  const cplx<T>* P = std::is_same<T, double>::value ? (const cplx<T>*)pj.d_P64
                                                    : (const cplx<T>*)pj.d_P32;
  // deterministic mode: per-chunk sums, then each atom's chunks added in order
  cplx<T>* Cpart = nullptr;
  if (c->deterministic) {
    if (gbc_ensure_work(c, 11, sizeof(cplx<T>) * pj.nchunks * 2 * MAXPJ * (size_t)nvec) != GBC_OK)
      return cudaErrorMemoryAllocation;
    Cpart = (cplx<T>*)c->work[11];
  }
  dim3 grid(pj.nchunks, (2 * nvec + kCols - 1) / kCols);
  nl_project<T, MAXPJ><<<grid, kCols, 0, s>>>(X, ldx, nvec, pj.d_chunks, pj.d_nodes, P,
                                              pj.d_atom_npj, pj.d_atom_pv_off, pj.d_atom_c_off,
                                              Cbuf, c->mesh.M, Cpart);
  if (!Cpart) return cudaGetLastError();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 g2(pj.natoms, 2 * pj.max_npj, (nvec + kCols - 1) / kCols);
  k_nl_chunk_sum<T, MAXPJ><<<g2, kCols, 0, s>>>(Cpart, Cbuf, pj.d_chunk_off, pj.d_atom_npj,
                                                pj.d_atom_c_off, nvec);
  return cudaGetLastError();
}

bool use_tc(const gbc_ctx* c) { return c->nl_engine == GBC_NL_TENSOR && tc_nonlocal_supported(c->proj); }

}  // namespace

template <typename T>
cudaError_t launch_nonlocal(gbc_ctx* c, const cplx<T>* X, cplx<T>* Y, int nvec, int ldx,
                            cplx<T>* Cbuf, cplx<T>* Cpbuf, cudaStream_t s, bool overwrite,
                            void* bpre) {
  const ProjDev& pj = c->proj;
  if (pj.natoms == 0 || nvec == 0 || pj.nchunks == 0 || pj.nexp_chunks == 0) return cudaSuccess;
  cudaError_t e = launch_nl_project<T>(c, X, nvec, ldx, Cbuf, s);
  if (e != cudaSuccess) return e;
  const cplx<T>* D = std::is_same<T, double>::value ? (const cplx<T>*)pj.d_delta64
                                                    : (const cplx<T>*)pj.d_delta32;
  dim3 g2(pj.natoms, 2 * pj.max_npj, (nvec + kCols - 1) / kCols);
  nl_couple<T><<<g2, kCols, 0, s>>>(Cbuf, Cpbuf, D, pj.d_atom_npj, pj.d_atom_delta_off,
                                   pj.d_atom_c_off, nvec);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if constexpr (std::is_same<T, float>::value) {
    if (use_tc(c)) return launch_tc_expand(pj, Y, nvec, ldx, Cpbuf, s, overwrite, bpre, c->d_cell_ctr);
  }
  const cplx<T>* P = std::is_same<T, double>::value ? (const cplx<T>*)pj.d_P64
                                                    : (const cplx<T>*)pj.d_P32;
  dim3 g3((unsigned)pj.nexp_chunks, (2 * nvec + kCols - 1) / kCols);
#define GBC_EXPAND(MP)                                                                        \
  nl_expand<T, MP><<<g3, kCols, 0, s>>>(Y, ldx, nvec, pj.d_exp_chunks, pj.d_own_node,           \
                                        pj.d_own_pos, pj.d_own_xptr, pj.d_own_xinc, P,         \
                                        pj.d_atom_npj, pj.d_atom_pv_off, pj.d_atom_c_off, Cpbuf, \
                                        overwrite ? 1 : 0, c->mesh.M)
  if (pj.max_npj <= 4) GBC_EXPAND(4);
  else if (pj.max_npj <= 8) GBC_EXPAND(8);
  else if (pj.max_npj <= 18) GBC_EXPAND(18);
  else GBC_EXPAND(GBC_MAX_NPJ);
#undef GBC_EXPAND
  return cudaGetLastError();
}

// C = (P_a x I2)^H X for every atom (rows c_off + 2chi + s), C zeroed first
template <typename T>
cudaError_t launch_nl_project(gbc_ctx* c, const cplx<T>* X, int nvec, int ldx, cplx<T>* Cbuf,
                              cudaStream_t s) {
  const ProjDev& pj = c->proj;
  if (pj.natoms == 0 || nvec == 0 || pj.nchunks == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(Cbuf, 0, sizeof(cplx<T>) * (size_t)pj.rows_total * nvec, s);
  if (e != cudaSuccess) return e;
  if constexpr (std::is_same<T, float>::value) {
    if (use_tc(c)) return launch_tc_project(pj, c->mesh.M, X, nvec, ldx, Cbuf, s);
  }
  if (pj.max_npj <= 4) return run_project<T, 4>(c, X, nvec, ldx, Cbuf, s);
  if (pj.max_npj <= 8) return run_project<T, 8>(c, X, nvec, ldx, Cbuf, s);
  if (pj.max_npj <= 18) return run_project<T, 18>(c, X, nvec, ldx, Cbuf, s);
  return run_project<T, GBC_MAX_NPJ>(c, X, nvec, ldx, Cbuf, s);
}
template cudaError_t launch_nl_project<float>(gbc_ctx*, const float2*, int, int, float2*,
                                              cudaStream_t);
template cudaError_t launch_nl_project<double>(gbc_ctx*, const double2*, int, int, double2*,
                                               cudaStream_t);

template cudaError_t launch_nonlocal<float>(gbc_ctx*, const float2*, float2*, int, int, float2*,
                                            float2*, cudaStream_t, bool, void*);
template cudaError_t launch_nonlocal<double>(gbc_ctx*, const double2*, double2*, int, int,
                                             double2*, double2*, cudaStream_t, bool, void*);

size_t nl_work_bytes(const gbc_ctx* c, int nvec, int ldx, size_t el, size_t* bpre_off) {
  const size_t cb = el * (size_t)c->proj.rows_total * (size_t)nvec;
  const size_t off = (2 * cb + 255) & ~(size_t)255;
  const size_t xb = el == sizeof(float2) ? tc_expand_bpre_bytes(c->proj, nvec, ldx) : 0;
  if (bpre_off) *bpre_off = xb ? off : 0;
  return std::max<size_t>(64, xb ? off + xb : 2 * cb);
}

GBC_CHECK_WORD_ACCESSOR(gbc_check_word_nl)
