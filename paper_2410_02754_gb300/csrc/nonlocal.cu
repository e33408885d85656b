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

constexpr int kChunk = 512;     // support nodes per projection block
constexpr int kStage = 32;      // nodes staged in shared memory at a time
constexpr int kCols = 128;      // threads (columns) per block

// C[(c_off + 2chi + s) * nvec + v] += sum_j conj(P[j][chi]) X[node_j][s][v]
template <typename T, int MAXPJ>
__global__ void __launch_bounds__(kCols)
nl_project(const cplx<T>* __restrict__ X, int ldx, int nvec, const int4* __restrict__ chunks,
           const long long* __restrict__ nodes, const cplx<T>* __restrict__ P,
           const int* __restrict__ atom_npj, const int* __restrict__ atom_pv_off,
           const int* __restrict__ atom_c_off, cplx<T>* __restrict__ Cbuf) {
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
      for (int t = 0; t < nb; ++t) {
        const C x = X[(Ns[t] * 2 + s) * ldx + v];
#pragma unroll
        for (int c = 0; c < MAXPJ; ++c)
          if (c < npj) cmac_conj(acc[c], Ps[t][c], x);
      }
    }
    __syncthreads();
  }
  if (ok) {
    const int r0 = atom_c_off[atom];
#pragma unroll
    for (int c = 0; c < MAXPJ; ++c)
      if (c < npj) catomic(&Cbuf[(size_t)(r0 + 2 * c + s) * nvec + v], acc[c]);
  }
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

// Y[node][s][v] += sum over atoms whose support holds node of sum_chi P[pos][chi] Cp[2chi+s][v]
// A block owns kExpNodes consecutive unique support nodes and 128 columns.
constexpr int kExpNodes = 16;
template <typename T>
__global__ void __launch_bounds__(kCols)
nl_expand(cplx<T>* __restrict__ Y, int ldx, int nvec, const long long* __restrict__ uniq_node,
          const int* __restrict__ uniq_ptr, const int2* __restrict__ uniq_inc, long long nuniq,
          const cplx<T>* __restrict__ P, const int* __restrict__ atom_npj,
          const int* __restrict__ atom_pv_off, const int* __restrict__ atom_c_off,
          const cplx<T>* __restrict__ Cp) {
  using C = cplx<T>;
  const long long u0 = (long long)blockIdx.x * kExpNodes;
  const long long u1 = min(nuniq, u0 + kExpNodes);
  const int col = blockIdx.y * kCols + threadIdx.x;
  if (col >= 2 * nvec) return;
  const int s = col / nvec, v = col % nvec;
  for (long long u = u0; u < u1; ++u) {
    C acc = cmake<C>(0, 0);
    for (int k = uniq_ptr[u]; k < uniq_ptr[u + 1]; ++k) {
      const int2 inc = uniq_inc[k];
      const int npj = atom_npj[inc.x];
      const C* Pr = P + atom_pv_off[inc.x] + (size_t)inc.y * npj;
      const C* Cr = Cp + (size_t)atom_c_off[inc.x] * nvec + v + (size_t)s * nvec;
      for (int c = 0; c < npj; ++c) cmac(acc, Pr[c], Cr[(size_t)(2 * c) * nvec]);
    }
    C* y = &Y[(uniq_node[u] * 2 + s) * ldx + v];
    C o = *y;
    o.x += acc.x;
    o.y += acc.y;
    *y = o;
  }
}

template <typename T, int MAXPJ>
cudaError_t run_project(gbc_ctx* c, const cplx<T>* X, int nvec, int ldx, cplx<T>* Cbuf,
                        cudaStream_t s) {
  const ProjDev& pj = c->proj;
  const cplx<T>* P = std::is_same<T, double>::value ? (const cplx<T>*)pj.d_P64
                                                    : (const cplx<T>*)pj.d_P32;
  dim3 grid(pj.nchunks, (2 * nvec + kCols - 1) / kCols);
  nl_project<T, MAXPJ><<<grid, kCols, 0, s>>>(X, ldx, nvec, pj.d_chunks, pj.d_nodes, P,
                                              pj.d_atom_npj, pj.d_atom_pv_off, pj.d_atom_c_off,
                                              Cbuf);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_nonlocal(gbc_ctx* c, const cplx<T>* X, cplx<T>* Y, int nvec, int ldx,
                            cplx<T>* Cbuf, cplx<T>* Cpbuf, cudaStream_t s) {
  const ProjDev& pj = c->proj;
  if (pj.natoms == 0 || nvec == 0 || pj.nchunks == 0 || pj.nuniq == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(Cbuf, 0, sizeof(cplx<T>) * (size_t)pj.rows_total * nvec, s);
  if (e != cudaSuccess) return e;
  if (pj.max_npj <= 4) e = run_project<T, 4>(c, X, nvec, ldx, Cbuf, s);
  else if (pj.max_npj <= 8) e = run_project<T, 8>(c, X, nvec, ldx, Cbuf, s);
  else if (pj.max_npj <= 18) e = run_project<T, 18>(c, X, nvec, ldx, Cbuf, s);
  else e = run_project<T, GBC_MAX_NPJ>(c, X, nvec, ldx, Cbuf, s);
  if (e != cudaSuccess) return e;
  const cplx<T>* D = std::is_same<T, double>::value ? (const cplx<T>*)pj.d_delta64
                                                    : (const cplx<T>*)pj.d_delta32;
  dim3 g2(pj.natoms, 2 * pj.max_npj, (nvec + kCols - 1) / kCols);
  nl_couple<T><<<g2, kCols, 0, s>>>(Cbuf, Cpbuf, D, pj.d_atom_npj, pj.d_atom_delta_off,
                                   pj.d_atom_c_off, nvec);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const cplx<T>* P = std::is_same<T, double>::value ? (const cplx<T>*)pj.d_P64
                                                    : (const cplx<T>*)pj.d_P32;
  dim3 g3((unsigned)((pj.nuniq + kExpNodes - 1) / kExpNodes), (2 * nvec + kCols - 1) / kCols);
  nl_expand<T><<<g3, kCols, 0, s>>>(Y, ldx, nvec, pj.d_uniq_node, pj.d_uniq_ptr, pj.d_uniq_inc,
                                   pj.nuniq, P, pj.d_atom_npj, pj.d_atom_pv_off, pj.d_atom_c_off,
                                   Cpbuf);
  return cudaGetLastError();
}

template cudaError_t launch_nonlocal<float>(gbc_ctx*, const float2*, float2*, int, int, float2*,
                                            float2*, cudaStream_t);
template cudaError_t launch_nonlocal<double>(gbc_ctx*, const double2*, double2*, int, int,
                                             double2*, double2*, cudaStream_t);
