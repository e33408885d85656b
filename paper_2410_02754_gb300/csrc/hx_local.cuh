// Cell-level apply of the local spinor Hamiltonian, matrix-free (sum
// factorisation), with atomic assembly into the global block.
//
// Paper: Sec. IV.B.2 (extract X^(e) = R^(e) X, cell products, assemble
// Y = sum_e R^(e)T Y^(e)) with the cell operator of Eq. FEHlocEl plus the
// k-terms of Eq. FEHloc in per-cell Hermitian form.  The dense cell matrix
// (N o V^eff) N^T of Sec. IV.B.1 is applied in factored form: interpolate to
// the Gauss points with N (n_p -> n_q per direction), multiply by
// w_q J [ (V + |k|^2/2) I + B . sigma ], test back with N^T.  The kinetic and
// -i k.grad parts use the tensor structure of the shared reference matrices:
//   K^k = sum_d G_d (x) B (x) B  (G_d in direction d, B in the other two),
//   G_d = 1/2 A_d - (i/2) k_d (C^ - C^T),
// applied as 7 one-dimensional contractions.
//
// Thread mapping: a CTA owns one cell and VB vectors; 64 "lanes" per vector
// walk the pencils of each 1-D contraction.  Each vector has three padded
// n_q^3 shared-memory buffers; per-point data are the two spin components.
#pragma once

#include <algorithm>
#include <type_traits>

#include "gbc_internal.h"

namespace gbc {

// One system of a launch: its blocks, fields, mesh and the first global work item.
template <typename T> struct SysDesc {
  const cplx<T>* X;
  cplx<T>* Y;
  const T* fields;   // [E][4][NQ^3]
  int ldx, nvec, vchunks, pad;
  long long item0;   // work items of this system: [item0, item0 + E * vchunks)
  MeshDev mesh;
};

// A launch covers up to GBC_MAX_BATCH systems that share p, the cell edges and
// the k-point (hence the 1-D tables); items run over all systems.
template <typename T> struct LocalArgs {
  SysDesc<T> sys[GBC_MAX_BATCH];
  int nsys;
  long long nitems;
};

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }

template <typename T> __device__ __forceinline__ void atomic_add_c(cplx<T>* p, cplx<T> v);
template <> __device__ __forceinline__ void atomic_add_c<float>(float2* p, float2 v) {
  atomicAdd(p, v);
}
template <> __device__ __forceinline__ void atomic_add_c<double>(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// point (x, y, z) -> index in a padded per-vector buffer
template <int NQ> __device__ __forceinline__ int pidx(int x, int y, int z) {
  return x + y * (NQ + 1) + z * (NQ + 1) * (NQ + 1);
}

template <typename T, int NP, int NQ, bool KPT, int VB>
__global__ void __launch_bounds__(VB * 64, sizeof(T) == 4 ? 3 : 2)
hx_local_kernel(const __grid_constant__ LocalArgs<T> a, const Tables1D<T, NP, NQ> tb) {
  using C = cplx<T>;
  constexpr int TPV = 64;
  constexpr int BUF = (NQ + 1) * (NQ + 1) * NQ;      // points per padded buffer
  constexpr int NQ3 = NQ * NQ * NQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // per-vector stride 3*BUF*2 + 1 complex: the 8-byte shift puts the vectors of a
  // CTA (adjacent threads) in different shared-memory banks
  constexpr int VSTRIDE = 3 * BUF * 2 + 1;
  C* buf = reinterpret_cast<C*>(smem_raw);             // [VB][VSTRIDE]
  T* fld = reinterpret_cast<T*>(buf + VB * VSTRIDE);   // [4][NQ3]

  const int v = threadIdx.x % VB;
  const int lane = threadIdx.x / VB;
  const long long nitems = a.nitems;
  auto locate = [&](long long it) {
    int q = 0;
#pragma unroll
    for (int r = 1; r < GBC_MAX_BATCH; ++r)
      if (r < a.nsys && it >= a.sys[r].item0) q = r;
    return q;
  };

  C* A = buf + v * VSTRIDE;
  C* Bb = A + BUF * 2;
  C* Cb = A + 2 * BUF * 2;

  // Persistent CTA: items (system, cell, vector chunk), vector chunk fastest, taken
  // with a grid stride so the CTAs running together work on neighbouring cells.
  // The next item's X^(e) and fields are loaded into registers while the current
  // one is computed (the loads are issued right after the current item is staged).
  constexpr int PPL = (NP * NP * NP + TPV - 1) / TPV;       // nodes per lane
  constexpr int FPT = (4 * NQ3 + VB * TPV - 1) / (VB * TPV); // field values per thread
  C pfx[PPL][2];
  T pff[FPT];
  auto prefetch = [&](long long it) {
    if (it >= nitems) return;
    const SysDesc<T>& d = a.sys[locate(it)];
    const long long li = it - d.item0;
    const int e = (int)(li / d.vchunks);
    const int vec = (int)(li % d.vchunks) * VB + v;
    const bool vok = vec < d.nvec;
    const int nx = d.mesh.ncell[0], ny = d.mesh.ncell[1];
    const int cx = e % nx, cy = (e / nx) % ny, cz = e / (nx * ny);
#pragma unroll
    for (int j = 0; j < PPL; ++j) {
      const int i = lane + j * TPV;
      pfx[j][0] = cmake<C>(0, 0);
      pfx[j][1] = cmake<C>(0, 0);
      if (i < NP * NP * NP && vok) {
        const long long I = gbc_node(d.mesh, cx, cy, cz, i % NP, (i / NP) % NP, i / (NP * NP));
        if (I >= 0) {
          pfx[j][0] = d.X[(I * 2 + 0) * d.ldx + vec];
          pfx[j][1] = d.X[(I * 2 + 1) * d.ldx + vec];
        }
      }
    }
    const T* fsrc = d.fields + (size_t)e * 4 * NQ3;
#pragma unroll
    for (int j = 0; j < FPT; ++j) {
      const int f = threadIdx.x + j * VB * TPV;
      pff[j] = f < 4 * NQ3 ? fsrc[f] : (T)0;
    }
  };
  prefetch(blockIdx.x);

  for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
  const SysDesc<T>& d = a.sys[locate(item)];
  const long long li = item - d.item0;
  const int e = (int)(li / d.vchunks);
  const int vec = (int)(li % d.vchunks) * VB + v;
  const bool vok = vec < d.nvec;
  const int nx = d.mesh.ncell[0], ny = d.mesh.ncell[1];
  const int cx = e % nx, cy = (e / nx) % ny, cz = e / (nx * ny);

  // ---- stage X^(e) (both spins) and the cell's fields from the prefetch registers
#pragma unroll
  for (int j = 0; j < PPL; ++j) {
    const int i = lane + j * TPV;
    if (i < NP * NP * NP) {
      const int q = pidx<NQ>(i % NP, (i / NP) % NP, i / (NP * NP));
      A[2 * q] = pfx[j][0];
      A[2 * q + 1] = pfx[j][1];
    }
  }
#pragma unroll
  for (int j = 0; j < FPT; ++j) {
    const int f = threadIdx.x + j * VB * TPV;
    if (f < 4 * NQ3) fld[f] = pff[j];
  }
  __syncthreads();
  prefetch(item + gridDim.x);

  // ===== kinetic / k part:  Y = G_x(B_y B_z X) + B_x(G_y B_z X + B_y G_z X)
  // z-stage: T1 = B_z X -> Bb, T2 = G_z X -> Cb
  for (int pid = lane; pid < NP * NP; pid += TPV) {
    const int x = pid % NP, y = pid / NP;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C in[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = A[2 * pidx<NQ>(x, y, j) + s];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T t1r = 0, t1i = 0, t2r = 0, t2i = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          t1r += tb.B[2][i][j] * in[j].x;
          t1i += tb.B[2][i][j] * in[j].y;
          t2r += tb.Gr[2][i][j] * in[j].x;
          t2i += tb.Gr[2][i][j] * in[j].y;
          if (KPT) {
            t2r -= tb.Gi[2][i][j] * in[j].y;
            t2i += tb.Gi[2][i][j] * in[j].x;
          }
        }
        Bb[2 * pidx<NQ>(x, y, i) + s] = cmake<C>(t1r, t1i);
        Cb[2 * pidx<NQ>(x, y, i) + s] = cmake<C>(t2r, t2i);
      }
    }
  }
  __syncthreads();
  // y-stage (in place): U1 = B_y T1 -> Bb, U2 = G_y T1 + B_y T2 -> Cb
  for (int pid = lane; pid < NP * NP; pid += TPV) {
    const int x = pid % NP, z = pid / NP;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C t1[NP], t2[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        t1[j] = Bb[2 * pidx<NQ>(x, j, z) + s];
        t2[j] = Cb[2 * pidx<NQ>(x, j, z) + s];
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T u1r = 0, u1i = 0, u2r = 0, u2i = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          u1r += tb.B[1][i][j] * t1[j].x;
          u1i += tb.B[1][i][j] * t1[j].y;
          u2r += tb.Gr[1][i][j] * t1[j].x + tb.B[1][i][j] * t2[j].x;
          u2i += tb.Gr[1][i][j] * t1[j].y + tb.B[1][i][j] * t2[j].y;
          if (KPT) {
            u2r -= tb.Gi[1][i][j] * t1[j].y;
            u2i += tb.Gi[1][i][j] * t1[j].x;
          }
        }
        Bb[2 * pidx<NQ>(x, i, z) + s] = cmake<C>(u1r, u1i);
        Cb[2 * pidx<NQ>(x, i, z) + s] = cmake<C>(u2r, u2i);
      }
    }
  }
  __syncthreads();
  // x-stage: Y = G_x U1 + B_x U2, kept in registers (one x-pencil per lane)
  constexpr int NPEN = (NP * NP + TPV - 1) / TPV;    // x-pencils per lane (1 for p <= 7)
  C yacc[NPEN][2][NP];
#pragma unroll
  for (int k = 0; k < NPEN; ++k) {
    const int pid = lane + k * TPV;
    if (pid >= NP * NP) break;
    const int y = pid % NP, z = pid / NP;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C u1[NP], u2[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        u1[j] = Bb[2 * pidx<NQ>(j, y, z) + s];
        u2[j] = Cb[2 * pidx<NQ>(j, y, z) + s];
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T yr = 0, yi = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          yr += tb.Gr[0][i][j] * u1[j].x + tb.B[0][i][j] * u2[j].x;
          yi += tb.Gr[0][i][j] * u1[j].y + tb.B[0][i][j] * u2[j].y;
          if (KPT) {
            yr -= tb.Gi[0][i][j] * u1[j].y;
            yi += tb.Gi[0][i][j] * u1[j].x;
          }
        }
        yacc[k][s][i] = cmake<C>(yr, yi);
      }
    }
  }
  __syncthreads();

  // ===== V_eff / B_xc part through the Gauss points
  // interp x: A (np,np,np) -> Bb (nq,np,np)
  for (int pid = lane; pid < NP * NP; pid += TPV) {
    const int y = pid % NP, z = pid / NP;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C in[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = A[2 * pidx<NQ>(j, y, z) + s];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T r = 0, im = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          r += tb.N[j][q] * in[j].x;
          im += tb.N[j][q] * in[j].y;
        }
        Bb[2 * pidx<NQ>(q, y, z) + s] = cmake<C>(r, im);
      }
    }
  }
  __syncthreads();
  // interp y: Bb (nq,np,np) -> Cb (nq,nq,np)
  for (int pid = lane; pid < NQ * NP; pid += TPV) {
    const int x = pid % NQ, z = pid / NQ;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C in[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = Bb[2 * pidx<NQ>(x, j, z) + s];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T r = 0, im = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          r += tb.N[j][q] * in[j].x;
          im += tb.N[j][q] * in[j].y;
        }
        Cb[2 * pidx<NQ>(x, q, z) + s] = cmake<C>(r, im);
      }
    }
  }
  __syncthreads();
  // interp z + pointwise spin operator: Cb (nq,nq,np) -> Bb (nq,nq,nq)
  for (int pid = lane; pid < NQ * NQ; pid += TPV) {
    const int x = pid % NQ, y = pid / NQ;
    C iu[NP], id[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      iu[j] = Cb[2 * pidx<NQ>(x, y, j)];
      id[j] = Cb[2 * pidx<NQ>(x, y, j) + 1];
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T ur = 0, ui = 0, dr = 0, di = 0;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        ur += tb.N[j][q] * iu[j].x;
        ui += tb.N[j][q] * iu[j].y;
        dr += tb.N[j][q] * id[j].x;
        di += tb.N[j][q] * id[j].y;
      }
      const int qq = (q * NQ + y) * NQ + x;
      const T V = fld[qq], bx = fld[NQ3 + qq], by = fld[2 * NQ3 + qq], bz = fld[3 * NQ3 + qq];
      // [(V + bz) u + (bx - i by) d ; (bx + i by) u + (V - bz) d]
      const T our = (V + bz) * ur + bx * dr + by * di;
      const T oui = (V + bz) * ui + bx * di - by * dr;
      const T odr = bx * ur - by * ui + (V - bz) * dr;
      const T odi = bx * ui + by * ur + (V - bz) * di;
      Bb[2 * pidx<NQ>(x, y, q)] = cmake<C>(our, oui);
      Bb[2 * pidx<NQ>(x, y, q) + 1] = cmake<C>(odr, odi);
    }
  }
  __syncthreads();
  // test z: Bb (nq,nq,nq) -> Cb (nq,nq,np)
  for (int pid = lane; pid < NQ * NQ; pid += TPV) {
    const int x = pid % NQ, y = pid / NQ;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C in[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) in[q] = Bb[2 * pidx<NQ>(x, y, q) + s];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T r = 0, im = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          r += tb.N[i][q] * in[q].x;
          im += tb.N[i][q] * in[q].y;
        }
        Cb[2 * pidx<NQ>(x, y, i) + s] = cmake<C>(r, im);
      }
    }
  }
  __syncthreads();
  // test y: Cb (nq,nq,np) -> Bb (nq,np,np)
  for (int pid = lane; pid < NQ * NP; pid += TPV) {
    const int x = pid % NQ, z = pid / NQ;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C in[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) in[q] = Cb[2 * pidx<NQ>(x, q, z) + s];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T r = 0, im = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          r += tb.N[i][q] * in[q].x;
          im += tb.N[i][q] * in[q].y;
        }
        Bb[2 * pidx<NQ>(x, i, z) + s] = cmake<C>(r, im);
      }
    }
  }
  __syncthreads();
  // test x: Bb (nq,np,np) -> add into the x-pencil registers, then assemble
#pragma unroll
  for (int k = 0; k < NPEN; ++k) {
    const int pid = lane + k * TPV;
    if (pid >= NP * NP) break;
    const int y = pid % NP, z = pid / NP;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C in[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) in[q] = Bb[2 * pidx<NQ>(q, y, z) + s];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T r = 0, im = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          r += tb.N[i][q] * in[q].x;
          im += tb.N[i][q] * in[q].y;
        }
        yacc[k][s][i].x += r;
        yacc[k][s][i].y += im;
      }
    }
    if (vok) {
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const long long I = gbc_node(d.mesh, cx, cy, cz, i, y, z);
        if (I < 0) continue;
        atomic_add_c<T>(&d.Y[(I * 2 + 0) * d.ldx + vec], yacc[k][0][i]);
        atomic_add_c<T>(&d.Y[(I * 2 + 1) * d.ldx + vec], yacc[k][1][i]);
      }
    }
  }
  }  // item loop
}

template <typename T, int NP, int NQ, int VB> constexpr size_t hx_local_smem() {
  return sizeof(cplx<T>) * (size_t)VB * (3 * ((NQ + 1) * (NQ + 1) * NQ) * 2 + 1) +
         sizeof(T) * 4 * NQ * NQ * NQ;
}

// build the per-launch 1-D tables from the context's FP64 host tables
template <typename T, int NP, int NQ>
inline Tables1D<T, NP, NQ> make_tables(const gbc_ctx* c) {
  Tables1D<T, NP, NQ> t;
  const HostTables& h = c->tab;
  for (int d = 0; d < 3; ++d) {
    const double hd = c->h[d];
    for (int i = 0; i < NP; ++i)
      for (int j = 0; j < NP; ++j) {
        t.B[d][i][j] = (T)(0.5 * hd * h.Bh[i * NP + j]);
        t.Gr[d][i][j] = (T)(0.5 * (2.0 / hd) * h.Ah[i * NP + j]);
        t.Gi[d][i][j] = (T)(-0.5 * c->k[d] * (h.Ch[i * NP + j] - h.Ch[j * NP + i]));
      }
  }
  for (int i = 0; i < NP; ++i)
    for (int q = 0; q < NQ; ++q) t.N[i][q] = (T)h.N1[i * NQ + q];
  return t;
}

// One launch over n systems that share p, the cell edges and the k-point; the
// first system's context provides the 1-D tables.
template <typename T, int NP, int VB>
cudaError_t launch_hx_group_p(const HxJob* jobs, int n, cudaStream_t s) {
  constexpr int NQ = NP + 1;   // nq = p + 2
  if (n < 1 || n > GBC_MAX_BATCH) return cudaErrorInvalidValue;
  LocalArgs<T> a;
  long long item = 0;
  for (int i = 0; i < GBC_MAX_BATCH; ++i) {
    SysDesc<T>& d = a.sys[i];
    if (i >= n) {
      d = a.sys[0];
      d.item0 = 0x7fffffffffffffffLL;
      continue;
    }
    const gbc_ctx* c = jobs[i].c;
    d.X = (const cplx<T>*)jobs[i].X;
    d.Y = (cplx<T>*)jobs[i].Y;
    d.fields = std::is_same<T, double>::value ? (const T*)c->d_fields64 : (const T*)c->d_fields32;
    d.ldx = jobs[i].ldx;
    d.nvec = jobs[i].nvec;
    d.vchunks = (jobs[i].nvec + VB - 1) / VB;
    d.pad = 0;
    d.item0 = item;
    d.mesh = c->mesh;
    item += (long long)c->mesh.E * d.vchunks;
  }
  a.nsys = n;
  a.nitems = item;
  if (item <= 0) return cudaSuccess;
  const gbc_ctx* c0 = jobs[0].c;
  const auto tb = make_tables<T, NP, NQ>(c0);
  const bool kpt = (c0->k[0] != 0.0 || c0->k[1] != 0.0 || c0->k[2] != 0.0);
  constexpr size_t smem = hx_local_smem<T, NP, NQ, VB>();
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  auto run = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, VB * 64, smem);
    if (e != cudaSuccess) return e;
    const long long nblk = std::min<long long>(item, (long long)nsm * std::max(per_sm, 1));
    kern<<<(unsigned)nblk, VB * 64, smem, s>>>(a, tb);
    return cudaGetLastError();
  };
  if (kpt) return run(hx_local_kernel<T, NP, NQ, true, VB>);
  return run(hx_local_kernel<T, NP, NQ, false, VB>);
}

// dispatch on p (nq = p + 2) for a fixed VB
template <typename T, int VB>
cudaError_t launch_hx_group(const HxJob* jobs, int n, cudaStream_t s) {
  switch (jobs[0].c->mesh.p) {
    case 2: return launch_hx_group_p<T, 3, VB>(jobs, n, s);
    case 3: return launch_hx_group_p<T, 4, VB>(jobs, n, s);
    case 4: return launch_hx_group_p<T, 5, VB>(jobs, n, s);
    case 5: return launch_hx_group_p<T, 6, VB>(jobs, n, s);
    case 6: return launch_hx_group_p<T, 7, VB>(jobs, n, s);
    case 7: return launch_hx_group_p<T, 8, VB>(jobs, n, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gbc
