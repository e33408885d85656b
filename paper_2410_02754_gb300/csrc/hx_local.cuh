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
#include <cmath>
#include <type_traits>
#include <vector>

#include "gbc_internal.h"

namespace gbc {

// One system of a launch: its blocks, fields, mesh and the first global work item.
template <typename T> struct SysDesc {
  const cplx<T>* X;
  cplx<T>* Y;
  cplx<T>* Ycell;    // non-null: per-cell results [E][n_p^3][2][nvec] instead of assembly
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
// padded strides: y by NQ + 1, z by (NQ + 1) NQ + 1 points
template <int NQ> __device__ __forceinline__ int pidx(int x, int y, int z) {
  return x + y * (NQ + 1) + z * ((NQ + 1) * NQ + 1);
}
template <int NQ> __host__ __device__ constexpr int pbuf_points() {   // max pidx + 1
  return (NQ - 1) * (1 + (NQ + 1) + ((NQ + 1) * NQ + 1)) + 1;
}

// ---------------------------------------------------------------------------
// even-odd form of the 1-D operators
//
// GLL nodes and Gauss points are symmetric about the cell centre, so every 1-D
// matrix used here is centro-symmetric (M[no-1-i][ni-1-j] = M[i][j]: mass,
// stiffness, interpolation) or centro-antisymmetric (= -M[i][j]: C^ - C^T).
// With e_j = x_j + x_{ni-1-j}, o_j = x_j - x_{ni-1-j} (j < ni/2) and the
// middle entry x_mid when ni is odd,
//   y_i          =      (E e)_i + (O o)_i + Mid_i x_mid
//   y_{no-1-i}   = S * ((E e)_i - (O o)_i + Mid_i x_mid),   i < (no+1)/2,
// E = (M_ij + M_i,ni-1-j)/2, O = (M_ij - M_i,ni-1-j)/2: about half the
// multiply-adds of the dense product.
// ---------------------------------------------------------------------------
template <typename T, int NO, int NI> struct EO {
  static constexpr int HO = (NO + 1) / 2;
  static constexpr int HI = NI / 2 > 0 ? NI / 2 : 1;
  T E[HO][HI];
  T O[HO][HI];
  T Mid[HO];
};

template <typename T, int NP, int NQ> struct TablesEO {
  EO<T, NP, NP> B[3];    // 1-D Gauss mass h_d/2 B^               (symmetric)
  EO<T, NP, NP> Gr[3];   // 1/2 A_d                                (symmetric)
  EO<T, NP, NP> Gi[3];   // -1/2 k_d (C^ - C^T)                    (antisymmetric)
  EO<T, NQ, NP> Ni;      // interpolation: y_q = sum_i l_i(xi_q) x_i (symmetric)
  EO<T, NP, NQ> Nt;      // testing:       y_i = sum_q l_i(xi_q) x_q (symmetric)
};

template <int S, typename T, int NO, int NI, typename C>
__device__ __forceinline__ void eo_apply(const EO<T, NO, NI>& M, const C (&x)[NI], C (&y)[NO]) {
  constexpr int HI = NI / 2, HO = (NO + 1) / 2;
  C e[HI > 0 ? HI : 1], o[HI > 0 ? HI : 1];
#pragma unroll
  for (int j = 0; j < HI; ++j) {
    e[j].x = x[j].x + x[NI - 1 - j].x;
    e[j].y = x[j].y + x[NI - 1 - j].y;
    o[j].x = x[j].x - x[NI - 1 - j].x;
    o[j].y = x[j].y - x[NI - 1 - j].y;
  }
#pragma unroll
  for (int i = 0; i < HO; ++i) {
    T er = 0, ei = 0, orr = 0, oi = 0;
#pragma unroll
    for (int j = 0; j < HI; ++j) {
      er += M.E[i][j] * e[j].x;
      ei += M.E[i][j] * e[j].y;
      orr += M.O[i][j] * o[j].x;
      oi += M.O[i][j] * o[j].y;
    }
    if (NI & 1) {
      er += M.Mid[i] * x[HI].x;
      ei += M.Mid[i] * x[HI].y;
    }
    y[i].x = er + orr;
    y[i].y = ei + oi;
    if (NO - 1 - i != i) {
      y[NO - 1 - i].x = S * (er - orr);
      y[NO - 1 - i].y = S * (ei - oi);
    }
  }
}

// complex operator Gr + i Gi (Gr symmetric, Gi antisymmetric) on complex data
template <bool KPT, typename T, int N, typename C>
__device__ __forceinline__ void g_apply(const EO<T, N, N>& Gr, const EO<T, N, N>& Gi,
                                        const C (&x)[N], C (&y)[N]) {
  eo_apply<1>(Gr, x, y);
  if (KPT) {
    C t[N];
    eo_apply<-1>(Gi, x, t);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      y[i].x -= t[i].y;
      y[i].y += t[i].x;
    }
  }
}

// host: even-odd split of a dense row-major NO x NI matrix (checks the symmetry)
template <typename T, int NO, int NI>
inline bool make_eo(const std::vector<double>& M, int S, EO<T, NO, NI>* out) {
  double mx = 0;
  for (double v : M) mx = std::max(mx, std::fabs(v));
  for (int i = 0; i < NO; ++i)
    for (int j = 0; j < NI; ++j)
      if (std::fabs(M[i * NI + j] - S * M[(NO - 1 - i) * NI + (NI - 1 - j)]) > 1e-10 * (mx + 1e-300))
        return false;
  for (int i = 0; i < EO<T, NO, NI>::HO; ++i) {
    for (int j = 0; j < EO<T, NO, NI>::HI; ++j) {
      out->E[i][j] = (T)0;
      out->O[i][j] = (T)0;
      if (j < NI / 2) {
        out->E[i][j] = (T)(0.5 * (M[i * NI + j] + M[i * NI + NI - 1 - j]));
        out->O[i][j] = (T)(0.5 * (M[i * NI + j] - M[i * NI + NI - 1 - j]));
      }
    }
    out->Mid[i] = (NI & 1) ? (T)M[i * NI + NI / 2] : (T)0;
  }
  return true;
}

template <typename T, int NP, int NQ>
inline bool make_tables_eo(const gbc_ctx* c, TablesEO<T, NP, NQ>* t) {
  const HostTables& h = c->tab;
  bool ok = true;
  for (int d = 0; d < 3; ++d) {
    const double hd = c->h[d];
    std::vector<double> B(NP * NP), Gr(NP * NP), Gi(NP * NP);
    for (int i = 0; i < NP; ++i)
      for (int j = 0; j < NP; ++j) {
        B[i * NP + j] = 0.5 * hd * h.Bh[i * NP + j];
        Gr[i * NP + j] = 0.5 * (2.0 / hd) * h.Ah[i * NP + j];
        Gi[i * NP + j] = -0.5 * c->k[d] * (h.Ch[i * NP + j] - h.Ch[j * NP + i]);
      }
    ok = ok && make_eo<T, NP, NP>(B, 1, &t->B[d]) && make_eo<T, NP, NP>(Gr, 1, &t->Gr[d]) &&
         make_eo<T, NP, NP>(Gi, -1, &t->Gi[d]);
  }
  std::vector<double> Ni(NQ * NP), Nt(NP * NQ);
  for (int i = 0; i < NP; ++i)
    for (int q = 0; q < NQ; ++q) {
      Ni[q * NP + i] = h.N1[i * NQ + q];
      Nt[i * NQ + q] = h.N1[i * NQ + q];
    }
  ok = ok && make_eo<T, NQ, NP>(Ni, 1, &t->Ni) && make_eo<T, NP, NQ>(Nt, 1, &t->Nt);
  return ok;
}

template <typename T, int NP, int NQ, bool KPT, int VB>
__global__ void __launch_bounds__(VB * 64, sizeof(T) == 4 ? 4 : 2)
hx_local_kernel(const __grid_constant__ LocalArgs<T> a, const TablesEO<T, NP, NQ> tb) {
  using C = cplx<T>;
  constexpr int TPV = 64;
  constexpr int NT = VB * TPV;
  constexpr int BUF = pbuf_points<NQ>();             // points per padded buffer
  constexpr int NQ3 = NQ * NQ * NQ;
  // per-vector stride = 8 (mod 16) complex: threads of neighbouring work units
  // (vector fastest, then spin, then pencil) fall into distinct banks
  constexpr int VBASE = 3 * BUF * 2;
  constexpr int VSTRIDE = VBASE + ((24 - VBASE % 16) % 16);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  auto Ab = [&](int v) { return buf + v * VSTRIDE; };
  auto Bb = [&](int v) { return buf + v * VSTRIDE + BUF * 2; };
  auto Cb = [&](int v) { return buf + v * VSTRIDE + 2 * BUF * 2; };

  const int v0 = threadIdx.x % VB;      // vector of this thread for gathering
  const int lane = threadIdx.x / VB;
  const long long nitems = a.nitems;
  auto locate = [&](long long it) {
    int q = 0;
#pragma unroll
    for (int r = 1; r < GBC_MAX_BATCH; ++r)
      if (r < a.nsys && it >= a.sys[r].item0) q = r;
    return q;
  };

  // work units of the single-spin stages: u -> (vector, spin, pencil), vector fastest
  constexpr int XU = VB * NP * NP * 2;          // units of the x-pencil stages
  constexpr int XR = (XU + NT - 1) / NT;        // rounds per thread

  for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
    const SysDesc<T>& d = a.sys[locate(item)];
    const long long li = item - d.item0;
    const int e = (int)(li / d.vchunks);
    const int vbase = (int)(li % d.vchunks) * VB;
    const int nx = d.mesh.ncell[0], ny = d.mesh.ncell[1];
    const int cx = e % nx, cy = (e / nx) % ny, cz = e / (nx * ny);

    // ---- extract X^(e) (both spins) into A
    {
      const int vec = vbase + v0;
      const bool vok = vec < d.nvec;
      for (int i = lane; i < NP * NP * NP; i += TPV) {
        const int ix = i % NP, iy = (i / NP) % NP, iz = i / (NP * NP);
        const long long I = gbc_node(d.mesh, cx, cy, cz, ix, iy, iz);
        C u = cmake<C>(0, 0), dn = cmake<C>(0, 0);
        if (I >= 0 && vok && GBC_IN_RANGE(GBC_SITE_HX64, I, d.mesh.M)) {
          u = d.X[(I * 2 + 0) * d.ldx + vec];
          dn = d.X[(I * 2 + 1) * d.ldx + vec];
        }
        const int q = pidx<NQ>(ix, iy, iz);
        Ab(v0)[2 * q] = u;
        Ab(v0)[2 * q + 1] = dn;
      }
    }
    const T* __restrict__ fld = d.fields + (size_t)e * 4 * NQ3;   // read through L1
    __syncthreads();

    // ===== kinetic / k part: Y = G_x(B_y B_z X) + B_x(G_y B_z X + B_y G_z X)
    // z-stage: T1 = B_z X -> Bb, T2 = G_z X -> Cb
    for (int u = threadIdx.x; u < VB * NP * NP * 2; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int x = pen % NP, y = pen / NP;
      C in[NP], t1[NP], t2[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = Ab(v)[2 * pidx<NQ>(x, y, j) + s];
      eo_apply<1>(tb.B[2], in, t1);
      g_apply<KPT>(tb.Gr[2], tb.Gi[2], in, t2);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        Bb(v)[2 * pidx<NQ>(x, y, i) + s] = t1[i];
        Cb(v)[2 * pidx<NQ>(x, y, i) + s] = t2[i];
      }
    }
    __syncthreads();
    // y-stage (in place): U1 = B_y T1 -> Bb, U2 = G_y T1 + B_y T2 -> Cb
    for (int u = threadIdx.x; u < VB * NP * NP * 2; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int x = pen % NP, z = pen / NP;
      C t1[NP], t2[NP], u1[NP], u2[NP], w2[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        t1[j] = Bb(v)[2 * pidx<NQ>(x, j, z) + s];
        t2[j] = Cb(v)[2 * pidx<NQ>(x, j, z) + s];
      }
      eo_apply<1>(tb.B[1], t1, u1);
      g_apply<KPT>(tb.Gr[1], tb.Gi[1], t1, u2);
      eo_apply<1>(tb.B[1], t2, w2);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        Bb(v)[2 * pidx<NQ>(x, i, z) + s] = u1[i];
        Cb(v)[2 * pidx<NQ>(x, i, z) + s] = cadd(u2[i], w2[i]);
      }
    }
    __syncthreads();
    // x-stage: Y = G_x U1 + B_x U2, kept in registers per work unit
    C yacc[XR][NP];
#pragma unroll
    for (int r = 0; r < XR; ++r) {
      const int u = threadIdx.x + r * NT;
      if (u >= XU) break;
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int y = pen % NP, z = pen / NP;
      C u1[NP], u2[NP], w2[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        u1[j] = Bb(v)[2 * pidx<NQ>(j, y, z) + s];
        u2[j] = Cb(v)[2 * pidx<NQ>(j, y, z) + s];
      }
      g_apply<KPT>(tb.Gr[0], tb.Gi[0], u1, yacc[r]);
      eo_apply<1>(tb.B[0], u2, w2);
#pragma unroll
      for (int i = 0; i < NP; ++i) yacc[r][i] = cadd(yacc[r][i], w2[i]);
    }
    __syncthreads();

    // ===== V_eff / B_xc part through the Gauss points
    // interp x: A (np,np,np) -> Bb (nq,np,np)
    for (int u = threadIdx.x; u < VB * NP * NP * 2; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int y = pen % NP, z = pen / NP;
      C in[NP], out[NQ];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = Ab(v)[2 * pidx<NQ>(j, y, z) + s];
      eo_apply<1>(tb.Ni, in, out);
#pragma unroll
      for (int q = 0; q < NQ; ++q) Bb(v)[2 * pidx<NQ>(q, y, z) + s] = out[q];
    }
    __syncthreads();
    // interp y: Bb (nq,np,np) -> Cb (nq,nq,np)
    for (int u = threadIdx.x; u < VB * NQ * NP * 2; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int x = pen % NQ, z = pen / NQ;
      C in[NP], out[NQ];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = Bb(v)[2 * pidx<NQ>(x, j, z) + s];
      eo_apply<1>(tb.Ni, in, out);
#pragma unroll
      for (int q = 0; q < NQ; ++q) Cb(v)[2 * pidx<NQ>(x, q, z) + s] = out[q];
    }
    __syncthreads();
    // interp z + pointwise spin operator: Cb (nq,nq,np) -> Bb (nq,nq,nq), both spins
    for (int u = threadIdx.x; u < VB * NQ * NQ; u += NT) {
      const int v = u % VB, pen = u / VB;
      const int x = pen % NQ, y = pen / NQ;
      C iu[NP], id[NP], ou[NQ], od[NQ];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        iu[j] = Cb(v)[2 * pidx<NQ>(x, y, j)];
        id[j] = Cb(v)[2 * pidx<NQ>(x, y, j) + 1];
      }
      eo_apply<1>(tb.Ni, iu, ou);
      eo_apply<1>(tb.Ni, id, od);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int qq = (q * NQ + y) * NQ + x;
        const T V = __ldg(fld + qq), bx = __ldg(fld + NQ3 + qq), by = __ldg(fld + 2 * NQ3 + qq),
                bz = __ldg(fld + 3 * NQ3 + qq);
        const T ur = ou[q].x, ui = ou[q].y, dr = od[q].x, di = od[q].y;
        // [(V + bz) u + (bx - i by) d ; (bx + i by) u + (V - bz) d]
        Bb(v)[2 * pidx<NQ>(x, y, q)] =
            cmake<C>((V + bz) * ur + bx * dr + by * di, (V + bz) * ui + bx * di - by * dr);
        Bb(v)[2 * pidx<NQ>(x, y, q) + 1] =
            cmake<C>(bx * ur - by * ui + (V - bz) * dr, bx * ui + by * ur + (V - bz) * di);
      }
    }
    __syncthreads();
    // test z: Bb (nq,nq,nq) -> Cb (nq,nq,np)
    for (int u = threadIdx.x; u < VB * NQ * NQ * 2; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int x = pen % NQ, y = pen / NQ;
      C in[NQ], out[NP];
#pragma unroll
      for (int q = 0; q < NQ; ++q) in[q] = Bb(v)[2 * pidx<NQ>(x, y, q) + s];
      eo_apply<1>(tb.Nt, in, out);
#pragma unroll
      for (int i = 0; i < NP; ++i) Cb(v)[2 * pidx<NQ>(x, y, i) + s] = out[i];
    }
    __syncthreads();
    // test y: Cb (nq,nq,np) -> Bb (nq,np,np)
    for (int u = threadIdx.x; u < VB * NQ * NP * 2; u += NT) {
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int x = pen % NQ, z = pen / NQ;
      C in[NQ], out[NP];
#pragma unroll
      for (int q = 0; q < NQ; ++q) in[q] = Cb(v)[2 * pidx<NQ>(x, q, z) + s];
      eo_apply<1>(tb.Nt, in, out);
#pragma unroll
      for (int i = 0; i < NP; ++i) Bb(v)[2 * pidx<NQ>(x, i, z) + s] = out[i];
    }
    __syncthreads();
    // test x: Bb (nq,np,np) -> add into the x-stage registers, then assemble
#pragma unroll
    for (int r = 0; r < XR; ++r) {
      const int u = threadIdx.x + r * NT;
      if (u >= XU) break;
      const int v = u % VB, s = (u / VB) & 1, pen = u / (2 * VB);
      const int y = pen % NP, z = pen / NP;
      C in[NQ], out[NP];
#pragma unroll
      for (int q = 0; q < NQ; ++q) in[q] = Bb(v)[2 * pidx<NQ>(q, y, z) + s];
      eo_apply<1>(tb.Nt, in, out);
      const int vec = vbase + v;
      if (vec < d.nvec) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          const long long I = gbc_node(d.mesh, cx, cy, cz, i, y, z);
          if (I < 0 || !GBC_IN_RANGE(GBC_SITE_HX64, I, d.mesh.M)) continue;
          if (d.Ycell)
            d.Ycell[(((long long)e * (NP * NP * NP) + i + NP * (y + NP * z)) * 2 + s) * d.nvec + vec] =
                cadd(yacc[r][i], out[i]);
          else
            atomic_add_c<T>(&d.Y[(I * 2 + s) * d.ldx + vec], cadd(yacc[r][i], out[i]));
        }
      }
    }
  }  // item loop
}

template <typename T, int NP, int NQ, int VB> constexpr size_t hx_local_smem() {
  constexpr int BUF = pbuf_points<NQ>();
  constexpr int VBASE = 3 * BUF * 2;
  constexpr int VSTRIDE = VBASE + ((24 - VBASE % 16) % 16);
  return sizeof(cplx<T>) * (size_t)VB * VSTRIDE;
}

template <typename T, int NP, int VB>
cudaError_t launch_hx_group_p(const HxJob* jobs, int n, cudaStream_t s) {
  static_assert(std::is_same<T, double>::value, "FP64 only (the FP32 cell apply is hx_cell.cuh)");
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
    d.Ycell = (cplx<T>*)jobs[i].Ycell;
    d.fields = (const T*)c->d_fields64;
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
  TablesEO<T, NP, NQ> tb;
  if (!make_tables_eo<T, NP, NQ>(c0, &tb)) return cudaErrorInvalidValue;
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

// Deterministic assembly: Y[I][s][v] += the results of every cell holding node I, added
// in a fixed order (cells by direction z, y, x, lower neighbour first).  Along each
// direction a node at grid index g is interior to cell g / p (local g % p), or, when
// g % p == 0, shared by cell g / p - 1 (local p; periodic wrap at 0) and cell g / p
// (local 0).
template <typename T>
__global__ void k_cell_gather(cplx<T>* __restrict__ Y, const cplx<T>* __restrict__ Ycell,
                              const MeshDev m, int nvec, int ldx) {
  const int np = m.p + 1;
  const long long np3 = (long long)np * np * np;
  const long long n = m.M * 2 * (long long)nvec;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(t % nvec);
    const long long rs = t / nvec;
    const int s = (int)(rs & 1);
    const long long I = rs >> 1;
    const long long f[3] = {I % m.nfree[0], (I / m.nfree[0]) % m.nfree[1],
                            I / ((long long)m.nfree[0] * m.nfree[1])};
    int cell[3][2], loc[3][2], cnt[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int g = (int)f[d] + (m.periodic[d] ? 0 : 1);
      const int q = g / m.p, r = g % m.p;
      if (r != 0) {
        cell[d][0] = q;
        loc[d][0] = r;
        cnt[d] = 1;
      } else {
        cnt[d] = 0;
        if (q > 0 || m.periodic[d]) {
          cell[d][cnt[d]] = q > 0 ? q - 1 : m.ncell[d] - 1;
          loc[d][cnt[d]++] = m.p;
        }
        if (q < m.ncell[d]) {
          cell[d][cnt[d]] = q;
          loc[d][cnt[d]++] = 0;
        }
      }
    }
    cplx<T> acc = cmake<cplx<T>>(0, 0);
    for (int a = 0; a < cnt[2]; ++a)
      for (int b = 0; b < cnt[1]; ++b)
        for (int c = 0; c < cnt[0]; ++c) {
          const long long e = cell[0][c] + (long long)m.ncell[0] * (cell[1][b] + (long long)m.ncell[1] * cell[2][a]);
          const long long l = loc[0][c] + np * (loc[1][b] + np * loc[2][a]);
          const cplx<T> y = Ycell[((e * np3 + l) * 2 + s) * nvec + v];
          acc.x += y.x;
          acc.y += y.y;
        }
    cplx<T>& o = Y[(I * 2 + s) * ldx + v];
    o.x += acc.x;
    o.y += acc.y;
  }
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
