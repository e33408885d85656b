// Quadrature-point gradient contraction for the backward pass of the filter.
//
//   g[e][c][q] += scale * w_q J * sum_v wv[v] Re( a_v(r_q)^H S_c b_v(r_q) ),
//   S = (I, sigma_x, sigma_y, sigma_z),  a_v(r_q) = sum_I A[I][.][v] N_I(r_q),
//
// i.e. the derivative of Re(a^H H b) with respect to V_eff and B_xc at every
// Gauss point (dH/dV_q = w_q J N(r_q) N(r_q)^T x I2 and dH/dB^d_q the same with
// sigma^d, Eq. FEHloc).  These are the density / magnetisation-density
// contractions of Eqs. rho and mag with the adjoint as the bra.
//
// Point-wise mode (A = B, wv = occupations): g[e][c][q] = scale * sum_v wv[v]
// Re(a_v^H S_c a_v), without w_q J, written (mode 1) or added (mode 2), is
// (rho, m_x, m_y, m_z) at the Gauss points (Eqs. rho, mag).
//
// One CTA owns one cell and walks all vectors in chunks of VB, so every g[e]
// row is written by exactly one CTA (no atomics).  Interpolation to the Gauss
// points is sum-factorised as in the cell apply (3 one-dimensional stages);
// the last stage leaves each lane with a z-pencil of Gauss-point values in
// registers, where the products are formed and accumulated.
#pragma once

#include "gbc_internal.h"

namespace gbc {

template <typename T> struct GradArgs {
  const cplx<T>* A;
  const cplx<T>* B;
  const double* wv;    // per-vector weights (null = 1)
  double* g;           // [E][4][NQ^3], accumulated
  int ldx, nvec;
  double scale;
  MeshDev mesh;
  int pointwise;       // 1: g = scale * sum, 2: g += scale * sum (no w_q J either way)
};

template <typename T, int NP, int NQ> struct InterpTab {
  T N[NP][NQ];
  double wq[NQ];
  double jac;
};

// Per-thread running sum over the vectors.  FP64 blocks add in FP64.  FP32 blocks
// add in FP32 with Kahan compensation (error ~2 ulp of the sum for any vector
// count) and convert once at the end: GB300's FP64 pipe is a small fraction of
// its FP32 rate, and a per-product FP64 add would dominate the kernel.
template <typename T> struct QAcc;
template <> struct QAcc<double> {
  double s;
  __device__ __forceinline__ void zero() { s = 0.0; }
  __device__ __forceinline__ void add(double w, double x) { s = fma(w, x, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct QAcc<float> {
  float s, c;   // sum, and the low-order part lost by the last additions (negated)
  __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float w, float x) {   // s += w x, compensated
    const float y = __fmaf_rn(w, x, -c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <int NQ> __device__ __forceinline__ int gidx(int x, int y, int z) {
  return x + y * (NQ + 1) + z * (NQ + 1) * (NQ + 1);
}

// interpolate the staged block in P1 (np^3 points, both spins) to the Gauss
// points; on return lane-owned z-pencils hold the values: out[s][qz]
template <typename T, int NP, int NQ, int TPV>
__device__ __forceinline__ void interp_to_pencils(cplx<T>* P1, cplx<T>* P2, int lane,
                                                  const InterpTab<T, NP, NQ>& tb,
                                                  cplx<T> (&out)[2][NQ]) {
  using C = cplx<T>;
  // x: P1 (np,np,np) -> P2 (nq,np,np)
  for (int pid = lane; pid < NP * NP; pid += TPV) {
    const int y = pid % NP, z = pid / NP;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C in[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = P1[2 * gidx<NQ>(j, y, z) + s];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T r = 0, im = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          r += tb.N[j][q] * in[j].x;
          im += tb.N[j][q] * in[j].y;
        }
        P2[2 * gidx<NQ>(q, y, z) + s] = cmake<C>(r, im);
      }
    }
  }
  __syncthreads();
  // y: P2 (nq,np,np) -> P1 (nq,nq,np)
  for (int pid = lane; pid < NQ * NP; pid += TPV) {
    const int x = pid % NQ, z = pid / NQ;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C in[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = P2[2 * gidx<NQ>(x, j, z) + s];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T r = 0, im = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          r += tb.N[j][q] * in[j].x;
          im += tb.N[j][q] * in[j].y;
        }
        P1[2 * gidx<NQ>(x, q, z) + s] = cmake<C>(r, im);
      }
    }
  }
  __syncthreads();
  // z: P1 (nq,nq,np) -> registers (lane owns pencil (x, y) = (lane % NQ, lane / NQ))
  if (lane < NQ * NQ) {
    const int x = lane % NQ, y = lane / NQ;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      C in[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) in[j] = P1[2 * gidx<NQ>(x, y, j) + s];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        T r = 0, im = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          r += tb.N[j][q] * in[j].x;
          im += tb.N[j][q] * in[j].y;
        }
        out[s][q] = cmake<C>(r, im);
      }
    }
  }
  __syncthreads();
}

template <typename T, int NP, int NQ, int VB, bool SAME>
__global__ void __launch_bounds__(VB * 64)
quad_grad_kernel(const GradArgs<T> a, const InterpTab<T, NP, NQ> tb) {
  using C = cplx<T>;
  constexpr int TPV = 64;
  constexpr int BUF = (NQ + 1) * (NQ + 1) * NQ;
  constexpr int VSTRIDE = 2 * BUF * 2 + 1;
  constexpr int NLOAD = (NP * NP * NP + TPV - 1) / TPV;   // cell nodes staged per lane
  // FP32: node rows computed once per CTA (fits the register budget of 3 CTAs per SM);
  // FP64 recomputes them per vector step (its accumulators leave no room)
  constexpr bool HOIST = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int v = threadIdx.x % VB;
  const int lane = threadIdx.x / VB;
  const int e = blockIdx.x;
  const int nx = a.mesh.ncell[0], ny = a.mesh.ncell[1];
  const int cx = e % nx, cy = (e / nx) % ny, cz = e / (nx * ny);
  C* P1 = buf + v * VSTRIDE;
  C* P2 = P1 + BUF * 2;
  // global row 2 I (< 2^31, checked by the launcher) and staging slot of the cell
  // nodes this lane loads (-1: none)
  auto node_of = [&](int k, int& row, int& slot) {
    const int i = lane + k * TPV;
    row = -1;
    slot = -1;
    if (i < NP * NP * NP) {
      const int ix = i % NP, iy = (i / NP) % NP, iz = i / (NP * NP);
      const long long I = gbc_node(a.mesh, cx, cy, cz, ix, iy, iz);
      row = I >= 0 ? (int)(2 * I) : -1;
      slot = gidx<NQ>(ix, iy, iz);
    }
  };
  int rows[HOIST ? NLOAD : 1], slots[HOIST ? NLOAD : 1];
  if constexpr (HOIST) {
#pragma unroll
    for (int k = 0; k < NLOAD; ++k) node_of(k, rows[k], slots[k]);
  }
  QAcc<T> acc[4][NQ];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[c][q].zero();

  for (int v0 = 0; v0 < a.nvec; v0 += VB) {
    const int vec = v0 + v;
    const bool vok = vec < a.nvec;
    C ua[2][NQ], ub[2][NQ];
#pragma unroll
    for (int which = 0; which < (SAME ? 1 : 2); ++which) {
      const cplx<T>* src = which == 0 ? a.A : a.B;
#pragma unroll(HOIST ? NLOAD : 1)
      for (int k = 0; k < NLOAD; ++k) {
        int row, slot;
        if constexpr (HOIST) {
          row = rows[k];
          slot = slots[k];
        } else {
          node_of(k, row, slot);
        }
        if (slot < 0) continue;
        C u = cmake<C>(0, 0), d = cmake<C>(0, 0);
        if (row >= 0 && vok) {
          u = src[(long long)row * a.ldx + vec];
          d = src[((long long)row + 1) * a.ldx + vec];
        }
        P1[2 * slot] = u;
        P1[2 * slot + 1] = d;
      }
      __syncthreads();
      if (which == 0)
        interp_to_pencils<T, NP, NQ, TPV>(P1, P2, lane, tb, ua);
      else
        interp_to_pencils<T, NP, NQ, TPV>(P1, P2, lane, tb, ub);
    }
    if (lane < NQ * NQ && vok) {
      const T w = (T)(a.wv ? a.wv[vec] : 1.0);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const C au = ua[0][q], ad = ua[1][q];
        if (SAME) {
          // |u|^2, |d|^2 and u* d: (rho, m) = (uu + dd, 2 Re, 2 Im, uu - dd)
          const T uu = au.x * au.x + au.y * au.y, dd = ad.x * ad.x + ad.y * ad.y;
          const T re = au.x * ad.x + au.y * ad.y, im = au.x * ad.y - au.y * ad.x;
          const T w2 = w + w;
          acc[0][q].add(w, uu + dd);
          acc[1][q].add(w2, re);
          acc[2][q].add(w2, im);
          acc[3][q].add(w, uu - dd);
        } else {
          const C bu = ub[0][q], bd = ub[1][q];
          // Re(a^H b), Re(a^H sx b), Re(a^H sy b), Re(a^H sz b)
          const T uu = au.x * bu.x + au.y * bu.y, dd = ad.x * bd.x + ad.y * bd.y;
          const T ud_re = au.x * bd.x + au.y * bd.y, du_re = ad.x * bu.x + ad.y * bu.y;
          const T ud_im = au.x * bd.y - au.y * bd.x, du_im = ad.x * bu.y - ad.y * bu.x;
          acc[0][q].add(w, uu + dd);
          acc[1][q].add(w, ud_re + du_re);
          acc[2][q].add(w, ud_im - du_im);
          acc[3][q].add(w, uu - dd);
        }
      }
    }
  }
  // reduce over the VB threads that own the same pencil, then write g[e]
  double* red = reinterpret_cast<double*>(smem_raw);   // [VB][64][4][NQ] overlays the buffers
  __syncthreads();
  if (lane < NQ * NQ) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < NQ; ++q) red[((v * 64 + lane) * 4 + c) * NQ + q] = acc[c][q].value();
  }
  __syncthreads();
  if (v == 0 && lane < NQ * NQ) {
    const int x = lane % NQ, y = lane / NQ;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int qz = 0; qz < NQ; ++qz) {
        double sum = 0.0;
        for (int w = 0; w < VB; ++w) sum += red[((w * 64 + lane) * 4 + c) * NQ + qz];
        const int q = (qz * NQ + y) * NQ + x;
        double* dst = &a.g[((size_t)e * 4 + c) * NQ * NQ * NQ + q];
        if (a.pointwise == 1) {
          *dst = a.scale * sum;
        } else if (a.pointwise == 2) {
          *dst += a.scale * sum;
        } else {
          const double wq = tb.wq[x] * tb.wq[y] * tb.wq[qz] * tb.jac;
          *dst += a.scale * wq * sum;
        }
      }
  }
}

template <typename T, int NP, int NQ, int VB> constexpr size_t quad_grad_smem() {
  const size_t bufs = sizeof(cplx<T>) * (size_t)VB * (2 * ((NQ + 1) * (NQ + 1) * NQ) * 2 + 1);
  const size_t red = sizeof(double) * (size_t)VB * 64 * 4 * NQ;
  return bufs > red ? bufs : red;
}

template <typename T, int NP, int VB>
cudaError_t launch_quad_grad_p(const gbc_ctx* c, const cplx<T>* A, const cplx<T>* B,
                               const double* wv, double scale, int nvec, int ldx, double* g,
                               int pointwise, cudaStream_t s) {
  constexpr int NQ = NP + 1;
  GradArgs<T> a{A, B, wv, g, ldx, nvec, scale, c->mesh, pointwise};
  InterpTab<T, NP, NQ> tb;
  for (int i = 0; i < NP; ++i)
    for (int q = 0; q < NQ; ++q) tb.N[i][q] = (T)c->tab.N1[i * NQ + q];
  for (int q = 0; q < NQ; ++q) tb.wq[q] = c->tab.gq_w[q];
  tb.jac = c->h[0] * c->h[1] * c->h[2] / 8.0;
  constexpr size_t smem = quad_grad_smem<T, NP, NQ, VB>();
  auto k = A == B ? quad_grad_kernel<T, NP, NQ, VB, true> : quad_grad_kernel<T, NP, NQ, VB, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (c->mesh.E <= 0 || nvec <= 0) return cudaSuccess;
  if (2 * (long long)c->mesh.M >= (1LL << 31)) return cudaErrorInvalidValue;   // 32-bit rows
  k<<<c->mesh.E, VB * 64, smem, s>>>(a, tb);
  return cudaGetLastError();
}

template <typename T, int VB>
cudaError_t launch_quad_grad_t(const gbc_ctx* c, const cplx<T>* A, const cplx<T>* B,
                               const double* wv, double scale, int nvec, int ldx, double* g,
                               int pointwise, cudaStream_t s) {
  switch (c->mesh.p) {
    case 2: return launch_quad_grad_p<T, 3, VB>(c, A, B, wv, scale, nvec, ldx, g, pointwise, s);
    case 3: return launch_quad_grad_p<T, 4, VB>(c, A, B, wv, scale, nvec, ldx, g, pointwise, s);
    case 4: return launch_quad_grad_p<T, 5, VB>(c, A, B, wv, scale, nvec, ldx, g, pointwise, s);
    case 5: return launch_quad_grad_p<T, 6, VB>(c, A, B, wv, scale, nvec, ldx, g, pointwise, s);
    case 6: return launch_quad_grad_p<T, 7, VB>(c, A, B, wv, scale, nvec, ldx, g, pointwise, s);
    case 7: return launch_quad_grad_p<T, 8, VB>(c, A, B, wv, scale, nvec, ldx, g, pointwise, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gbc
