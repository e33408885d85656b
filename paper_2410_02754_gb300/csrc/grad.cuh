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
};

template <typename T, int NP, int NQ> struct InterpTab {
  T N[NP][NQ];
  double wq[NQ];
  double jac;
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
