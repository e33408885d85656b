// Block kernels of the ChFSI cycle: the fused Chebyshev recurrence epilogue,
// M_D-weighted Gram matrices with FP64 accumulation, block rotation X <- X Q,
// and the FP64 vector helpers of the Lanczos bound estimate.
//
// Paper: Eq. chebfilt (three-term recurrence on M_D^-1 H, scaled), Sec. III.B.2
// (Rayleigh-Ritz: X^H H X, X^H M X, U = X Q).
#include <type_traits>

#include "gbc_internal.h"

namespace {

// Xout = a (M_D^-1 Y - c Xcur) - b Xprev ; Y <- 0
// (Xout may alias Xprev; Xprev may be null when b == 0)
template <typename T>
__global__ void k_cheb_step(cplx<T>* __restrict__ Y, const cplx<T>* Xcur, const cplx<T>* Xprev,
                            cplx<T>* Xout, const T* __restrict__ invmd, long long rows, int nvec,
                            int ldx, T a, T cshift, T b) {
  const long long n = rows * (long long)nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nvec;
    const int v = (int)(i - r * nvec);
    const long long o = r * ldx + v;
    const T w = invmd[r >> 1];
    const cplx<T> y = Y[o];
    const cplx<T> x = Xcur[o];
    cplx<T> out;
    out.x = a * (w * y.x - cshift * x.x);
    out.y = a * (w * y.y - cshift * x.y);
    if (Xprev) {
      const cplx<T> xp = Xprev[o];
      out.x -= b * xp.x;
      out.y -= b * xp.y;
    }
    Xout[o] = out;
    Y[o] = cmake<cplx<T>>(0, 0);
  }
}

// The same recurrence update for several systems in one launch (batched filter).
template <typename T>
__global__ void k_cheb_batch(const __grid_constant__ ChebBatch b) {
  const long long n = b.total;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int q = 0;
    for (int r = 1; r < b.njobs; ++r)
      if (i >= b.job[r].start) q = r;
    const ChebJob& j = b.job[q];
    const long long li = i - j.start;
    const long long r = li / j.nvec;
    const int v = (int)(li - r * j.nvec);
    const long long o = r * j.ldx + v;
    cplx<T>* Y = (cplx<T>*)j.Y;
    const cplx<T>* Xc = (const cplx<T>*)j.Xcur;
    const cplx<T>* Xp = (const cplx<T>*)j.Xprev;
    cplx<T>* Xo = (cplx<T>*)j.Xout;
    const T w = ((const T*)j.invmd)[r >> 1];
    const T a = (T)j.a, c = (T)j.c, bb = (T)j.b;
    const cplx<T> y = Y[o], x = Xc[o];
    cplx<T> out;
    out.x = a * (w * y.x - c * x.x);
    out.y = a * (w * y.y - c * x.y);
    if (Xp) {
      const cplx<T> xp = Xp[o];
      out.x -= bb * xp.x;
      out.y -= bb * xp.y;
    }
    Xo[o] = out;
    Y[o] = cmake<cplx<T>>(0, 0);
  }
}

// S[i][j] += sum_rows w(row) conj(X[row][i]) Y[row][j], FP64 accumulation.
// Block: 32 x 32 tile of S, 256 threads with 2 x 2 outputs each; rows staged
// 32 at a time; the grid's y dimension splits the rows into chunks.
constexpr int GT = 32;
template <typename T>
__global__ void __launch_bounds__(256)
k_gram(const cplx<T>* __restrict__ X, const cplx<T>* __restrict__ Yb, const double* __restrict__ md,
       long long rows, int nvec, int ldx, long long rows_per_chunk, double2* __restrict__ S) {
  __shared__ double2 xs[GT][GT + 1];
  __shared__ double2 ys[GT][GT + 1];
  // S is Hermitian: only the tiles on and above the diagonal (ti <= tj) are
  // computed; launch_hermitize mirrors them into the lower triangle
  const int ntile = (nvec + GT - 1) / GT;
  int ti = 0, tj = blockIdx.x;
  while (tj >= ntile - ti) {
    tj -= ntile - ti;
    ++ti;
  }
  tj += ti;
  const int i0 = ti * GT, j0 = tj * GT;
  const long long r0 = blockIdx.y * rows_per_chunk;
  const long long r1 = min(rows, r0 + rows_per_chunk);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double2 acc[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0, 0);
  for (long long rb = r0; rb < r1; rb += GT) {
    for (int t = threadIdx.x; t < GT * GT; t += 256) {
      const int rr = t / GT, cc = t % GT;
      const long long r = rb + rr;
      double2 xv = make_double2(0, 0), yv = make_double2(0, 0);
      if (r < r1) {
        const double w = md ? md[r >> 1] : 1.0;
        if (i0 + cc < nvec) {
          const cplx<T> t1 = X[r * ldx + i0 + cc];
          xv = make_double2((double)t1.x * w, (double)t1.y * w);
        }
        if (j0 + cc < nvec) {
          const cplx<T> t2 = Yb[r * ldx + j0 + cc];
          yv = make_double2((double)t2.x, (double)t2.y);
        }
      }
      xs[rr][cc] = xv;
      ys[rr][cc] = yv;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < GT; ++rr) {
      const double2 x0 = xs[rr][2 * tx], x1 = xs[rr][2 * tx + 1];
      const double2 y0 = ys[rr][2 * ty], y1 = ys[rr][2 * ty + 1];
      // conj(x) * y
      acc[0][0].x += x0.x * y0.x + x0.y * y0.y;
      acc[0][0].y += x0.x * y0.y - x0.y * y0.x;
      acc[0][1].x += x0.x * y1.x + x0.y * y1.y;
      acc[0][1].y += x0.x * y1.y - x0.y * y1.x;
      acc[1][0].x += x1.x * y0.x + x1.y * y0.y;
      acc[1][0].y += x1.x * y0.y - x1.y * y0.x;
      acc[1][1].x += x1.x * y1.x + x1.y * y1.y;
      acc[1][1].y += x1.x * y1.y - x1.y * y1.x;
    }
    __syncthreads();
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + 2 * tx + a, j = j0 + 2 * ty + b;
      if (i < nvec && j < nvec) {
        atomicAdd(&S[(size_t)i * nvec + j].x, acc[a][b].x);
        atomicAdd(&S[(size_t)i * nvec + j].y, acc[a][b].y);
      }
    }
}

// S = X^H diag(w) Y (Hermitian, upper-triangle tiles as k_gram) for an FP32 block
// X and Y either the same FP32 block (w = M_D: CholGS) or an FP64 block (w = 1:
// Rayleigh-Ritz with Y = H X), in float-float arithmetic on the FP32 pipes.  The
// X side carries the weight as a two-FP32 value (x*wh exact by FMA, + x*wl), an
// FP64 Y entry is split into two FP32 words on load; per real product the rounded
// product of the high words and its exact error, plus the two cross terms, are
// TwoSum-accumulated into (hi, lo), and each CTA adds hi + lo to S in FP64.
__device__ __forceinline__ void ff_acc(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float pe = __fmaf_rn(ah, bh, -p);                  // ah*bh - p, exact
  const float small = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
  const float t = __fadd_rn(sh, p);                        // TwoSum(sh, p)
  const float bb = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, __fadd_rn(pe, small)));
}

template <typename TY>
__global__ void __launch_bounds__(256)
k_gram_ff(const float2* __restrict__ X, int ldx, const cplx<TY>* __restrict__ Yb, int ldy,
          const double* __restrict__ md, long long rows, int nvec, long long rows_per_chunk,
          double2* __restrict__ S) {
  __shared__ float2 xh[GT][GT + 1], xl[GT][GT + 1];
  __shared__ float2 yh[GT][GT + 1], yl[GT][GT + 1];
  const int ntile = (nvec + GT - 1) / GT;
  int ti = 0, tj = blockIdx.x;
  while (tj >= ntile - ti) {
    tj -= ntile - ti;
    ++ti;
  }
  tj += ti;
  const int i0 = ti * GT, j0 = tj * GT;
  const long long r0 = blockIdx.y * rows_per_chunk;
  const long long r1 = min(rows, r0 + rows_per_chunk);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float ah[2][2][2], al[2][2][2];   // [a][b][re / im]
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int q = 0; q < 2; ++q) ah[a][b][q] = al[a][b][q] = 0.f;
  for (long long rb = r0; rb < r1; rb += GT) {
    for (int t = threadIdx.x; t < GT * GT; t += 256) {
      const int rr = t / GT, cc = t % GT;
      const long long r = rb + rr;
      float2 vh = make_float2(0.f, 0.f), vl = vh, uh = vh, ul = vh;
      if (r < r1) {
        if (i0 + cc < nvec) {
          const float2 x = X[r * ldx + i0 + cc];
          if (md) {
            const double w = md[r >> 1];
            const float wh = (float)w, wl = (float)(w - (double)wh);
            const float ph = __fmul_rn(x.x, wh), qh = __fmul_rn(x.y, wh);
            vh = make_float2(ph, qh);
            vl = make_float2(__fmaf_rn(x.x, wl, __fmaf_rn(x.x, wh, -ph)),
                             __fmaf_rn(x.y, wl, __fmaf_rn(x.y, wh, -qh)));
          } else {
            vh = x;
          }
        }
        if (j0 + cc < nvec) {
          const cplx<TY> y = Yb[r * ldy + j0 + cc];
          const float hx = (float)y.x, hy = (float)y.y;
          uh = make_float2(hx, hy);
          ul = make_float2((float)((double)y.x - (double)hx), (float)((double)y.y - (double)hy));
        }
      }
      xh[rr][cc] = vh;
      xl[rr][cc] = vl;
      yh[rr][cc] = uh;
      yl[rr][cc] = ul;
    }
    __syncthreads();
#pragma unroll 2
    for (int rr = 0; rr < GT; ++rr) {
      float2 xa[2], xb[2], ya[2], yb[2];
      xa[0] = xh[rr][2 * tx];
      xa[1] = xh[rr][2 * tx + 1];
      xb[0] = xl[rr][2 * tx];
      xb[1] = xl[rr][2 * tx + 1];
      ya[0] = yh[rr][2 * ty];
      ya[1] = yh[rr][2 * ty + 1];
      yb[0] = yl[rr][2 * ty];
      yb[1] = yl[rr][2 * ty + 1];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          // conj(x) * y: re = xr yr + xi yi, im = xr yi - xi yr
          ff_acc(ah[a][b][0], al[a][b][0], xa[a].x, xb[a].x, ya[b].x, yb[b].x);
          ff_acc(ah[a][b][0], al[a][b][0], xa[a].y, xb[a].y, ya[b].y, yb[b].y);
          ff_acc(ah[a][b][1], al[a][b][1], xa[a].x, xb[a].x, ya[b].y, yb[b].y);
          ff_acc(ah[a][b][1], al[a][b][1], -xa[a].y, -xb[a].y, ya[b].x, yb[b].x);
        }
    }
    __syncthreads();
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + 2 * tx + a, j = j0 + 2 * ty + b;
      if (i < nvec && j < nvec) {
        atomicAdd(&S[(size_t)i * nvec + j].x, (double)ah[a][b][0] + (double)al[a][b][0]);
        atomicAdd(&S[(size_t)i * nvec + j].y, (double)ah[a][b][1] + (double)al[a][b][1]);
      }
    }
}

// Out[row][j] = sum_i X[row][i] Q[i][j]; 64 x 64 output tile, K-steps of 16.
constexpr int RT = 64, KT = 16;
template <typename T>
__global__ void __launch_bounds__(256)
k_rotate(const cplx<T>* __restrict__ X, const double2* __restrict__ Q, cplx<T>* __restrict__ Out,
         long long rows, int nvec, int ldx) {
  using C = cplx<T>;
  __shared__ C xs[RT][KT + 1];
  __shared__ C qs[KT][RT + 1];
  const int ntj = (nvec + RT - 1) / RT;
  const long long r0 = (long long)(blockIdx.x / ntj) * RT;
  const int j0 = (blockIdx.x % ntj) * RT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  C acc[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) acc[a][b] = cmake<C>(0, 0);
  for (int k0 = 0; k0 < nvec; k0 += KT) {
    for (int t = threadIdx.x; t < RT * KT; t += 256) {
      const int rr = t / KT, kk = t % KT;
      const long long r = r0 + rr;
      C v = cmake<C>(0, 0);
      if (r < rows && k0 + kk < nvec) v = X[r * ldx + k0 + kk];
      xs[rr][kk] = v;
    }
    for (int t = threadIdx.x; t < KT * RT; t += 256) {
      const int kk = t / RT, jj = t % RT;
      C v = cmake<C>(0, 0);
      if (k0 + kk < nvec && j0 + jj < nvec) {
        const double2 q = Q[(size_t)(k0 + kk) * nvec + j0 + jj];
        v = cmake<C>(q.x, q.y);
      }
      qs[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      C xv[4], qv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xv[a] = xs[ty + 16 * a][kk];
#pragma unroll
      for (int b = 0; b < 4; ++b) qv[b] = qs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc[a][b].x += xv[a].x * qv[b].x - xv[a].y * qv[b].y;
          acc[a][b].y += xv[a].x * qv[b].y + xv[a].y * qv[b].x;
        }
    }
    __syncthreads();
  }
  for (int a = 0; a < 4; ++a) {
    const long long r = r0 + ty + 16 * a;
    if (r >= rows) continue;
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      if (j < nvec) Out[r * ldx + j] = acc[a][b];
    }
  }
}

template <typename T>
__global__ void k_copy_block(const cplx<T>* __restrict__ X, cplx<T>* __restrict__ Out,
                             long long rows, int nvec, int ldx) {
  const long long n = rows * (long long)nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nvec;
    const int v = (int)(i - r * nvec);
    Out[r * ldx + v] = X[r * ldx + v];
  }
}

// ---- residual-split recurrence (Hamiltonian-times-residual form) ------------------
// R = ((M_D^-1 HX - c X)/e - X lam_hat[col]) from FP64 inputs, stored in T;
// also Z1 = sigma1 R.
template <typename T>
__global__ void k_split_init(const double2* __restrict__ HX, const double2* __restrict__ X64,
                             const double* __restrict__ invmd, const double* __restrict__ lam_hat,
                             cplx<T>* __restrict__ R, cplx<T>* __restrict__ Z1, long long rows,
                             int nvec, int ldx, int ld64, double c, double inv_e, double sigma1) {
  const long long n = rows * (long long)nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nvec;
    const int v = (int)(i - r * nvec);
    const double w = invmd[r >> 1];
    const double2 h = HX[r * ld64 + v], x = X64[r * ld64 + v];
    const double lh = lam_hat[v];
    const double rr = (w * h.x - c * x.x) * inv_e - lh * x.x;
    const double ri = (w * h.y - c * x.y) * inv_e - lh * x.y;
    R[r * ldx + v] = cmake<cplx<T>>(rr, ri);
    Z1[r * ldx + v] = cmake<cplx<T>>(sigma1 * rr, sigma1 * ri);
  }
}

// Zout = a (M_D^-1 Y - c Zcur) - b Zprev + g[col] R ; Y <- 0   (Zout may alias Zprev)
template <typename T>
__global__ void k_split_step(cplx<T>* __restrict__ Y, const cplx<T>* Zcur, const cplx<T>* Zprev,
                             cplx<T>* Zout, const cplx<T>* __restrict__ R,
                             const T* __restrict__ invmd, const double* __restrict__ g,
                             long long rows, int nvec, int ldx, T a, T cshift, T b) {
  const long long n = rows * (long long)nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nvec;
    const int v = (int)(i - r * nvec);
    const long long o = r * ldx + v;
    const T w = invmd[r >> 1];
    const cplx<T> y = Y[o], z = Zcur[o], zp = Zprev[o], rv = R[o];
    const T gv = (T)g[v];
    cplx<T> out;
    out.x = a * (w * y.x - cshift * z.x) - b * zp.x + gv * rv.x;
    out.y = a * (w * y.y - cshift * z.y) - b * zp.y + gv * rv.y;
    Zout[o] = out;
    Y[o] = cmake<cplx<T>>(0, 0);
  }
}

// X = X D[col] + Z
template <typename T>
__global__ void k_split_final(cplx<T>* X, const cplx<T>* __restrict__ Z, const double* __restrict__ D,
                              long long rows, int nvec, int ldx) {
  const long long n = rows * (long long)nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nvec;
    const int v = (int)(i - r * nvec);
    const long long o = r * ldx + v;
    const T d = (T)D[v];
    const cplx<T> x = X[o], z = Z[o];
    X[o] = cmake<cplx<T>>(d * x.x + z.x, d * x.y + z.y);
  }
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ X, int ldx, B* __restrict__ Out, int ldo,
                          long long rows, int nvec) {
  const long long n = rows * (long long)nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nvec;
    const int v = (int)(i - r * nvec);
    const A a = X[r * ldx + v];
    B b;
    b.x = a.x;
    b.y = a.y;
    Out[r * ldo + v] = b;
  }
}

// ---- FP64 vector helpers (Lanczos) -------------------------------------------
// out += sum_I md[I] sum_s conj(a[I][s]) b[I][s]   (n = M spinors); with part, each
// block's sum goes to part[blockIdx.x] instead (k_sum_parts adds them in order)
__global__ void k_mdot(const double2* __restrict__ a, const double2* __restrict__ b,
                       const double* __restrict__ md, long long n, double2* out, double2* part) {
  __shared__ double2 red[256];
  double2 acc = make_double2(0, 0);
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < n;
       I += (long long)gridDim.x * blockDim.x) {
    const double w = md[I];
    for (int s = 0; s < 2; ++s) {
      const double2 x = a[2 * I + s], y = b[2 * I + s];
      acc.x += w * (x.x * y.x + x.y * y.y);
      acc.y += w * (x.x * y.y - x.y * y.x);
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[threadIdx.x].x += red[threadIdx.x + s].x;
      red[threadIdx.x].y += red[threadIdx.x + s].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (part) {
      part[blockIdx.x] = red[0];
    } else {
      atomicAdd(&out->x, red[0].x);
      atomicAdd(&out->y, red[0].y);
    }
  }
}

// out = sum_b part[b], b = 0 .. nb-1 in order (one thread)
__global__ void k_sum_parts(const double2* __restrict__ part, int nb, double2* out) {
  double2 acc = make_double2(0, 0);
  for (int b = 0; b < nb; ++b) {
    acc.x += part[b].x;
    acc.y += part[b].y;
  }
  *out = acc;
}

// y -= (alpha_scale * alpha) x   (alpha read on the device)
__global__ void k_axpy_c(double2* y, const double2* __restrict__ x, const double2* alpha,
                         double alpha_scale, long long n) {
  const double2 al = make_double2(alpha->x * alpha_scale, alpha->y * alpha_scale);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    y[i].x -= al.x * v.x - al.y * v.y;
    y[i].y -= al.x * v.y + al.y * v.x;
  }
}

__global__ void k_scale_c(double2* y, const double2* __restrict__ x, double scale, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    y[i] = make_double2(x[i].x * scale, x[i].y * scale);
  }
}

__global__ void k_divmass(double2* y, const double* __restrict__ invmd, long long M) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 2 * M;
       i += (long long)gridDim.x * blockDim.x) {
    const double w = invmd[i >> 1];
    y[i].x *= w;
    y[i].y *= w;
  }
}

inline unsigned grid_for(long long n, int threads = 256) {
  long long g = (n + threads - 1) / threads;
  const long long cap = 64LL * gbc_sm_count();
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

// Recurrence update on the listed node rows only (the rows the fused cell
// apply leaves to atomics: nodes on cell faces), Y zeroed there for the next step
// except on the first nkeep listed rows, which the next step's nonlocal expansion
// overwrites (rows in some atom's support).
template <typename T>
__global__ void k_cheb_rows(cplx<T>* __restrict__ Y, const cplx<T>* Xcur, const cplx<T>* Xprev,
                            cplx<T>* Xout, const T* __restrict__ invmd,
                            const long long* __restrict__ rows, long long nrows, long long nkeep,
                            long long M, int nvec, int ldx, T a, T cshift, T b) {
  const long long n = nrows * 2 * (long long)nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long rs = i / nvec;
    const int v = (int)(i - rs * nvec);
    const long long node = rows[rs >> 1];
    if (!GBC_IN_RANGE(GBC_SITE_FACE_ROW, node, M)) continue;
    const long long o = (node * 2 + (rs & 1)) * ldx + v;
    const T w = invmd[node];
    const cplx<T> y = Y[o];
    const cplx<T> x = Xcur[o];
    cplx<T> out;
    out.x = a * (w * y.x - cshift * x.x);
    out.y = a * (w * y.y - cshift * x.y);
    if (Xprev) {
      const cplx<T> xp = Xprev[o];
      out.x -= b * xp.x;
      out.y -= b * xp.y;
    }
    Xout[o] = out;
    if ((rs >> 1) >= nkeep) Y[o] = cmake<cplx<T>>(0, 0);   // rows below nkeep: overwritten next step
  }
}

template <typename T>
cudaError_t launch_cheb_rows(cplx<T>* Y, const cplx<T>* Xcur, const cplx<T>* Xprev, cplx<T>* Xout,
                             const T* invmd, const long long* rows, long long nrows, long long nkeep,
                             long long M, int nvec, int ldx, double a, double cshift, double b,
                             cudaStream_t s) {
  if (nrows <= 0 || nvec <= 0) return cudaSuccess;
  k_cheb_rows<T><<<grid_for(nrows * 2 * nvec), 256, 0, s>>>(Y, Xcur, Xprev, Xout, invmd, rows,
                                                            nrows, nkeep, M, nvec, ldx, (T)a,
                                                            (T)cshift, (T)b);
  return cudaGetLastError();
}
template cudaError_t launch_cheb_rows<float>(float2*, const float2*, const float2*, float2*,
                                             const float*, const long long*, long long, long long,
                                             long long, int, int, double, double, double,
                                             cudaStream_t);
template cudaError_t launch_cheb_rows<double>(double2*, const double2*, const double2*, double2*,
                                              const double*, const long long*, long long, long long,
                                              long long, int, int, double, double, double,
                                              cudaStream_t);

// launch_cheb_rows over several systems in one launch (batched filter)
template <typename T>
__global__ void k_cheb_rows_batch(const __grid_constant__ ChebRowsBatch b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < b.total;
       i += (long long)gridDim.x * blockDim.x) {
    int q = 0;
    for (int r = 1; r < b.njobs; ++r)
      if (i >= b.job[r].start) q = r;
    const ChebRowsJob& j = b.job[q];
    const long long li = i - j.start;
    const long long rs = li / j.nvec;
    const int v = (int)(li - rs * j.nvec);
    const long long node = j.rows[rs >> 1];
    if (!GBC_IN_RANGE(GBC_SITE_FACE_ROW, node, j.M)) continue;
    const long long o = (node * 2 + (rs & 1)) * j.ldx + v;
    cplx<T>* Y = (cplx<T>*)j.Y;
    const cplx<T> y = Y[o];
    const cplx<T> x = ((const cplx<T>*)j.Xcur)[o];
    const T w = ((const T*)j.invmd)[node];
    const T a = (T)j.a, c = (T)j.c, bb = (T)j.b;
    cplx<T> out;
    out.x = a * (w * y.x - c * x.x);
    out.y = a * (w * y.y - c * x.y);
    if (j.Xprev) {
      const cplx<T> xp = ((const cplx<T>*)j.Xprev)[o];
      out.x -= bb * xp.x;
      out.y -= bb * xp.y;
    }
    ((cplx<T>*)j.Xout)[o] = out;
    if ((rs >> 1) >= j.nkeep) Y[o] = cmake<cplx<T>>(0, 0);
  }
}

template <typename T>
cudaError_t launch_cheb_rows_batch(const ChebRowsBatch& b, cudaStream_t s) {
  if (b.total <= 0) return cudaSuccess;
  k_cheb_rows_batch<T><<<grid_for(b.total), 256, 0, s>>>(b);
  return cudaGetLastError();
}
template cudaError_t launch_cheb_rows_batch<float>(const ChebRowsBatch&, cudaStream_t);
template cudaError_t launch_cheb_rows_batch<double>(const ChebRowsBatch&, cudaStream_t);

template <typename T>
cudaError_t launch_cheb_step(const cplx<T>* Y, const cplx<T>* Xcur, const cplx<T>* Xprev,
                             cplx<T>* Xout, const T* invmd, long long M, int nvec, int ldx,
                             double a, double cshift, double b, cudaStream_t s) {
  const long long rows = 2 * M;
  k_cheb_step<T><<<grid_for(rows * nvec), 256, 0, s>>>(const_cast<cplx<T>*>(Y), Xcur, Xprev, Xout,
                                                       invmd, rows, nvec, ldx, (T)a, (T)cshift,
                                                       (T)b);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cheb_batch(const ChebBatch& b, cudaStream_t s) {
  if (b.total <= 0) return cudaSuccess;
  k_cheb_batch<T><<<grid_for(b.total), 256, 0, s>>>(b);
  return cudaGetLastError();
}
template cudaError_t launch_cheb_batch<float>(const ChebBatch&, cudaStream_t);
template cudaError_t launch_cheb_batch<double>(const ChebBatch&, cudaStream_t);

template <typename T>
cudaError_t launch_gram(const cplx<T>* X, const cplx<T>* Y, const double* md, long long M,
                        int nvec, int ldx, double2* S, cudaStream_t s) {
  const long long rows = 2 * M;
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(double2) * (size_t)nvec * nvec, s);
  if (e != cudaSuccess) return e;
  const int ntile = (nvec + GT - 1) / GT;
  const long long tiles = (long long)ntile * (ntile + 1) / 2;   // upper-triangle tiles
  // enough row chunks to fill the GPU a few times over
  long long nchunk = (8LL * gbc_sm_count() + tiles - 1) / tiles;
  long long per = (rows + nchunk - 1) / nchunk;
  per = ((per + GT - 1) / GT) * GT;
  if (per < GT) per = GT;
  nchunk = (rows + per - 1) / per;
  dim3 grid((unsigned)tiles, (unsigned)nchunk);
  k_gram<T><<<grid, 256, 0, s>>>(X, Y, md, rows, nvec, ldx, per, S);
  return cudaGetLastError();
}

// Out[row][j] = sum_i X[row][i] Q[i][j] for an FP32 block X and an FP64 Q given as
// Q = Qh + Ql (FP32 pairs), accumulated in two-FP32 (float-float) arithmetic on
// the FP32 pipes and rounded to FP32 once: the result of an FP64 product rounded
// to FP32, at several times the FP64 rate.  Per real product x*q: the rounded
// product and its exact error (FMA), a TwoSum into the high word, the error
// terms and x*Ql into the low word.  Intrinsics keep every step uncontracted.
__device__ __forceinline__ void ff_mac(float& sh, float& sl, float x, float qh, float ql) {
  const float p = __fmul_rn(x, qh);
  const float pe = __fmaf_rn(x, qh, -p);                   // x*qh - p, exact
  const float t = __fadd_rn(sh, p);                        // TwoSum(sh, p)
  const float bb = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  sh = t;
  sl = __fmaf_rn(x, ql, __fadd_rn(sl, __fadd_rn(err, pe)));
}

__global__ void __launch_bounds__(256)
k_rotate_ff(const float2* __restrict__ X, const float2* __restrict__ Qh,
            const float2* __restrict__ Ql, float2* __restrict__ Out, long long rows, int nvec,
            int ldx) {
  __shared__ float2 xs[RT][KT + 1];
  __shared__ float2 qhs[KT][RT + 1];
  __shared__ float2 qls[KT][RT + 1];
  const int ntj = (nvec + RT - 1) / RT;
  const long long r0 = (long long)(blockIdx.x / ntj) * RT;
  const int j0 = (blockIdx.x % ntj) * RT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float2 ah[4][4], al[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      ah[a][b] = make_float2(0.f, 0.f);
      al[a][b] = make_float2(0.f, 0.f);
    }
  for (int k0 = 0; k0 < nvec; k0 += KT) {
    for (int t = threadIdx.x; t < RT * KT; t += 256) {
      const int rr = t / KT, kk = t % KT;
      const long long r = r0 + rr;
      float2 v = make_float2(0.f, 0.f);
      if (r < rows && k0 + kk < nvec) v = X[r * ldx + k0 + kk];
      xs[rr][kk] = v;
    }
    for (int t = threadIdx.x; t < KT * RT; t += 256) {
      const int kk = t / RT, jj = t % RT;
      float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
      if (k0 + kk < nvec && j0 + jj < nvec) {
        h = Qh[(size_t)(k0 + kk) * nvec + j0 + jj];
        l = Ql[(size_t)(k0 + kk) * nvec + j0 + jj];
      }
      qhs[kk][jj] = h;
      qls[kk][jj] = l;
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < KT; ++kk) {
      float2 xv[4], hv[4], lv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xv[a] = xs[ty + 16 * a][kk];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        hv[b] = qhs[kk][tx + 16 * b];
        lv[b] = qls[kk][tx + 16 * b];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          // (x.re + i x.im)(q.re + i q.im)
          ff_mac(ah[a][b].x, al[a][b].x, xv[a].x, hv[b].x, lv[b].x);
          ff_mac(ah[a][b].x, al[a][b].x, -xv[a].y, hv[b].y, lv[b].y);
          ff_mac(ah[a][b].y, al[a][b].y, xv[a].x, hv[b].y, lv[b].y);
          ff_mac(ah[a][b].y, al[a][b].y, xv[a].y, hv[b].x, lv[b].x);
        }
    }
    __syncthreads();
  }
  for (int a = 0; a < 4; ++a) {
    const long long r = r0 + ty + 16 * a;
    if (r >= rows) continue;
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      if (j < nvec)
        Out[r * ldx + j] = make_float2(__fadd_rn(ah[a][b].x, al[a][b].x),
                                       __fadd_rn(ah[a][b].y, al[a][b].y));
    }
  }
}

// Q (FP64, n x n) -> Qh = fl32(Q), Ql = fl32(Q - Qh)
__global__ void k_split_q(const double2* __restrict__ Q, float2* __restrict__ Qh,
                          float2* __restrict__ Ql, long long n2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n2) return;
  const double2 q = Q[t];
  const float hx = (float)q.x, hy = (float)q.y;
  Qh[t] = make_float2(hx, hy);
  Ql[t] = make_float2((float)(q.x - (double)hx), (float)(q.y - (double)hy));
}

template <typename T>
cudaError_t launch_rotate(const cplx<T>* X, const double2* Q, cplx<T>* Out, long long M, int nvec,
                          int ldx, cudaStream_t s) {
  const long long rows = 2 * M;
  const long long nb = ((rows + RT - 1) / RT) * ((nvec + RT - 1) / RT);
  k_rotate<T><<<(unsigned)nb, 256, 0, s>>>(X, Q, Out, rows, nvec, ldx);
  return cudaGetLastError();
}

template <typename TY>
cudaError_t launch_gram_ff(const float2* X, int ldx, const cplx<TY>* Y, int ldy, const double* md,
                           long long M, int nvec, double2* S, cudaStream_t s) {
  const long long rows = 2 * M;
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(double2) * (size_t)nvec * nvec, s);
  if (e != cudaSuccess) return e;
  const int ntile = (nvec + GT - 1) / GT;
  const long long tiles = (long long)ntile * (ntile + 1) / 2;   // upper-triangle tiles
  long long nchunk = (8LL * gbc_sm_count() + tiles - 1) / tiles;
  long long per = (rows + nchunk - 1) / nchunk;
  per = ((per + GT - 1) / GT) * GT;
  if (per < GT) per = GT;
  nchunk = (rows + per - 1) / per;
  dim3 grid((unsigned)tiles, (unsigned)nchunk);
  k_gram_ff<TY><<<grid, 256, 0, s>>>(X, ldx, Y, ldy, md, rows, nvec, per, S);
  return cudaGetLastError();
}
template cudaError_t launch_gram_ff<float>(const float2*, int, const float2*, int, const double*,
                                           long long, int, double2*, cudaStream_t);
template cudaError_t launch_gram_ff<double>(const float2*, int, const double2*, int, const double*,
                                            long long, int, double2*, cudaStream_t);

cudaError_t launch_rotate_ff(const float2* X, const double2* Q, float2* Qsplit, float2* Out,
                             long long M, int nvec, int ldx, cudaStream_t s) {
  const long long n2 = (long long)nvec * nvec;
  k_split_q<<<grid_for(n2), 256, 0, s>>>(Q, Qsplit, Qsplit + n2, n2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long rows = 2 * M;
  const long long nb = ((rows + RT - 1) / RT) * ((nvec + RT - 1) / RT);
  k_rotate_ff<<<(unsigned)nb, 256, 0, s>>>(X, Qsplit, Qsplit + n2, Out, rows, nvec, ldx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy_block(const cplx<T>* X, cplx<T>* Out, long long M, int nvec, int ldx,
                              cudaStream_t s) {
  const long long rows = 2 * M;
  k_copy_block<T><<<grid_for(rows * nvec), 256, 0, s>>>(X, Out, rows, nvec, ldx);
  return cudaGetLastError();
}

cudaError_t launch_convert_block(const float2* X, int ldx, double2* Out, int ldo, long long M,
                                 int nvec, cudaStream_t s) {
  k_convert<float2, double2><<<grid_for(2 * M * nvec), 256, 0, s>>>(X, ldx, Out, ldo, 2 * M, nvec);
  return cudaGetLastError();
}
cudaError_t launch_convert_block(const double2* X, int ldx, float2* Out, int ldo, long long M,
                                 int nvec, cudaStream_t s) {
  k_convert<double2, float2><<<grid_for(2 * M * nvec), 256, 0, s>>>(X, ldx, Out, ldo, 2 * M, nvec);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_split_init(const double2* HX, const double2* X64, const double* invmd,
                              const double* lam_hat, cplx<T>* R, cplx<T>* Z1, long long M, int nvec,
                              int ldx, int ld64, double c, double inv_e, double sigma1,
                              cudaStream_t s) {
  k_split_init<T><<<grid_for(2 * M * nvec), 256, 0, s>>>(HX, X64, invmd, lam_hat, R, Z1, 2 * M,
                                                         nvec, ldx, ld64, c, inv_e, sigma1);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_split_step(cplx<T>* Y, const cplx<T>* Zcur, const cplx<T>* Zprev, cplx<T>* Zout,
                              const cplx<T>* R, const T* invmd, const double* g, long long M,
                              int nvec, int ldx, double a, double cshift, double b, cudaStream_t s) {
  k_split_step<T><<<grid_for(2 * M * nvec), 256, 0, s>>>(Y, Zcur, Zprev, Zout, R, invmd, g, 2 * M,
                                                         nvec, ldx, (T)a, (T)cshift, (T)b);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_split_final(cplx<T>* X, const cplx<T>* Z, const double* D, long long M, int nvec,
                               int ldx, cudaStream_t s) {
  k_split_final<T><<<grid_for(2 * M * nvec), 256, 0, s>>>(X, Z, D, 2 * M, nvec, ldx);
  return cudaGetLastError();
}
#define INST_SPLIT(T)                                                                          \
  template cudaError_t launch_split_init<T>(const double2*, const double2*, const double*,     \
                                            const double*, cplx<T>*, cplx<T>*, long long, int, \
                                            int, int, double, double, double, cudaStream_t);   \
  template cudaError_t launch_split_step<T>(cplx<T>*, const cplx<T>*, const cplx<T>*, cplx<T>*, \
                                            const cplx<T>*, const T*, const double*, long long, \
                                            int, int, double, double, double, cudaStream_t);   \
  template cudaError_t launch_split_final<T>(cplx<T>*, const cplx<T>*, const double*, long long, \
                                             int, int, cudaStream_t);
INST_SPLIT(float)
INST_SPLIT(double)

cudaError_t launch_mdot(const double2* a, const double2* b, const double* md, long long n,
                        double2* out, cudaStream_t s, double2* part) {
  const unsigned nb = grid_for(n);
  if (part) {
    k_mdot<<<nb, 256, 0, s>>>(a, b, md, n, out, part);
    k_sum_parts<<<1, 1, 0, s>>>(part, (int)nb, out);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double2), s);
  if (e != cudaSuccess) return e;
  k_mdot<<<nb, 256, 0, s>>>(a, b, md, n, out, nullptr);
  return cudaGetLastError();
}
size_t mdot_part_bytes(long long n) { return sizeof(double2) * grid_for(n); }
cudaError_t launch_axpy_c(double2* y, const double2* x, const double2* alpha_dev,
                          double alpha_scale, long long n, cudaStream_t s) {
  k_axpy_c<<<grid_for(n), 256, 0, s>>>(y, x, alpha_dev, alpha_scale, n);
  return cudaGetLastError();
}
cudaError_t launch_scale_c(double2* y, const double2* x, double scale, long long n,
                           cudaStream_t s) {
  k_scale_c<<<grid_for(n), 256, 0, s>>>(y, x, scale, n);
  return cudaGetLastError();
}
cudaError_t launch_divmass(double2* y, const double* invmd, long long M, cudaStream_t s) {
  k_divmass<<<grid_for(2 * M), 256, 0, s>>>(y, invmd, M);
  return cudaGetLastError();
}

#define INST(T)                                                                                 \
  template cudaError_t launch_cheb_step<T>(const cplx<T>*, const cplx<T>*, const cplx<T>*,      \
                                           cplx<T>*, const T*, long long, int, int, double,     \
                                           double, double, cudaStream_t);                        \
  template cudaError_t launch_gram<T>(const cplx<T>*, const cplx<T>*, const double*, long long, \
                                      int, int, double2*, cudaStream_t);                        \
  template cudaError_t launch_rotate<T>(const cplx<T>*, const double2*, cplx<T>*, long long,    \
                                        int, int, cudaStream_t);                                 \
  template cudaError_t launch_copy_block<T>(const cplx<T>*, cplx<T>*, long long, int, int,      \
                                            cudaStream_t);
INST(float)
INST(double)

GBC_CHECK_WORD_ACCESSOR(gbc_check_word_blas)
