// Self-consistent-field steps around the eigensolver, on the device.
//
// * gbc_scf_fields: V_eff = V_ext + V_xc and B_xc at the Gauss points from the
//   densities (rho, m) of gbc_density_dev, written into the context's fields.
//   The exchange-correlation term is a closed-form stand-in for the paper's PBE
//   (Eqs. disvxc / disbxc for a functional without gradients): exchange-only
//   local spin density for a noncollinear density, rho_up/dn = (rho +- |m|)/2,
//   e = -(3/4) c (rho_up^(4/3) + rho_dn^(4/3)), c = (6/pi)^(1/3),
//   V_xc = (v_up + v_dn)/2, B_xc = (v_up - v_dn)/2 m/|m|, v_s = -c rho_s^(1/3).
// * gbc_anderson_mix: Anderson mixing of Sec. III.B.1, next input =
//   sum_j b_j ((1 - alpha) x_j + alpha f_j) with sum_j b_j = 1 and b minimising
//   || sum_j b_j (f_j - x_j) || in the inner product of Eq. innerPdt,
//   <(r1, m1), (r2, m2)> = (1/2)(int r1 r2 + int m1.m2) by Gauss quadrature:
//   b = G^-1 1 / (1^T G^-1 1), G_jk = <f_j - x_j, f_k - x_k>.
// Density arrays are [E][4][nq^3] doubles (rho, m_x, m_y, m_z per cell).
#include <cmath>
#include <vector>

#include "gbc_internal.h"

namespace {

constexpr int kMaxHist = 8;

__global__ void k_lsda_fields(const double* __restrict__ dens, const double* __restrict__ vext,
                              long long E, int nq3, double cx, double* __restrict__ raw,
                              double* __restrict__ eout) {
  const long long n = E * nq3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / nq3, q = i % nq3;
    const double* d = dens + e * 4 * nq3 + q;
    const double rho = d[0], mx = d[nq3], my = d[2 * nq3], mz = d[3 * nq3];
    const double am = sqrt(mx * mx + my * my + mz * mz);
    const double up = fmax(0.5 * (rho + am), 0.0), dn = fmax(0.5 * (rho - am), 0.0);
    const double cu = cbrt(up), cd = cbrt(dn);
    const double vu = -cx * cu, vd = -cx * cd;
    const double f = am > 0.0 ? 0.5 * (vu - vd) / am : 0.0;
    raw[i] = vext[i] + 0.5 * (vu + vd);
    raw[n + i] = f * mx;
    raw[2 * n + i] = f * my;
    raw[3 * n + i] = f * mz;
    if (eout) eout[i] = -0.75 * cx * (up * cu + dn * cd);
  }
}

struct Hist {
  const double* x[kMaxHist];
  const double* f[kMaxHist];
};
struct QW {
  double w[GBC_MAX_P + 2];   // 1-D Gauss weights
};

// G_jk += (1/2) sum_points w_q J r_j r_k over the 4 components, r_j = f_j - x_j
__global__ void k_residual_gram(Hist h, int nh, long long E, int nq, double jac, QW qw,
                                double* __restrict__ G) {
  const int nq3 = nq * nq * nq;
  const long long n = E * nq3;
  double acc[kMaxHist * (kMaxHist + 1) / 2];
#pragma unroll
  for (int t = 0; t < kMaxHist * (kMaxHist + 1) / 2; ++t) acc[t] = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / nq3;
    const int q = (int)(i % nq3);
    const double w = 0.5 * jac * qw.w[q % nq] * qw.w[(q / nq) % nq] * qw.w[q / (nq * nq)];
    for (int c = 0; c < 4; ++c) {
      const long long o = (e * 4 + c) * nq3 + q;
      double r[kMaxHist];
#pragma unroll
      for (int j = 0; j < kMaxHist; ++j) r[j] = j < nh ? h.f[j][o] - h.x[j][o] : 0.0;
      int t = 0;
#pragma unroll
      for (int j = 0; j < kMaxHist; ++j)
#pragma unroll
        for (int k = 0; k <= j; ++k, ++t) acc[t] += w * r[j] * r[k];
    }
  }
  // block reduction: warp shuffles, then one lane per warp into shared memory
  __shared__ double red[32][kMaxHist * (kMaxHist + 1) / 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kMaxHist * (kMaxHist + 1) / 2; ++t) {
    double v = acc[t];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][t] = v;
  }
  __syncthreads();
  if (threadIdx.x < kMaxHist * (kMaxHist + 1) / 2) {
    double v = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) v += red[wi][threadIdx.x];
    atomicAdd(&G[threadIdx.x], v);
  }
}

struct Coef {
  double b[kMaxHist];
};

__global__ void k_mix(Hist h, int nh, Coef cf, double alpha, long long n,
                      double* __restrict__ xnext) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int j = 0; j < nh; ++j) v += cf.b[j] * ((1.0 - alpha) * h.x[j][i] + alpha * h.f[j][i]);
    xnext[i] = v;
  }
}

unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)std::min<long long>(std::max<long long>(b, 1), 8LL * gbc_sm_count());
}

}  // namespace

extern "C" {

gbc_status gbc_scf_fields(gbc_ctx* c, const double* dens, const double* vext, double* exc,
                          void* stream) {
  if (!c) return GBC_EINVAL;
  if (!dens || !vext) return gbc_fail(c, GBC_EINVAL, "null argument");
  if (!c->mesh_set) return gbc_fail(c, GBC_ESTATE, "gbc_set_mesh first");
  if (!gbc_is_device_ptr(dens) || !gbc_is_device_ptr(vext) || (exc && !gbc_is_device_ptr(exc)))
    return gbc_fail(c, GBC_EINVAL, "dens, vext and exc must be device memory");
  GBC_CU(c, cudaSetDevice(c->dev));
  const long long nq3 = (long long)c->nq * c->nq * c->nq;
  const long long n = (long long)c->mesh.E * nq3;
  if (!c->d_rawfields) GBC_CU(c, cudaMalloc(&c->d_rawfields, sizeof(double) * 4 * n));
  cudaStream_t s = (cudaStream_t)stream;
  k_lsda_fields<<<grid_for(n), 256, 0, s>>>(dens, vext, c->mesh.E, (int)nq3,
                                            std::cbrt(6.0 / M_PI), c->d_rawfields, exc);
  GBC_CU(c, cudaGetLastError());
  // the fields are rebuilt by the next hot-path call on the library's own stream
  GBC_CU(c, cudaStreamSynchronize(s));
  c->fields_set = true;
  c->fields_dirty = true;
  return GBC_OK;
}

gbc_status gbc_anderson_mix(gbc_ctx* c, const double* const* xin, const double* const* xout,
                            int nhist, double alpha, double* xnext, double* coeffs,
                            double* resnorm, void* stream) {
  if (!c) return GBC_EINVAL;
  if (!xin || !xout || !xnext) return gbc_fail(c, GBC_EINVAL, "null argument");
  if (!gbc_is_device_ptr(xnext)) return gbc_fail(c, GBC_EINVAL, "xnext must be device memory");
  if (nhist < 1 || nhist > kMaxHist) return gbc_fail(c, GBC_EINVAL, "need 1 <= nhist <= 8");
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return gbc_fail(c, GBC_EINVAL, "alpha > 0 required");
  if (!c->mesh_set) return gbc_fail(c, GBC_ESTATE, "gbc_set_mesh first");
  Hist h{};
  for (int j = 0; j < nhist; ++j) {
    if (!gbc_is_device_ptr(xin[j]) || !gbc_is_device_ptr(xout[j]))
      return gbc_fail(c, GBC_EINVAL, "history entries must be device memory");
    h.x[j] = xin[j];
    h.f[j] = xout[j];
  }
  GBC_CU(c, cudaSetDevice(c->dev));
  cudaStream_t s = (cudaStream_t)stream;
  const int nq = c->nq;
  const long long n = (long long)c->mesh.E * nq * nq * nq;
  constexpr int NT = kMaxHist * (kMaxHist + 1) / 2;
  GBC_TRY(gbc_ensure_small(c, sizeof(double) * NT));   // small dense scratch
  double* dG = (double*)c->d_small;
  GBC_CU(c, cudaMemsetAsync(dG, 0, sizeof(double) * NT, s));
  QW qw{};
  for (int q = 0; q < nq; ++q) qw.w[q] = c->tab.gq_w[q];
  const double jac = c->h[0] * c->h[1] * c->h[2] / 8.0;
  k_residual_gram<<<grid_for(n), 256, 0, s>>>(h, nhist, c->mesh.E, nq, jac, qw, dG);
  GBC_CU(c, cudaGetLastError());
  double Gp[NT];
  GBC_CU(c, cudaMemcpyAsync(Gp, dG, sizeof(Gp), cudaMemcpyDeviceToHost, s));
  GBC_CU(c, cudaStreamSynchronize(s));
  // solve G y = 1 (Gaussian elimination, partial pivoting), b = y / sum(y)
  std::vector<double> A((size_t)nhist * nhist), y(nhist, 1.0);
  for (int j = 0, t = 0; j < kMaxHist; ++j)
    for (int k = 0; k <= j; ++k, ++t)
      if (j < nhist) A[(size_t)j * nhist + k] = A[(size_t)k * nhist + j] = Gp[t];
  const double gmax = [&] {
    double m = 0.0;
    for (int j = 0; j < nhist; ++j) m = std::fmax(m, A[(size_t)j * nhist + j]);
    return m;
  }();
  if (resnorm) *resnorm = std::sqrt(std::fmax(A[(size_t)(nhist - 1) * nhist + nhist - 1], 0.0));
  for (int col = 0; col < nhist; ++col) {
    int piv = col;
    for (int r = col + 1; r < nhist; ++r)
      if (std::fabs(A[(size_t)r * nhist + col]) > std::fabs(A[(size_t)piv * nhist + col])) piv = r;
    if (!(std::fabs(A[(size_t)piv * nhist + col]) > 1e-14 * gmax))
      return gbc_fail(c, GBC_ENOTPD, "residual Gram matrix is singular (repeated residuals?)");
    if (piv != col) {
      for (int k = 0; k < nhist; ++k) std::swap(A[(size_t)col * nhist + k], A[(size_t)piv * nhist + k]);
      std::swap(y[col], y[piv]);
    }
    for (int r = col + 1; r < nhist; ++r) {
      const double f = A[(size_t)r * nhist + col] / A[(size_t)col * nhist + col];
      for (int k = col; k < nhist; ++k) A[(size_t)r * nhist + k] -= f * A[(size_t)col * nhist + k];
      y[r] -= f * y[col];
    }
  }
  for (int r = nhist - 1; r >= 0; --r) {
    double v = y[r];
    for (int k = r + 1; k < nhist; ++k) v -= A[(size_t)r * nhist + k] * y[k];
    y[r] = v / A[(size_t)r * nhist + r];
  }
  double ysum = 0.0;
  for (int j = 0; j < nhist; ++j) ysum += y[j];
  if (!(std::fabs(ysum) > 0.0) || !std::isfinite(ysum))
    return gbc_fail(c, GBC_ENOTPD, "Anderson coefficients undefined");
  Coef cf{};
  for (int j = 0; j < nhist; ++j) {
    cf.b[j] = y[j] / ysum;
    if (coeffs) coeffs[j] = cf.b[j];
  }
  k_mix<<<grid_for(4 * n), 256, 0, s>>>(h, nhist, cf, alpha, 4 * n, xnext);
  GBC_CU(c, cudaGetLastError());
  GBC_CU(c, cudaStreamSynchronize(s));
  return GBC_OK;
}

}  // extern "C"
