// Backward pass of the scaled Chebyshev filter (vector-Jacobian product) and
// the gradients of the energy L = sum_i w_i y_i^H H y_i.
//
// Paper: Eq. chebfilt (the recurrence being differentiated), Eqs. FEHloc /
// FEHnloc (dH/dV_eff, dH/dB_xc at the Gauss points, dH/dDelta_a through the
// projector coefficients), Eqs. rho / mag (the bilinear densities that the
// quadrature-point gradients are).  With L = (M_D^-1 H - c)/e and the recurrence
// X_{k+1} = alpha_k L X_k - beta_k X_{k-1}, the adjoint Lt = M_D^-1 Lambda obeys
// the same recurrence backwards:
//   Lt_m = M_D^-1 G_Y,  Lt_k = alpha_k L Lt_{k+1} - beta_{k+1} Lt_{k+2},
//   grad_X0 = M_D Lt_0,
//   dL/dtheta = sum_k (alpha_k / e) Re(Lt_{k+1}^H (dH/dtheta) X_k),
// so the backward reuses the H.X and recurrence kernels.  X_k is checkpointed
// in pairs every ``ckpt_every`` degrees and recomputed segment by segment.
#include <algorithm>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "gbc_internal.h"

namespace {

inline unsigned gfor(long long n) {
  long long g = (n + 255) / 256;
  return (unsigned)std::max(1LL, std::min(g, 64LL * gbc_sm_count()));
}

// Out[row][v] = w[row / 2] * In[row][v]
template <typename T>
__global__ void k_rowscale(const cplx<T>* __restrict__ In, cplx<T>* __restrict__ Out,
                           const double* __restrict__ w, long long rows, int nvec, int ldx) {
  const long long n = rows * (long long)nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nvec;
    const int v = (int)(i - r * nvec);
    const T s = (T)w[r >> 1];
    const cplx<T> x = In[r * ldx + v];
    Out[r * ldx + v] = cmake<cplx<T>>(s * x.x, s * x.y);
  }
}

// G[row][v] = f * w[v] * G[row][v]
template <typename T>
__global__ void k_colscale(cplx<T>* G, const double* __restrict__ w, double f, long long rows,
                           int nvec, int ldx) {
  const long long n = rows * (long long)nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nvec;
    const int v = (int)(i - r * nvec);
    const T s = (T)(f * w[v]);
    cplx<T>& g = G[r * ldx + v];
    g.x *= s;
    g.y *= s;
  }
}

// dots[v] += sum_rows Re(conj(A[row][v]) B[row][v])  (FP64 accumulation); with part,
// block x's sum goes to part[x][v] instead (k_coldot_parts adds them in order)
template <typename T>
__global__ void k_coldot(const cplx<T>* __restrict__ A, const cplx<T>* __restrict__ B,
                         long long rows, int nvec, int ldx, double* dots, double* part) {
  const int v = blockIdx.y * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  double acc = 0.0;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const cplx<T> a = A[r * ldx + v], b = B[r * ldx + v];
    acc += (double)a.x * (double)b.x + (double)a.y * (double)b.y;
  }
  if (part) part[(size_t)blockIdx.x * nvec + v] = acc;
  else atomicAdd(&dots[v], acc);
}

// dots[v] += sum_b part[b][v], b = 0 .. nb-1 in order
__global__ void k_coldot_parts(const double* __restrict__ part, int nb, int nvec, double* dots) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  double acc = 0.0;
  for (int b = 0; b < nb; ++b) acc += part[(size_t)b * nvec + v];
  dots[v] += acc;
}

// gD[atom][r][s] += f * sum_v wv[v] Ca[r][v] conj(Cb[s][v])   (rows c_off + r)
template <typename T>
__global__ void k_delta_grad(const cplx<T>* __restrict__ Ca, const cplx<T>* __restrict__ Cb,
                             const double* __restrict__ wv, double f, int nvec,
                             const int* __restrict__ atom_npj, const int* __restrict__ atom_c_off,
                             const int* __restrict__ atom_delta_off, double2* gD) {
  const int atom = blockIdx.x, r = blockIdx.y, sidx = threadIdx.x;
  const int n2 = 2 * atom_npj[atom];
  if (r >= n2 || sidx >= n2) return;
  const size_t ra = (size_t)(atom_c_off[atom] + r) * nvec;
  const size_t rb = (size_t)(atom_c_off[atom] + sidx) * nvec;
  double re = 0, im = 0;
  for (int v = 0; v < nvec; ++v) {
    const double w = wv ? wv[v] : 1.0;
    const cplx<T> a = Ca[ra + v], b = Cb[rb + v];
    // a * conj(b)
    re += w * ((double)a.x * b.x + (double)a.y * b.y);
    im += w * ((double)a.y * b.x - (double)a.x * b.y);
  }
  double2* g = &gD[atom_delta_off[atom] + (size_t)r * n2 + sidx];
  g->x += f * re;
  g->y += f * im;
}

// per-atom Hermitian part of gD: (G + G^H) / 2
__global__ void k_delta_herm(double2* gD, const int* __restrict__ atom_npj,
                             const int* __restrict__ atom_delta_off) {
  const int atom = blockIdx.x, r = blockIdx.y, sidx = threadIdx.x;
  const int n2 = 2 * atom_npj[atom];
  if (r >= n2 || sidx >= n2 || sidx < r) return;
  double2* G = gD + atom_delta_off[atom];
  if (sidx == r) {
    G[(size_t)r * n2 + r].y = 0.0;
    return;
  }
  const double2 a = G[(size_t)r * n2 + sidx], b = G[(size_t)sidx * n2 + r];
  const double re = 0.5 * (a.x + b.x), im = 0.5 * (a.y - b.y);
  G[(size_t)r * n2 + sidx] = make_double2(re, im);
  G[(size_t)sidx * n2 + r] = make_double2(re, -im);
}

}  // namespace

namespace {

template <typename T>
cudaError_t quad_grad(const gbc_ctx* c, const cplx<T>* A, const cplx<T>* B, const double* wv,
                      double scale, int nvec, int ldx, double* g, cudaStream_t s,
                      int pointwise = 0) {
  if (std::is_same<T, double>::value)
    return launch_quad_grad_f64(c, (const double2*)A, (const double2*)B, wv, scale, nvec, ldx, g,
                                pointwise, s);
  return launch_quad_grad_f32(c, (const float2*)A, (const float2*)B, wv, scale, nvec, ldx, g,
                              pointwise, s);
}

// projector-coefficient outer products for the Delta gradient
template <typename T>
gbc_status delta_grad(gbc_ctx* c, const cplx<T>* A, const cplx<T>* B, const double* wv, double f,
                      int nvec, int ldx, cplx<T>* Ca, cplx<T>* Cb, double2* gD, cudaStream_t s) {
  const ProjDev& pj = c->proj;
  if (pj.natoms == 0) return GBC_OK;
  GBC_CU(c, launch_nl_project<T>(c, A, nvec, ldx, Ca, s));
  const cplx<T>* Cbp = Ca;
  if (B != A) {
    GBC_CU(c, launch_nl_project<T>(c, B, nvec, ldx, Cb, s));
    Cbp = Cb;
  }
  dim3 grid(pj.natoms, 2 * pj.max_npj);
  k_delta_grad<T><<<grid, 2 * pj.max_npj, 0, s>>>(Ca, Cbp, wv, f, nvec, pj.d_atom_npj,
                                                  pj.d_atom_c_off, pj.d_atom_delta_off, gD);
  GBC_CU(c, cudaGetLastError());
  return GBC_OK;
}

// device accumulators: g [E][4][nq^3] (FP64), gD (complex FP64), scratch for the
// projector coefficients, per-vector weights and column dots
struct GradScratch {
  double* g;
  double2* gD;
  void* Ca;
  void* Cb;
  double* wv;
  double* dots;
};

gbc_status grad_scratch(gbc_ctx* c, int nvec, GradScratch* gs) {
  const size_t nq3 = (size_t)c->nq * c->nq * c->nq;
  const size_t ng = (size_t)c->mesh.E * 4 * nq3;
  const size_t nd = c->proj.natoms ? (size_t)c->proj.delta_off[c->proj.natoms] : 0;
  const size_t el = c->prec == GBC_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t nc = std::max<size_t>(1, (size_t)c->proj.rows_total * nvec);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t bytes = up(ng * 8) + up(std::max<size_t>(nd, 1) * 16) + 2 * up(nc * el) +
                       2 * up((size_t)nvec * 8);
  GBC_TRY(gbc_ensure_work(c, 9, bytes));
  char* p = (char*)c->work[9];
  gs->g = (double*)p;
  p += up(ng * 8);
  gs->gD = (double2*)p;
  p += up(std::max<size_t>(nd, 1) * 16);
  gs->Ca = p;
  p += up(nc * el);
  gs->Cb = p;
  p += up(nc * el);
  gs->wv = (double*)p;
  p += up((size_t)nvec * 8);
  gs->dots = (double*)p;
  return GBC_OK;
}

// copy g [E][4][q] (device) to the host arrays g0 [E][q] and g13 [3][E][q]
// (either may be null).  Synchronous.
gbc_status download_quad(gbc_ctx* c, const double* g, double* g0, double* g13, cudaStream_t s) {
  const size_t nq3 = (size_t)c->nq * c->nq * c->nq;
  const size_t E = (size_t)c->mesh.E;
  std::vector<double> h(E * 4 * nq3);
  GBC_CU(c, cudaMemcpyAsync(h.data(), g, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  GBC_CU(c, cudaStreamSynchronize(s));
  for (size_t e = 0; e < E; ++e)
    for (int comp = 0; comp < 4; ++comp) {
      double* dst = comp == 0 ? g0 : (g13 ? g13 + (size_t)(comp - 1) * E * nq3 : nullptr);
      if (!dst) continue;
      std::copy(&h[(e * 4 + comp) * nq3], &h[(e * 4 + comp) * nq3] + nq3, dst + e * nq3);
    }
  return GBC_OK;
}

// copy g [E][4][q] to the four host arrays and the Hermitian-projected gD to host
gbc_status grad_download(gbc_ctx* c, const GradScratch& gs, double* gV, double* gB, double* gDelta,
                         cudaStream_t s) {
  const ProjDev& pj = c->proj;
  if (pj.natoms) {
    dim3 grid(pj.natoms, 2 * pj.max_npj);
    k_delta_herm<<<grid, 2 * pj.max_npj, 0, s>>>(gs.gD, pj.d_atom_npj, pj.d_atom_delta_off);
    GBC_CU(c, cudaGetLastError());
    if (gDelta)
      GBC_CU(c, cudaMemcpyAsync(gDelta, gs.gD, sizeof(double2) * pj.delta_off[pj.natoms],
                                cudaMemcpyDeviceToHost, s));
  }
  return download_quad(c, gs.g, gV, gB, s);
}

template <typename T>
gbc_status filter_vjp_t(gbc_ctx* c, const cplx<T>* X0, const cplx<T>* GY, cplx<T>* GX, double* gV,
                        double* gB, double* gDelta, int nvec, int ldx, int m, double lT,
                        double lmax, double lmin, int K, cudaStream_t s) {
  using C = cplx<T>;
  const double cc = 0.5 * (lmax + lT), e = 0.5 * (lmax - lT);
  std::vector<double> sig(m), alpha(m), beta(m + 1, 0.0);
  sig[0] = e / (lmin - cc);
  for (int k = 1; k < m; ++k) sig[k] = 1.0 / (2.0 / sig[0] - sig[k - 1]);
  alpha[0] = sig[0];
  for (int k = 1; k < m; ++k) {
    alpha[k] = 2.0 * sig[k];
    beta[k] = sig[k - 1] * sig[k];
  }
  // checkpoints: X_j for j % K in {0, 1}, j <= m - 1
  std::vector<int> ck_slot(m, -1);
  int nck = 0;
  for (int j = 0; j < m; ++j)
    if (j % K == 0 || j % K == 1) ck_slot[j] = nck++;
  const int nseg = std::max(K, 3);
  const size_t bb = sizeof(C) * 2 * (size_t)c->mesh.M * ldx;
  GBC_TRY(gbc_ensure_work(c, 8, bb * (size_t)(nck + nseg + 3)));
  GBC_TRY(gbc_ensure_work(c, 0, bb));
  char* pool = (char*)c->work[8];
  auto blk = [&](int i) { return (C*)(pool + bb * (size_t)i); };
  C* Y = (C*)c->work[0];
  auto lam = [&](int j) { return blk(nck + nseg + (j % 3)); };
  GradScratch gs;
  GBC_TRY(grad_scratch(c, nvec, &gs));
  const size_t nq3 = (size_t)c->nq * c->nq * c->nq;
  GBC_CU(c, cudaMemsetAsync(gs.g, 0, sizeof(double) * c->mesh.E * 4 * nq3, s));
  if (c->proj.natoms)
    GBC_CU(c, cudaMemsetAsync(gs.gD, 0, sizeof(double2) * c->proj.delta_off[c->proj.natoms], s));
  GBC_CU(c, cudaMemsetAsync(Y, 0, bb, s));
  const T* invmd = std::is_same<T, double>::value ? (const T*)c->d_invmd : (const T*)c->d_invmd32;
  const long long rows = 2 * c->mesh.M;
  // ---- forward, keeping the checkpoint pairs
  std::vector<C*> xp(m, nullptr);
  for (int j = 0; j < m; ++j) xp[j] = ck_slot[j] >= 0 ? blk(ck_slot[j]) : blk(nck + (j % 3));
  GBC_CU(c, launch_copy_block<T>(X0, xp[0], c->mesh.M, nvec, ldx, s));
  for (int k = 0; k + 1 < m; ++k) {
    GBC_TRY(gbc_apply_h_dev(c, xp[k], Y, nvec, ldx, false, s));
    GBC_CU(c, launch_cheb_step<T>(Y, xp[k], k ? xp[k - 1] : nullptr, xp[k + 1], invmd, c->mesh.M,
                                  nvec, ldx, alpha[k] / e, cc, beta[k], s));
  }
  // ---- adjoint seed Lt_m = M_D^-1 G_Y
  k_rowscale<T><<<gfor(rows * nvec), 256, 0, s>>>(GY, lam(m), c->d_invmd, rows, nvec, ldx);
  GBC_CU(c, cudaGetLastError());
  // ---- segments from the last to the first
  const int nsegs = (m + K - 1) / K;
  for (int sg = nsegs - 1; sg >= 0; --sg) {
    const int k0 = sg * K, k1 = std::min(m, k0 + K);
    std::vector<C*> seg(k1 - k0, nullptr);
    for (int j = k0; j < k1; ++j) seg[j - k0] = ck_slot[j] >= 0 ? blk(ck_slot[j]) : blk(nck + (j - k0));
    for (int k = k0 + 1; k + 1 < k1; ++k) {      // recompute X_{k+1} from X_k, X_{k-1}
      if (ck_slot[k + 1] >= 0) continue;
      GBC_TRY(gbc_apply_h_dev(c, seg[k - k0], Y, nvec, ldx, false, s));
      GBC_CU(c, launch_cheb_step<T>(Y, seg[k - k0], seg[k - 1 - k0], seg[k + 1 - k0], invmd,
                                    c->mesh.M, nvec, ldx, alpha[k] / e, cc, beta[k], s));
    }
    for (int k = k1 - 1; k >= k0; --k) {
      const double f = alpha[k] / e;
      C* Xk = seg[k - k0];
      C* Lt1 = lam(k + 1);
      GBC_CU(c, quad_grad<T>(c, Lt1, Xk, nullptr, f, nvec, ldx, gs.g, s));
      GBC_TRY(delta_grad<T>(c, Lt1, Xk, nullptr, f, nvec, ldx, (C*)gs.Ca, (C*)gs.Cb, gs.gD, s));
      GBC_TRY(gbc_apply_h_dev(c, Lt1, Y, nvec, ldx, false, s));
      const bool has2 = k + 2 <= m;
      GBC_CU(c, launch_cheb_step<T>(Y, Lt1, has2 ? lam(k + 2) : nullptr, lam(k), invmd, c->mesh.M,
                                    nvec, ldx, alpha[k] / e, cc, has2 ? beta[k + 1] : 0.0, s));
    }
  }
  // ---- grad_X0 = M_D Lt_0
  k_rowscale<T><<<gfor(rows * nvec), 256, 0, s>>>(lam(0), GX, c->d_md, rows, nvec, ldx);
  GBC_CU(c, cudaGetLastError());
  return grad_download(c, gs, gV, gB, gDelta, s);
}

template <typename T>
gbc_status energy_grad_t(gbc_ctx* c, const cplx<T>* Y, const double* w, cplx<T>* GY, double* loss,
                         double* gV, double* gB, double* gDelta, int nvec, int ldx, cudaStream_t s) {
  GradScratch gs;
  GBC_TRY(grad_scratch(c, nvec, &gs));
  const size_t nq3 = (size_t)c->nq * c->nq * c->nq;
  GBC_CU(c, cudaMemsetAsync(gs.g, 0, sizeof(double) * c->mesh.E * 4 * nq3, s));
  if (c->proj.natoms)
    GBC_CU(c, cudaMemsetAsync(gs.gD, 0, sizeof(double2) * c->proj.delta_off[c->proj.natoms], s));
  GBC_CU(c, cudaMemcpyAsync(gs.wv, w, sizeof(double) * nvec, cudaMemcpyHostToDevice, s));
  GBC_CU(c, cudaMemsetAsync(gs.dots, 0, sizeof(double) * nvec, s));
  const long long rows = 2 * c->mesh.M;
  // H Y -> GY, the loss from the column dots, then G_Y = 2 H Y diag(w)
  GBC_TRY(gbc_apply_h_dev(c, Y, GY, nvec, ldx, true, s));
  dim3 gd((unsigned)std::min<long long>(rows, 4096), (nvec + 127) / 128);
  double* part = nullptr;
  if (c->deterministic) {
    GBC_TRY(gbc_ensure_work(c, 12, sizeof(double) * gd.x * (size_t)nvec));
    part = (double*)c->work[12];
  }
  k_coldot<T><<<gd, 128, 0, s>>>(Y, GY, rows, nvec, ldx, gs.dots, part);
  GBC_CU(c, cudaGetLastError());
  if (part) {
    k_coldot_parts<<<(nvec + 127) / 128, 128, 0, s>>>(part, (int)gd.x, nvec, gs.dots);
    GBC_CU(c, cudaGetLastError());
  }
  k_colscale<T><<<gfor(rows * nvec), 256, 0, s>>>(GY, gs.wv, 2.0, rows, nvec, ldx);
  GBC_CU(c, cudaGetLastError());
  GBC_CU(c, quad_grad<T>(c, Y, Y, gs.wv, 1.0, nvec, ldx, gs.g, s));
  GBC_TRY(delta_grad<T>(c, Y, Y, gs.wv, 1.0, nvec, ldx, (cplx<T>*)gs.Ca, (cplx<T>*)gs.Cb, gs.gD, s));
  std::vector<double> dots(nvec);
  GBC_CU(c, cudaMemcpyAsync(dots.data(), gs.dots, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s));
  GBC_TRY(grad_download(c, gs, gV, gB, gDelta, s));
  double L = 0;
  for (int v = 0; v < nvec; ++v) L += w[v] * dots[v];
  if (loss) *loss = L;
  return GBC_OK;
}

// rho and m at the Gauss points (Eqs. rho, mag) into out [E][4][nq^3] (device)
template <typename T>
cudaError_t density_t(const gbc_ctx* c, const cplx<T>* X, const double* occ_dev, double* out,
                      int nvec, int ldx, int accumulate, cudaStream_t s) {
  return quad_grad<T>(c, X, X, occ_dev, 1.0, nvec, ldx, out, s, accumulate ? 2 : 1);
}

gbc_status density_check(gbc_ctx* c, const void* X, const double* occ, const double* out, int nvec,
                         int ldx) {
  if (!X || !occ || !out) return gbc_fail(c, GBC_EINVAL, "null argument");
  if (nvec < 1 || ldx < nvec) return gbc_fail(c, GBC_EINVAL, "need 1 <= nvec <= ldx");
  GBC_TRY(gbc_prepare(c));
  if (c->mesh.p > 6) return gbc_fail(c, GBC_EUNSUPPORTED, "densities support p <= 6");
  return GBC_OK;
}

}  // namespace

extern "C" {

gbc_status gbc_density_dev(gbc_ctx* c, const void* X, const double* occ, double* out, int nvec,
                           int ldx, int accumulate, void* stream) {
  if (!c) return GBC_EINVAL;
  GBC_TRY(density_check(c, X, occ, out, nvec, ldx));
  if (!gbc_is_device_ptr(X) || !gbc_is_device_ptr(occ) || !gbc_is_device_ptr(out))
    return gbc_fail(c, GBC_EINVAL, "X, occ and out must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->prec == GBC_FP64)
    GBC_CU(c, density_t<double>(c, (const double2*)X, occ, out, nvec, ldx, accumulate, s));
  else
    GBC_CU(c, density_t<float>(c, (const float2*)X, occ, out, nvec, ldx, accumulate, s));
  return GBC_OK;
}

gbc_status gbc_density(gbc_ctx* c, const void* X, const double* occ, double* rho, double* mag,
                       int nvec, int ldx, void* stream) {
  if (!c) return GBC_EINVAL;
  GBC_TRY(density_check(c, X, occ, rho, nvec, ldx));
  if (!gbc_is_device_ptr(X)) return gbc_fail(c, GBC_EINVAL, "X must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  GradScratch gs;
  GBC_TRY(grad_scratch(c, nvec, &gs));
  GBC_CU(c, cudaMemcpyAsync(gs.wv, occ, sizeof(double) * nvec, cudaMemcpyHostToDevice, s));
  if (c->prec == GBC_FP64)
    GBC_CU(c, density_t<double>(c, (const double2*)X, gs.wv, gs.g, nvec, ldx, 0, s));
  else
    GBC_CU(c, density_t<float>(c, (const float2*)X, gs.wv, gs.g, nvec, ldx, 0, s));
  return download_quad(c, gs.g, rho, mag, s);
}

gbc_status gbc_filter_vjp(gbc_ctx* c, const void* X0, const void* GY, void* GX, double* gV,
                          double* gB, double* gDelta, int nvec, int ldx, int degree, double lT,
                          double lmax, double lmin, int ckpt_every, void* stream) {
  if (!c) return GBC_EINVAL;
  if (!X0 || !GY || !GX) return gbc_fail(c, GBC_EINVAL, "null block pointer");
  if (nvec < 1 || ldx < nvec) return gbc_fail(c, GBC_EINVAL, "need 1 <= nvec <= ldx");
  if (degree < 1 || ckpt_every < 1) return gbc_fail(c, GBC_EINVAL, "degree, ckpt_every >= 1 required");
  if (!(lmin < lT && lT < lmax)) return gbc_fail(c, GBC_EINVAL, "need lmin < lT < lmax");
  GBC_TRY(gbc_prepare(c));
  if (c->mesh.p > 6) return gbc_fail(c, GBC_EUNSUPPORTED, "backward supports p <= 6");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->prec == GBC_FP64)
    return filter_vjp_t<double>(c, (const double2*)X0, (const double2*)GY, (double2*)GX, gV, gB,
                                gDelta, nvec, ldx, degree, lT, lmax, lmin, ckpt_every, s);
  return filter_vjp_t<float>(c, (const float2*)X0, (const float2*)GY, (float2*)GX, gV, gB, gDelta,
                             nvec, ldx, degree, lT, lmax, lmin, ckpt_every, s);
}

gbc_status gbc_filter_backward(gbc_ctx* c, const void* X0, const void* GY, void* GX, double* gV,
                               double* gB, double* gDelta, int nvec, int ldx, int degree,
                               double lT, double lmax, double lmin, int ckpt_every, void* stream) {
  return gbc_filter_vjp(c, X0, GY, GX, gV, gB, gDelta, nvec, ldx, degree, lT, lmax, lmin,
                        ckpt_every, stream);
}

gbc_status gbc_energy_grad(gbc_ctx* c, const void* Y, const double* w, void* GY, double* loss,
                           double* gV, double* gB, double* gDelta, int nvec, int ldx,
                           void* stream) {
  if (!c) return GBC_EINVAL;
  if (!Y || !GY || !w) return gbc_fail(c, GBC_EINVAL, "null argument");
  if (Y == GY) return gbc_fail(c, GBC_EINVAL, "Y and GY must be distinct");
  if (nvec < 1 || ldx < nvec) return gbc_fail(c, GBC_EINVAL, "need 1 <= nvec <= ldx");
  GBC_TRY(gbc_prepare(c));
  if (c->mesh.p > 6) return gbc_fail(c, GBC_EUNSUPPORTED, "gradients support p <= 6");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->prec == GBC_FP64)
    return energy_grad_t<double>(c, (const double2*)Y, w, (double2*)GY, loss, gV, gB, gDelta, nvec,
                                 ldx, s);
  return energy_grad_t<float>(c, (const float2*)Y, w, (float2*)GY, loss, gV, gB, gDelta, nvec, ldx,
                              s);
}

gbc_status gbc_set_delta(gbc_ctx* c, const double* delta) {
  if (!c) return GBC_EINVAL;
  if (!delta) return gbc_fail(c, GBC_EINVAL, "null delta");
  const ProjDev& pj = c->proj;
  if (pj.natoms == 0) return gbc_fail(c, GBC_ESTATE, "no projectors set");
  GBC_CU(c, cudaSetDevice(c->dev));
  const size_t n = pj.delta_off[pj.natoms];
  std::vector<float2> d32(n);
  for (size_t i = 0; i < n; ++i) d32[i] = make_float2((float)delta[2 * i], (float)delta[2 * i + 1]);
  GBC_CU(c, cudaDeviceSynchronize());
  GBC_CU(c, cudaMemcpy(pj.d_delta64, delta, sizeof(double2) * n, cudaMemcpyHostToDevice));
  GBC_CU(c, cudaMemcpy(pj.d_delta32, d32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
  return GBC_OK;
}

}  // extern "C"
