// C-ABI entry points of libgbchfsi (declared in include/gbchfsi.h).
//
// Host control logic only: argument checks, lazy (re)build of the operator
// tables, workspace management and the order of kernel launches.  Every
// arithmetic step of the hot path runs in the CUDA kernels of this library.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "gbc_internal.h"

// ---------------------------------------------------------------------------
// errors and workspaces
// ---------------------------------------------------------------------------
gbc_status gbc_fail(gbc_ctx* c, gbc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

gbc_status gbc_cuda_fail(gbc_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
                  ") in " + where;
  return gbc_fail(c, e == cudaErrorMemoryAllocation ? GBC_ENOMEM : GBC_ECUDA, m);
}

int gbc_sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < 64 && cache[dev] > 0) return cache[dev];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  if (dev < 64) cache[dev] = n;
  return n;
}

bool gbc_is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();   // clear the sticky-free error of an unknown pointer
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

gbc_status gbc_ensure_work(gbc_ctx* c, int slot, size_t bytes) {
  if (c->work_bytes[slot] >= bytes) return GBC_OK;
  if (c->work[slot]) cudaFree(c->work[slot]);
  c->work[slot] = nullptr;
  c->work_bytes[slot] = 0;
  GBC_CU(c, cudaMalloc(&c->work[slot], bytes));
  c->work_bytes[slot] = bytes;
  return GBC_OK;
}

gbc_status gbc_ensure_small(gbc_ctx* c, size_t bytes) {
  if (c->small_bytes >= bytes) return GBC_OK;
  if (c->d_small) cudaFree(c->d_small);
  c->d_small = nullptr;
  c->small_bytes = 0;
  GBC_CU(c, cudaMalloc(&c->d_small, bytes));
  c->small_bytes = bytes;
  return GBC_OK;
}

gbc_status gbc_prepare(gbc_ctx* c) {
  if (!c->mesh_set) return gbc_fail(c, GBC_ESTATE, "gbc_set_mesh has not been called");
  if (!c->fields_set) return gbc_fail(c, GBC_ESTATE, "gbc_set_fields has not been called");
  GBC_CU(c, cudaSetDevice(c->dev));
  if (c->fields_dirty) {
    GBC_TRY(setup_fields(c));
    c->fields_dirty = false;
  }
  if (c->proj_dirty) {
    GBC_TRY(setup_projectors(c));
    c->proj_dirty = false;
  }
  return GBC_OK;
}

static cudaEvent_t pool_event(gbc_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

TimerScope::TimerScope(gbc_ctx* c_, int fam_, cudaStream_t s_) : c(c_), fam(fam_), s(s_) {
  if (!c->timing) return;
  a = pool_event(c);
  b = pool_event(c);
  if (a) cudaEventRecord(a, s);
}

TimerScope::~TimerScope() {
  if (!c->timing || !a || !b) return;
  cudaEventRecord(b, s);
  c->timed.push_back({fam, a, b});
}

namespace {

gbc_status check_block(gbc_ctx* c, const void* X, int nvec, int ldx) {
  if (!X) return gbc_fail(c, GBC_EINVAL, "null block pointer");
  if (nvec < 0 || ldx < 1 || nvec > ldx) return gbc_fail(c, GBC_EINVAL, "need 0 <= nvec <= ldx, ldx >= 1");
  return GBC_OK;
}

// Y = H X in the context precision (Y zeroed first)
template <typename T>
gbc_status apply_h_t(gbc_ctx* c, const cplx<T>* X, cplx<T>* Y, int nvec, int ldx, cudaStream_t s,
                     bool zero = true) {
  if (zero) GBC_CU(c, cudaMemsetAsync(Y, 0, sizeof(cplx<T>) * 2 * (size_t)c->mesh.M * ldx, s));
  if (nvec == 0) return GBC_OK;
  cudaError_t e;
  {
    TimerScope ts(c, FAM_HX_LOCAL, s);
    if (std::is_same<T, double>::value && c->deterministic) {
      // per-cell results, then every node's cell contributions added in a fixed order
      const long long np = c->mesh.p + 1;
      GBC_TRY(gbc_ensure_work(c, 10, sizeof(double2) * (size_t)c->mesh.E * np * np * np * 2 * nvec));
      e = launch_hx_local_f64(c, (const double2*)X, (double2*)Y, nvec, ldx, s, c->work[10]);
      if (e == cudaSuccess)
        e = launch_cell_gather_f64(c, (const double2*)c->work[10], (double2*)Y, nvec, ldx, s);
    } else if (std::is_same<T, double>::value) {
      e = launch_hx_local_f64(c, (const double2*)X, (double2*)Y, nvec, ldx, s);
    } else if (c->prec == GBC_TF32 || c->prec == GBC_BF16X3) {
      GBC_TRY(tcl_apply(c, (const float2*)X, (float2*)Y, nvec, ldx, c->prec == GBC_BF16X3 ? 1 : 0, s));
      e = cudaSuccess;
    } else {
      e = launch_hx_local_f32(c, (const float2*)X, (float2*)Y, nvec, ldx, s);
    }
  }
  if (e != cudaSuccess) return gbc_cuda_fail(c, e, "hx_local");
  if (c->proj.natoms > 0) {
    const size_t cb = sizeof(cplx<T>) * (size_t)c->proj.rows_total * nvec;
    GBC_TRY(gbc_ensure_work(c, 2, 2 * cb));
    cplx<T>* C1 = (cplx<T>*)c->work[2];
    cplx<T>* C2 = C1 + (size_t)c->proj.rows_total * nvec;
    {
      TimerScope ts(c, FAM_NONLOCAL, s);
      e = launch_nonlocal<T>(c, X, Y, nvec, ldx, C1, C2, s);
    }
    if (e != cudaSuccess) return gbc_cuda_fail(c, e, "nonlocal");
  }
  return GBC_OK;
}

// X <- p_m(H~) X in place, the sigma-scaled three-term recurrence of Eq. chebfilt.
// FP64: the H.X accumulation (cell apply, nonlocal step) then one recurrence
// pass over every row.  FP32: the recurrence is fused into the applies -- the
// nonlocal step writes P C' into the accumulator's support rows, the cell apply
// finishes the rows interior to a cell in its epilogue, and a row pass finishes
// the rows on cell faces (see hx_cell.cuh).
template <typename T>
gbc_status filter_t(gbc_ctx* c, cplx<T>* X, int nvec, int ldx, int m, double lT, double lmax,
                    double lmin, cudaStream_t s) {
  const double cc = 0.5 * (lmax + lT), e = 0.5 * (lmax - lT);
  std::vector<double> sig(m);
  sig[0] = e / (lmin - cc);
  for (int k = 1; k < m; ++k) sig[k] = 1.0 / (2.0 / sig[0] - sig[k - 1]);
  const size_t bytes = sizeof(cplx<T>) * 2 * (size_t)c->mesh.M * ldx;
  GBC_TRY(gbc_ensure_work(c, 0, bytes));
  GBC_TRY(gbc_ensure_work(c, 1, bytes));
  cplx<T>* Y = (cplx<T>*)c->work[0];
  cplx<T>* W = (cplx<T>*)c->work[1];
  const T* invmd = std::is_same<T, double>::value ? (const T*)c->d_invmd : (const T*)c->d_invmd32;
  GBC_CU(c, cudaMemsetAsync(Y, 0, bytes, s));
  // step k: X_{k+1} = a_k (M_D^-1 H X_k - c X_k) - b_k X_{k-1}; X_1 -> W, then
  // X_{k+1} written over X_{k-1}
  for (int k = 0; k < m; ++k) {
    cplx<T>* cur = k == 0 ? X : ((k & 1) ? W : X);
    cplx<T>* prev = k == 0 ? nullptr : ((k & 1) ? X : W);
    cplx<T>* out = k == 0 ? W : prev;
    const double a = k == 0 ? sig[0] / e : 2.0 * sig[k] / e;
    const double b = k == 0 ? 0.0 : sig[k - 1] * sig[k];
    if (std::is_same<T, double>::value || nvec == 0 || c->prec != GBC_FP32) {
      GBC_TRY(apply_h_t<T>(c, cur, Y, nvec, ldx, s, false));
      TimerScope ts(c, FAM_CHEB, s);
      GBC_CU(c, launch_cheb_step<T>(Y, cur, prev, out, invmd, c->mesh.M, nvec, ldx, a, cc, b, s));
      continue;
    }
    if (c->proj.natoms > 0) {
      size_t xoff = 0;
      GBC_TRY(gbc_ensure_work(c, 2, nl_work_bytes(c, nvec, ldx, sizeof(cplx<T>), &xoff)));
      cplx<T>* C1 = (cplx<T>*)c->work[2];
      cplx<T>* C2 = C1 + (size_t)c->proj.rows_total * nvec;
      void* bpre = xoff ? (char*)c->work[2] + xoff : nullptr;
      TimerScope ts(c, FAM_NONLOCAL, s);
      GBC_CU(c, launch_nonlocal<T>(c, cur, Y, nvec, ldx, C1, C2, s, true, bpre));
    }
    {
      TimerScope ts(c, FAM_HX_LOCAL, s);
      CellJob j{c, cur, Y, nvec, ldx, out, prev, a, cc, b};
      GBC_CU(c, launch_cell_f32(&j, 1, c->cell_var, s));
    }
    TimerScope ts(c, FAM_CHEB, s);
    GBC_CU(c, launch_cheb_rows<T>(Y, cur, prev, out, invmd, c->d_face_rows, c->nface,
                                  c->proj.natoms > 0 ? c->nface_supp : 0, c->mesh.M, nvec, ldx,
                                  a, cc, b, s));
  }
  if (m & 1) GBC_CU(c, launch_copy_block<T>(W, X, c->mesh.M, nvec, ldx, s));
  return GBC_OK;
}

template <typename T>
gbc_status cholgs_t(gbc_ctx* c, cplx<T>* X, int nvec, int ldx, cudaStream_t s) {
  const size_t nn = (size_t)nvec * nvec;
  GBC_TRY(gbc_ensure_work(c, 3, sizeof(double2) * 2 * nn + sizeof(double) * nvec + 256));
  double2* S = (double2*)c->work[3];
  double2* Q = S + nn;
  {
    TimerScope ts(c, FAM_GRAM, s);
    GBC_CU(c, launch_gram<T>(X, X, c->d_md, c->mesh.M, nvec, ldx, S, s));
  }
  GBC_CU(c, launch_hermitize(S, nvec, s));
  {
    TimerScope ts(c, FAM_DENSE, s);
    GBC_TRY(dense_cholesky_inv_h(c, S, nvec, Q, s));
  }
  const size_t bytes = sizeof(cplx<T>) * 2 * (size_t)c->mesh.M * ldx;
  GBC_TRY(gbc_ensure_work(c, 1, bytes));
  cplx<T>* W = (cplx<T>*)c->work[1];
  {
    TimerScope ts(c, FAM_ROTATE, s);
    GBC_CU(c, launch_rotate<T>(X, Q, W, c->mesh.M, nvec, ldx, s));
  }
  GBC_CU(c, launch_copy_block<T>(W, X, c->mesh.M, nvec, ldx, s));
  GBC_CU(c, cudaStreamSynchronize(s));
  return GBC_OK;
}

template <typename T>
gbc_status rr_t(gbc_ctx* c, cplx<T>* X, int nvec, int ldx, double* ritz, cudaStream_t s) {
  const size_t nn = (size_t)nvec * nvec;
  const size_t bytes = sizeof(cplx<T>) * 2 * (size_t)c->mesh.M * ldx;
  GBC_TRY(gbc_ensure_work(c, 0, bytes));
  GBC_TRY(gbc_ensure_work(c, 1, bytes));
  GBC_TRY(gbc_ensure_work(c, 3, sizeof(double2) * 2 * nn + sizeof(double) * nvec + 256));
  double2* Hp = (double2*)c->work[3];
  double2* Q = Hp + nn;
  double* ev = (double*)(Q + nn);
  cplx<T>* HX = (cplx<T>*)c->work[0];
  GBC_TRY(apply_h_t<T>(c, X, HX, nvec, ldx, s));
  {
    TimerScope ts(c, FAM_GRAM, s);
    GBC_CU(c, launch_gram<T>(X, HX, nullptr, c->mesh.M, nvec, ldx, Hp, s));
  }
  GBC_CU(c, launch_hermitize(Hp, nvec, s));
  {
    TimerScope ts(c, FAM_DENSE, s);
    GBC_TRY(dense_eigh(c, Hp, nvec, ev, Q, s));
  }
  cplx<T>* W = (cplx<T>*)c->work[1];
  {
    TimerScope ts(c, FAM_ROTATE, s);
    GBC_CU(c, launch_rotate<T>(X, Q, W, c->mesh.M, nvec, ldx, s));
  }
  GBC_CU(c, launch_copy_block<T>(W, X, c->mesh.M, nvec, ldx, s));
  GBC_CU(c, cudaMemcpyAsync(ritz, ev, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s));
  GBC_CU(c, cudaStreamSynchronize(s));
  return GBC_OK;
}

// Residual-split filter (Hamiltonian-times-residual form of the recurrence):
// with H^ = (H~ - c)/e, Lambda^ = (Lambda - c)/e, R = H^ X - X Lambda^ and
// D_k = T_k(Lambda^)/T_k(tau),  X_m = X D_m + Z_m,  Z_1 = sigma_1 R,
// Z_{k+1} = 2 sigma_{k+1} H^ Z_k - sigma_k sigma_{k+1} Z_{k-1} + 2 sigma_{k+1} R D_k.
// R is formed from an FP64 H.X of an FP64 copy of X; only the Z recurrence runs
// in the context precision.  Work slots: 0 accumulator, 4 FP64 copy of X,
// 5 FP64 H.X, 6 R, 7 / 1 the two Z buffers, 3 the per-column coefficient tables.
template <typename T>
gbc_status filter_split_t(gbc_ctx* c, cplx<T>* X, int nvec, int ldx, int m, double lT,
                          double lmax, double lmin, const double* ritz, cudaStream_t s) {
  const double cc = 0.5 * (lmax + lT), e = 0.5 * (lmax - lT);
  std::vector<double> sig(m);
  sig[0] = e / (lmin - cc);
  for (int k = 1; k < m; ++k) sig[k] = 1.0 / (2.0 / sig[0] - sig[k - 1]);
  // per-column tables: lam_hat, g_k = 2 sigma_{k+1} D_k (k = 1..m-1), D_m
  std::vector<double> lam(nvec), tab((size_t)(m + 1) * nvec, 0.0);
  for (int v = 0; v < nvec; ++v) {
    lam[v] = (ritz[v] - cc) / e;
    double Dp = 1.0, Dc = sig[0] * lam[v];
    for (int k = 1; k < m; ++k) {
      tab[(size_t)(k - 1) * nvec + v] = 2.0 * sig[k] * Dc;
      const double Dn = 2.0 * sig[k] * lam[v] * Dc - sig[k - 1] * sig[k] * Dp;
      Dp = Dc;
      Dc = Dn;
    }
    tab[(size_t)m * nvec + v] = Dc;
    tab[(size_t)(m - 1) * nvec + v] = lam[v];
  }
  const size_t b64 = sizeof(double2) * 2 * (size_t)c->mesh.M * nvec;
  const size_t bT = sizeof(cplx<T>) * 2 * (size_t)c->mesh.M * ldx;
  GBC_TRY(gbc_ensure_work(c, 0, std::max(b64, bT)));
  GBC_TRY(gbc_ensure_work(c, 4, b64));
  GBC_TRY(gbc_ensure_work(c, 5, b64));
  GBC_TRY(gbc_ensure_work(c, 6, bT));
  GBC_TRY(gbc_ensure_work(c, 7, bT));
  GBC_TRY(gbc_ensure_work(c, 1, bT));
  GBC_TRY(gbc_ensure_work(c, 3, sizeof(double) * tab.size() + 256));
  double* dtab = (double*)c->work[3];
  GBC_CU(c, cudaMemcpyAsync(dtab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, s));
  const double* d_lam = dtab + (size_t)(m - 1) * nvec;
  const double* d_Dm = dtab + (size_t)m * nvec;
  double2* X64 = (double2*)c->work[4];
  double2* HX64 = (double2*)c->work[5];
  cplx<T>* R = (cplx<T>*)c->work[6];
  cplx<T>* Za = (cplx<T>*)c->work[7];
  cplx<T>* Zb = (cplx<T>*)c->work[1];
  cplx<T>* Y = (cplx<T>*)c->work[0];
  // R and Z_1 from the FP64 operator
  if (std::is_same<T, double>::value)
    GBC_CU(c, launch_copy_block<double>((const double2*)X, X64, c->mesh.M, nvec, nvec, s));
  else
    GBC_CU(c, launch_convert_block((const float2*)X, ldx, X64, nvec, c->mesh.M, nvec, s));
  GBC_TRY(apply_h_t<double>(c, X64, HX64, nvec, nvec, s));
  GBC_CU(c, launch_split_init<T>(HX64, X64, c->d_invmd, d_lam, R, Za, c->mesh.M, nvec, ldx, nvec,
                                 cc, 1.0 / e, sig[0], s));
  // Z_0 = 0 lives in Zb
  GBC_CU(c, cudaMemsetAsync(Zb, 0, bT, s));
  GBC_CU(c, cudaMemsetAsync(Y, 0, bT, s));
  const T* invmd = std::is_same<T, double>::value ? (const T*)c->d_invmd : (const T*)c->d_invmd32;
  // Z_1 in Za, Z_0 in Zb; Z_{k+1} overwrites Z_{k-1}
  for (int k = 1; k < m; ++k) {
    cplx<T>* cur = (k & 1) ? Za : Zb;
    cplx<T>* prev = (k & 1) ? Zb : Za;
    GBC_TRY(apply_h_t<T>(c, cur, Y, nvec, ldx, s, false));
    TimerScope ts(c, FAM_CHEB, s);
    GBC_CU(c, launch_split_step<T>(Y, cur, prev, prev, R, invmd, dtab + (size_t)(k - 1) * nvec,
                                   c->mesh.M, nvec, ldx, 2.0 * sig[k] / e, cc,
                                   sig[k - 1] * sig[k], s));
  }
  cplx<T>* Zm = (m & 1) ? Za : Zb;
  GBC_CU(c, launch_split_final<T>(X, Zm, d_Dm, c->mesh.M, nvec, ldx, s));
  return GBC_OK;
}

// The mixed path keeps complex64 blocks for the filter but runs CholGS and
// CholGS and Rayleigh-Ritz of an FP32 block.  The projected matrices are FP64-
// accurate: S = X^H M_D X and Hp = X^H (H X) are accumulated in float-float
// arithmetic on the FP32 pipes; Rayleigh-Ritz needs an FP64 H.X (an FP32 one
// would put a first-order error eps32 * ||H~|| into X^H H X and hence into the
// Ritz values), computed on an FP64 copy of X (work slot 4).  The rotations
// X <- X Q act on the FP32 block in float-float arithmetic as well: the FP64
// product rounded to FP32.
gbc_status rotate_mixed(gbc_ctx* c, float2* X, int nvec, int ldx, const double2* Q, float2* Qsplit,
                        cudaStream_t s) {
  const size_t bytes = sizeof(float2) * 2 * (size_t)c->mesh.M * ldx;
  GBC_TRY(gbc_ensure_work(c, 1, bytes));
  float2* W = (float2*)c->work[1];
  {
    TimerScope ts(c, FAM_ROTATE, s);
    GBC_CU(c, launch_rotate_ff(X, Q, Qsplit, W, c->mesh.M, nvec, ldx, s));
  }
  GBC_CU(c, launch_copy_block<float>(W, X, c->mesh.M, nvec, ldx, s));
  return GBC_OK;
}

gbc_status cholgs_mixed(gbc_ctx* c, float2* X, int nvec, int ldx, cudaStream_t s) {
  const size_t nn = (size_t)nvec * nvec;
  GBC_TRY(gbc_ensure_work(c, 3, sizeof(double2) * 3 * nn + sizeof(double) * nvec + 256));
  double2* S = (double2*)c->work[3];
  double2* Q = S + nn;
  float2* Qsplit = (float2*)(Q + nn);   // 2 nn float2
  {
    TimerScope ts(c, FAM_GRAM, s);
    GBC_CU(c, launch_gram_ff<float>(X, ldx, X, ldx, c->d_md, c->mesh.M, nvec, S, s));
  }
  GBC_CU(c, launch_hermitize(S, nvec, s));
  {
    TimerScope ts(c, FAM_DENSE, s);
    GBC_TRY(dense_cholesky_inv_h(c, S, nvec, Q, s));
  }
  GBC_TRY(rotate_mixed(c, X, nvec, ldx, Q, Qsplit, s));
  GBC_CU(c, cudaStreamSynchronize(s));
  return GBC_OK;
}

gbc_status rr_mixed(gbc_ctx* c, float2* X, int nvec, int ldx, double* ritz, cudaStream_t s) {
  const size_t nn = (size_t)nvec * nvec;
  const size_t bytes64 = sizeof(double2) * 2 * (size_t)c->mesh.M * nvec;
  GBC_TRY(gbc_ensure_work(c, 4, bytes64));
  GBC_TRY(gbc_ensure_work(c, 0, bytes64));
  GBC_TRY(gbc_ensure_work(c, 3, sizeof(double2) * 3 * nn + sizeof(double) * nvec + 256));
  double2* X64 = (double2*)c->work[4];
  double2* HX = (double2*)c->work[0];
  double2* Hp = (double2*)c->work[3];
  double2* Q = Hp + nn;
  float2* Qsplit = (float2*)(Q + nn);
  double* ev = (double*)(Q + 2 * nn);
  GBC_CU(c, launch_convert_block(X, ldx, X64, nvec, c->mesh.M, nvec, s));
  GBC_TRY(apply_h_t<double>(c, X64, HX, nvec, nvec, s));
  {
    TimerScope ts(c, FAM_GRAM, s);
    GBC_CU(c, launch_gram_ff<double>(X, ldx, HX, nvec, nullptr, c->mesh.M, nvec, Hp, s));
  }
  GBC_CU(c, launch_hermitize(Hp, nvec, s));
  {
    TimerScope ts(c, FAM_DENSE, s);
    GBC_TRY(dense_eigh(c, Hp, nvec, ev, Q, s));
  }
  GBC_TRY(rotate_mixed(c, X, nvec, ldx, Q, Qsplit, s));
  GBC_CU(c, cudaMemcpyAsync(ritz, ev, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s));
  GBC_CU(c, cudaStreamSynchronize(s));
  return GBC_OK;
}

}  // namespace

// H.X in the context precision for the other translation units (Y zeroed
// first when ``zero``)
gbc_status gbc_apply_h_dev(gbc_ctx* c, const void* X, void* Y, int nvec, int ldx, bool zero,
                           cudaStream_t s) {
  if (c->prec == GBC_FP64)
    return apply_h_t<double>(c, (const double2*)X, (double2*)Y, nvec, ldx, s, zero);
  return apply_h_t<float>(c, (const float2*)X, (float2*)Y, nvec, ldx, s, zero);
}

// ---------------------------------------------------------------------------
// public API
// ---------------------------------------------------------------------------
// one guarded store for gbc_check_selftest
namespace {
__device__ int g_check_selftest_buf[64];
__global__ void k_check_selftest(long long i) {
  if (GBC_IN_RANGE(GBC_SITE_SELFTEST, i, 64)) g_check_selftest_buf[i] = 1;
}
}  // namespace

extern "C" {

const char* gbc_version(void) { return "gbchfsi 0.1 (sm_103a)"; }

gbc_status gbc_create(gbc_ctx** out, int device_ordinal) {
  if (!out) return GBC_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device_ordinal < 0 || device_ordinal >= n)
    return GBC_EINVAL;
  gbc_ctx* c = new (std::nothrow) gbc_ctx();
  if (!c) return GBC_ENOMEM;
  c->dev = device_ordinal;
  if (cudaSetDevice(device_ordinal) != cudaSuccess || cudaMalloc(&c->d_flag, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->d_cell_ctr, sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(c->d_flag);
    delete c;
    return GBC_ECUDA;
  }
  *out = c;
  return GBC_OK;
}

void gbc_destroy(gbc_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  cudaDeviceSynchronize();
  free_projectors(c->proj);
  tcl_free(c->tcl);
  for (auto& t : c->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  void* ptrs[] = {c->d_md, c->d_invmd, c->d_invmd32, c->d_rawfields, c->d_fields64, c->d_fields32,
                  c->d_small, c->d_flag, c->d_face_rows, c->d_cell_ctr};
  for (void* p : ptrs) cudaFree(p);
  for (void* p : c->work) cudaFree(p);
  delete c;
}

const char* gbc_last_error(const gbc_ctx* c) { return c ? c->err.c_str() : "null context"; }

gbc_status gbc_set_mesh(gbc_ctx* c, const int ncell[3], const double h[3], int p, int nq,
                        const int periodic[3]) {
  if (!c) return GBC_EINVAL;
  if (!ncell || !h || !periodic) return gbc_fail(c, GBC_EINVAL, "null argument");
  if (p < 2 || p > GBC_MAX_P) return gbc_fail(c, GBC_EUNSUPPORTED, "p must be in [2, 7]");
  if (nq != p + 2) return gbc_fail(c, GBC_EUNSUPPORTED, "this build requires nq == p + 2");
  for (int d = 0; d < 3; ++d) {
    if (ncell[d] < 1 || !(h[d] > 0)) return gbc_fail(c, GBC_EINVAL, "ncell >= 1 and h > 0 required");
    if (!periodic[d] && ncell[d] * p < 2) return gbc_fail(c, GBC_EINVAL, "no free nodes");
  }
  GBC_CU(c, cudaSetDevice(c->dev));
  MeshDev m{};
  long long M = 1, E = 1;
  for (int d = 0; d < 3; ++d) {
    m.ncell[d] = ncell[d];
    m.period[d] = ncell[d] * p;
    m.periodic[d] = periodic[d] ? 1 : 0;
    m.nfree[d] = periodic[d] ? ncell[d] * p : ncell[d] * p - 1;
    M *= m.nfree[d];
    E *= ncell[d];
    c->h[d] = h[d];
  }
  if (E > 0x7fffffffLL / 64) return gbc_fail(c, GBC_EINVAL, "too many cells");
  m.p = p;
  m.E = (int)E;
  m.M = M;
  c->mesh = m;
  c->nq = nq;
  c->k[0] = c->k[1] = c->k[2] = 0.0;
  free_projectors(c->proj);
  cudaFree(c->d_rawfields);
  cudaFree(c->d_fields64);
  cudaFree(c->d_fields32);
  c->d_rawfields = nullptr;
  c->d_fields64 = nullptr;
  c->d_fields32 = nullptr;
  c->fields_set = false;
  c->fields_dirty = true;
  c->proj_dirty = false;
  GBC_TRY(setup_tables(c));
  GBC_TRY(setup_mass(c));
  GBC_TRY(setup_face_rows(c));
  c->mesh_set = true;
  return GBC_OK;
}

gbc_status gbc_set_kpoint(gbc_ctx* c, const double k[3]) {
  if (!c) return GBC_EINVAL;
  if (!k) return gbc_fail(c, GBC_EINVAL, "null k");
  if (!c->mesh_set) return gbc_fail(c, GBC_ESTATE, "gbc_set_mesh first");
  for (int d = 0; d < 3; ++d) {
    if (!std::isfinite(k[d])) return gbc_fail(c, GBC_EINVAL, "non-finite k");
    c->k[d] = k[d];
  }
  c->fields_dirty = true;
  if (c->proj.natoms > 0) c->proj_dirty = true;
  return GBC_OK;
}

gbc_status gbc_set_fields(gbc_ctx* c, const double* veff, const double* bx, const double* by,
                          const double* bz) {
  if (!c) return GBC_EINVAL;
  if (!veff || !bx || !by || !bz) return gbc_fail(c, GBC_EINVAL, "null field");
  if (!c->mesh_set) return gbc_fail(c, GBC_ESTATE, "gbc_set_mesh first");
  GBC_CU(c, cudaSetDevice(c->dev));
  const size_t n = (size_t)c->mesh.E * c->nq * c->nq * c->nq;
  if (!c->d_rawfields) GBC_CU(c, cudaMalloc(&c->d_rawfields, sizeof(double) * 4 * n));
  const double* src[4] = {veff, bx, by, bz};
  for (int i = 0; i < 4; ++i)
    GBC_CU(c, cudaMemcpy(c->d_rawfields + i * n, src[i], sizeof(double) * n, cudaMemcpyHostToDevice));
  c->fields_set = true;
  c->fields_dirty = true;
  return GBC_OK;
}

gbc_status gbc_set_projectors(gbc_ctx* c, int natoms, const int* npj, const int* nsupp,
                              const int* supp_cell, const int* supp_img, const double* pvals,
                              const double* delta) {
  if (!c) return GBC_EINVAL;
  if (!c->mesh_set) return gbc_fail(c, GBC_ESTATE, "gbc_set_mesh first");
  if (natoms < 0) return gbc_fail(c, GBC_EINVAL, "natoms < 0");
  GBC_CU(c, cudaSetDevice(c->dev));
  GBC_CU(c, cudaDeviceSynchronize());
  free_projectors(c->proj);
  c->proj_dirty = false;
  if (natoms == 0) return GBC_OK;
  if (!npj || !nsupp || !supp_cell || !supp_img || !pvals || !delta)
    return gbc_fail(c, GBC_EINVAL, "null projector argument");
  for (int a = 0; a < natoms; ++a) {
    if (npj[a] < 1 || npj[a] > GBC_MAX_NPJ) return gbc_fail(c, GBC_EUNSUPPORTED, "npj must be in [1, 32]");
    if (nsupp[a] < 0) return gbc_fail(c, GBC_EINVAL, "nsupp < 0");
  }
  GBC_TRY(build_projector_structure(c, natoms, npj, nsupp, supp_cell, supp_img, pvals, delta));
  c->proj_dirty = true;
  return GBC_OK;
}

gbc_status gbc_set_precision(gbc_ctx* c, gbc_precision prec) {
  if (!c) return GBC_EINVAL;
  if (prec != GBC_FP64 && prec != GBC_FP32 && prec != GBC_TF32 && prec != GBC_BF16X3)
    return gbc_fail(c, GBC_EUNSUPPORTED, "unknown precision");
  c->prec = prec;
  return GBC_OK;
}

gbc_status gbc_set_deterministic(gbc_ctx* c, int on) {
  if (!c) return GBC_EINVAL;
  if (c->deterministic != (on != 0) && c->proj.natoms > 0) c->proj_dirty = true;   // P rebuilt
  c->deterministic = on != 0;
  return GBC_OK;
}

gbc_status gbc_get_deterministic(const gbc_ctx* c, int* on) {
  if (!c || !on) return GBC_EINVAL;
  *on = c->deterministic ? 1 : 0;
  return GBC_OK;
}

gbc_status gbc_set_nonlocal_engine(gbc_ctx* c, int engine) {
  if (!c) return GBC_EINVAL;
  if (engine != GBC_NL_SIMT && engine != GBC_NL_TENSOR)
    return gbc_fail(c, GBC_EINVAL, "unknown nonlocal engine");
  c->nl_engine = engine;
  return GBC_OK;
}

gbc_status gbc_get_nonlocal_engine(const gbc_ctx* c, int* engine) {
  if (!c || !engine) return GBC_EINVAL;
  *engine = (c->nl_engine == GBC_NL_TENSOR && tc_nonlocal_supported(c->proj)) ? GBC_NL_TENSOR
                                                                               : GBC_NL_SIMT;
  return GBC_OK;
}

gbc_status gbc_sync_status(gbc_ctx* c, void* stream) {
  if (!c) return GBC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int err = 0;
  GBC_CU(c, tc_nonlocal_error(&err, s));
  int err2 = 0;
  GBC_CU(c, tcl_error(&err2, s));
  err |= err2;
  if (err) {
    GBC_CU(c, tc_nonlocal_reset(s));
    GBC_CU(c, cudaStreamSynchronize(s));
    return gbc_fail(c, GBC_ETIMEOUT, "a tensor-core wait expired; results since the last check are invalid");
  }
  // checked build: the first index out of range of every translation unit (all read,
  // so all are cleared)
  using Reader = cudaError_t (*)(unsigned long long*, cudaStream_t);
  static const Reader readers[] = {gbc_check_word_cell0, gbc_check_word_cell1, gbc_check_word_cell2,
                                   gbc_check_word_cell3, gbc_check_word_cell4, gbc_check_word_hx64,
                                   gbc_check_word_blas,  gbc_check_word_nl,    gbc_check_word_nltc,
                                   gbc_check_word_api};
  unsigned long long first = 0;
  for (Reader rd : readers) {
    unsigned long long w = 0;
    GBC_CU(c, rd(&w, s));
    if (w && !first) first = w;
  }
  if (first) {
    static const char* site[] = {"?", "FP32 cell apply (gather)", "FP32 cell apply (assembly)",
                                 "face-row recurrence", "nonlocal support node", "nonlocal P table",
                                 "FP64 cell apply", "self-test"};
    const int st = (int)(first >> 48);
    const long long idx = (long long)(first & 0xFFFFFFFFFFFFULL);
    return gbc_fail(c, GBC_ECHECK, std::string("checked build: index ") + std::to_string(idx) +
                                       " out of range at site " + std::to_string(st) + " (" +
                                       site[(st >= 1 && st <= 7) ? st : 0] +
                                       "); the access was skipped, results are invalid");
  }
  return GBC_OK;
}

gbc_status gbc_build_info(int* checked) {
  if (!checked) return GBC_EINVAL;
  *checked = GBC_CHECKED_BUILD;
  return GBC_OK;
}

gbc_status gbc_check_selftest(long long index, void* stream) {
  if (!GBC_CHECKED_BUILD && (index < 0 || index >= 64)) return GBC_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  k_check_selftest<<<1, 1, 0, s>>>(index);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return GBC_ECUDA;
  return GBC_OK;
}

gbc_status gbc_get_nnodes(const gbc_ctx* c, long long* nnodes) {
  if (!c || !nnodes) return GBC_EINVAL;
  if (!c->mesh_set) return GBC_ESTATE;
  *nnodes = c->mesh.M;
  return GBC_OK;
}

gbc_status gbc_get_ndof(const gbc_ctx* c, long long* nnodes) { return gbc_get_nnodes(c, nnodes); }

gbc_status gbc_get_mass(gbc_ctx* c, double* md) {
  if (!c) return GBC_EINVAL;
  if (!md) return gbc_fail(c, GBC_EINVAL, "null output");
  if (!c->mesh_set) return gbc_fail(c, GBC_ESTATE, "gbc_set_mesh first");
  GBC_CU(c, cudaSetDevice(c->dev));
  GBC_CU(c, cudaMemcpy(md, c->d_md, sizeof(double) * c->mesh.M, cudaMemcpyDeviceToHost));
  return GBC_OK;
}

gbc_status gbc_apply_h(gbc_ctx* c, const void* X, void* Y, int nvec, int ldx, void* stream) {
  if (!c) return GBC_EINVAL;
  GBC_TRY(check_block(c, X, nvec, ldx));
  GBC_TRY(check_block(c, Y, nvec, ldx));
  if (X == Y) return gbc_fail(c, GBC_EINVAL, "X and Y must be distinct");
  GBC_TRY(gbc_prepare(c));
  cudaStream_t s = (cudaStream_t)stream;
  if (c->prec == GBC_FP64) return apply_h_t<double>(c, (const double2*)X, (double2*)Y, nvec, ldx, s);
  return apply_h_t<float>(c, (const float2*)X, (float2*)Y, nvec, ldx, s);
}

gbc_status gbc_filter(gbc_ctx* c, void* X, int nvec, int ldx, int degree, double lT, double lmax,
                      double lmin, void* stream) {
  if (!c) return GBC_EINVAL;
  GBC_TRY(check_block(c, X, nvec, ldx));
  if (degree < 1) return gbc_fail(c, GBC_EINVAL, "degree >= 1 required");
  if (!(lmin < lT && lT < lmax)) return gbc_fail(c, GBC_EINVAL, "need lmin < lT < lmax");
  GBC_TRY(gbc_prepare(c));
  cudaStream_t s = (cudaStream_t)stream;
  if (nvec == 0) return GBC_OK;
  if (c->prec == GBC_FP64) return filter_t<double>(c, (double2*)X, nvec, ldx, degree, lT, lmax, lmin, s);
  return filter_t<float>(c, (float2*)X, nvec, ldx, degree, lT, lmax, lmin, s);
}

gbc_status gbc_filter_residual(gbc_ctx* c, void* X, int nvec, int ldx, int degree, double lT,
                               double lmax, double lmin, const double* ritz, void* stream) {
  if (!c) return GBC_EINVAL;
  GBC_TRY(check_block(c, X, nvec, ldx));
  if (!ritz) return gbc_fail(c, GBC_EINVAL, "null ritz");
  if (degree < 1) return gbc_fail(c, GBC_EINVAL, "degree >= 1 required");
  if (!(lmin < lT && lT < lmax)) return gbc_fail(c, GBC_EINVAL, "need lmin < lT < lmax");
  GBC_TRY(gbc_prepare(c));
  cudaStream_t s = (cudaStream_t)stream;
  if (nvec == 0) return GBC_OK;
  if (c->prec == GBC_FP64)
    return filter_split_t<double>(c, (double2*)X, nvec, ldx, degree, lT, lmax, lmin, ritz, s);
  return filter_split_t<float>(c, (float2*)X, nvec, ldx, degree, lT, lmax, lmin, ritz, s);
}

gbc_status gbc_cholgs(gbc_ctx* c, void* X, int nvec, int ldx, void* stream) {
  if (!c) return GBC_EINVAL;
  GBC_TRY(check_block(c, X, nvec, ldx));
  if (nvec < 1 || nvec > 512) return gbc_fail(c, GBC_EINVAL, "nvec must be in [1, 512]");
  GBC_TRY(gbc_prepare(c));
  cudaStream_t s = (cudaStream_t)stream;
  if (c->prec == GBC_FP64) return cholgs_t<double>(c, (double2*)X, nvec, ldx, s);
  return cholgs_mixed(c, (float2*)X, nvec, ldx, s);
}

gbc_status gbc_rayleigh_ritz(gbc_ctx* c, void* X, int nvec, int ldx, double* ritz, void* stream) {
  if (!c) return GBC_EINVAL;
  GBC_TRY(check_block(c, X, nvec, ldx));
  if (!ritz) return gbc_fail(c, GBC_EINVAL, "null ritz");
  if (nvec < 1 || nvec > 512) return gbc_fail(c, GBC_EINVAL, "nvec must be in [1, 512]");
  GBC_TRY(gbc_prepare(c));
  cudaStream_t s = (cudaStream_t)stream;
  if (c->prec == GBC_FP64) return rr_t<double>(c, (double2*)X, nvec, ldx, ritz, s);
  return rr_mixed(c, (float2*)X, nvec, ldx, ritz, s);
}

gbc_status gbc_lanczos_bounds(gbc_ctx* c, const void* v0, int steps, double* lmin, double* lmax,
                              void* stream) {
  if (!c) return GBC_EINVAL;
  if (!v0 || !lmin || !lmax) return gbc_fail(c, GBC_EINVAL, "null argument");
  if (steps < 1 || steps > 64) return gbc_fail(c, GBC_EINVAL, "steps must be in [1, 64]");
  GBC_TRY(gbc_prepare(c));
  cudaStream_t s = (cudaStream_t)stream;
  const long long M = c->mesh.M;
  const size_t vb = sizeof(double2) * 2 * (size_t)M;
  // work slot 0: w ; slot 1: the Krylov basis (steps + 1 vectors)
  GBC_TRY(gbc_ensure_work(c, 0, vb));
  GBC_TRY(gbc_ensure_work(c, 1, vb * (steps + 1)));
  const int kmax = steps;
  GBC_TRY(gbc_ensure_work(c, 3, sizeof(double2) * (2 * (size_t)kmax * kmax + 8 * kmax + 64) +
                                    sizeof(double) * kmax));
  double2* w = (double2*)c->work[0];
  double2* V = (double2*)c->work[1];
  double2* T = (double2*)c->work[3];                 // kmax x kmax tridiagonal (complex storage)
  double2* Qt = T + (size_t)kmax * kmax;
  double2* coef = Qt + (size_t)kmax * kmax;         // scratch inner products
  double* ev = (double*)(coef + 8 * kmax + 64);
  const long long n2 = 2 * M;
  // v_1 = v0 / ||v0||_M
  double2 h;
  double2* part = nullptr;   // deterministic mode: block sums added in order
  if (c->deterministic) {
    GBC_TRY(gbc_ensure_work(c, 12, mdot_part_bytes(M)));
    part = (double2*)c->work[12];
  }
  GBC_CU(c, launch_mdot((const double2*)v0, (const double2*)v0, c->d_md, M, coef, s, part));
  GBC_CU(c, cudaMemcpyAsync(&h, coef, sizeof(double2), cudaMemcpyDeviceToHost, s));
  GBC_CU(c, cudaStreamSynchronize(s));
  if (!(h.x > 0)) return gbc_fail(c, GBC_EINVAL, "zero start vector");
  GBC_CU(c, launch_scale_c(V, (const double2*)v0, 1.0 / std::sqrt(h.x), n2, s));
  std::vector<double> alpha(kmax), beta(kmax);
  for (int j = 0; j < kmax; ++j) {
    double2* vj = V + (size_t)j * n2;
    // w = M_D^-1 H v_j
    GBC_TRY(apply_h_t<double>(c, vj, w, 1, 1, s));
    GBC_CU(c, launch_divmass(w, c->d_invmd, M, s));
    // alpha_j = <v_j, w>_M ; w -= alpha v_j + beta_{j-1} v_{j-1}; two passes of full
    // reorthogonalisation against v_0..v_j
    GBC_CU(c, launch_mdot(vj, w, c->d_md, M, coef, s, part));
    GBC_CU(c, cudaMemcpyAsync(&h, coef, sizeof(double2), cudaMemcpyDeviceToHost, s));
    GBC_CU(c, cudaStreamSynchronize(s));
    alpha[j] = h.x;
    GBC_CU(c, launch_axpy_c(w, vj, coef, 1.0, n2, s));
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = 0; i <= j; ++i) {
        double2* vi = V + (size_t)i * n2;
        GBC_CU(c, launch_mdot(vi, w, c->d_md, M, coef + 1 + i, s, part));
        GBC_CU(c, launch_axpy_c(w, vi, coef + 1 + i, 1.0, n2, s));
      }
    }
    GBC_CU(c, launch_mdot(w, w, c->d_md, M, coef, s, part));
    GBC_CU(c, cudaMemcpyAsync(&h, coef, sizeof(double2), cudaMemcpyDeviceToHost, s));
    GBC_CU(c, cudaStreamSynchronize(s));
    beta[j] = std::sqrt(std::max(h.x, 0.0));
    if (j + 1 <= kmax) {
      const double inv = beta[j] > 0 ? 1.0 / beta[j] : 0.0;
      GBC_CU(c, launch_scale_c(V + (size_t)(j + 1) * n2, w, inv, n2, s));
    }
  }
  // eigenvalues of the tridiagonal T_k on the device
  std::vector<double2> Th((size_t)kmax * kmax, make_double2(0, 0));
  for (int j = 0; j < kmax; ++j) {
    Th[(size_t)j * kmax + j] = make_double2(alpha[j], 0);
    if (j + 1 < kmax) {
      Th[(size_t)j * kmax + j + 1] = make_double2(beta[j], 0);
      Th[(size_t)(j + 1) * kmax + j] = make_double2(beta[j], 0);
    }
  }
  GBC_CU(c, cudaMemcpyAsync(T, Th.data(), sizeof(double2) * Th.size(), cudaMemcpyHostToDevice, s));
  GBC_TRY(dense_eigh(c, T, kmax, ev, Qt, s));
  std::vector<double> evh(kmax);
  GBC_CU(c, cudaMemcpyAsync(evh.data(), ev, sizeof(double) * kmax, cudaMemcpyDeviceToHost, s));
  GBC_CU(c, cudaStreamSynchronize(s));
  *lmin = evh[0];
  *lmax = evh[kmax - 1] + std::fabs(beta[kmax - 1]);
  return GBC_OK;
}

gbc_status gbc_set_timing(gbc_ctx* c, int enable) {
  if (!c) return GBC_EINVAL;
  GBC_CU(c, cudaSetDevice(c->dev));
  GBC_CU(c, cudaDeviceSynchronize());
  for (auto& t : c->timed) {
    c->event_pool.push_back(t.a);
    c->event_pool.push_back(t.b);
  }
  c->timed.clear();
  c->timing = enable != 0;
  return GBC_OK;
}

gbc_status gbc_get_timing(gbc_ctx* c, int family, double* total_ms, long long* launches) {
  if (!c) return GBC_EINVAL;
  if (family < 0 || family >= FAM_COUNT || !total_ms || !launches)
    return gbc_fail(c, GBC_EINVAL, "bad timing query");
  GBC_CU(c, cudaSetDevice(c->dev));
  double tot = 0;
  long long n = 0;
  for (auto& t : c->timed) {
    if (t.family != family) continue;
    GBC_CU(c, cudaEventSynchronize(t.b));
    float ms = 0;
    GBC_CU(c, cudaEventElapsedTime(&ms, t.a, t.b));
    tot += ms;
    ++n;
  }
  *total_ms = tot;
  *launches = n;
  return GBC_OK;
}

}  // extern "C"

GBC_CHECK_WORD_ACCESSOR(gbc_check_word_api)
