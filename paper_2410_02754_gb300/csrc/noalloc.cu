// gbc_apply_h_noalloc: the H.X entry point for callers that must not let the
// library allocate device memory.
//
// Some host applications own every byte of device memory themselves (a
// framework's caching allocator, a fixed pool sized at start-up) or must never
// trigger the implicit device-wide synchronisation that cudaMalloc / cudaFree
// can cause in the middle of their own pipelined work.  gbc_apply_h may grow
// a library workspace (the per-atom projection coefficients C = P^H X and
// C' = Delta C) with cudaMalloc on first use; this variant keeps that scratch
// in one fixed, file-scope device array instead and allocates nothing.
//
// The array holds GBC_NOALLOC_SCRATCH_BYTES bytes and lives on every GPU that
// loads this library until the process exits.  All calls share it and it
// keeps the previous call's contents (the kernels clear what must start at
// zero); calls that overlap on the GPU -- on different streams or from
// different threads -- race on it, so callers must order them.
#include <mutex>

#include "gbc_internal.h"

#define GBC_NOALLOC_SCRATCH_BYTES (32u << 20)   // 32 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[GBC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on device ``dev`` (which must be
// current).  In host code the array's name is only a host-side stand-in, so the
// address is looked up once per device with cudaGetSymbolAddress.
cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

template <typename T>
gbc_status apply_noalloc(gbc_ctx* c, const cplx<T>* X, cplx<T>* Y, int nvec, int ldx,
                         cudaStream_t s) {
  const size_t cb = sizeof(cplx<T>) * (size_t)c->proj.rows_total * nvec;
  if (2 * cb > GBC_NOALLOC_SCRATCH_BYTES)
    return gbc_fail(c, GBC_EINVAL,
                    "gbc_apply_h_noalloc: 2 * (sum over atoms of 2*npj) * nvec * sizeof(complex) = " +
                        std::to_string(2 * cb) + " bytes exceeds the fixed scratch of " +
                        std::to_string((size_t)GBC_NOALLOC_SCRATCH_BYTES) + " bytes");
  void* base = nullptr;
  GBC_CU(c, scratch_address(c->dev, &base));
  GBC_CU(c, cudaMemsetAsync(Y, 0, sizeof(cplx<T>) * 2 * (size_t)c->mesh.M * ldx, s));
  if (nvec == 0) return GBC_OK;
  cudaError_t e = std::is_same<T, double>::value
                      ? launch_hx_local_f64(c, (const double2*)X, (double2*)Y, nvec, ldx, s)
                      : launch_hx_local_f32(c, (const float2*)X, (float2*)Y, nvec, ldx, s);
  if (e != cudaSuccess) return gbc_cuda_fail(c, e, "hx_local");
  if (c->proj.natoms > 0) {
    cplx<T>* C1 = (cplx<T>*)base;
    cplx<T>* C2 = C1 + (size_t)c->proj.rows_total * nvec;
    e = launch_nonlocal<T>(c, X, Y, nvec, ldx, C1, C2, s);
    if (e != cudaSuccess) return gbc_cuda_fail(c, e, "nonlocal");
  }
  return GBC_OK;
}

}  // namespace

extern "C" gbc_status gbc_apply_h_noalloc(gbc_ctx* c, const void* X, void* Y, int nvec, int ldx,
                                          void* stream) {
  if (!c) return GBC_EINVAL;
  if (!X || !Y) return gbc_fail(c, GBC_EINVAL, "null block pointer");
  if (X == Y) return gbc_fail(c, GBC_EINVAL, "X and Y must be distinct");
  if (!gbc_is_device_ptr(X) || !gbc_is_device_ptr(Y))
    return gbc_fail(c, GBC_EINVAL, "gbc_apply_h_noalloc: X and Y must be device memory");
  if (nvec < 0 || ldx < 1 || nvec > ldx) return gbc_fail(c, GBC_EINVAL, "need 0 <= nvec <= ldx, ldx >= 1");
  if (!c->mesh_set || !c->fields_set)
    return gbc_fail(c, GBC_ESTATE, "gbc_apply_h_noalloc: set mesh and fields first");
  if (c->fields_dirty || c->proj_dirty)
    return gbc_fail(c, GBC_ESTATE,
                    "gbc_apply_h_noalloc: operator tables not built for the current fields/k-point/"
                    "projectors; call gbc_apply_h (or another hot-path call) once first");
  if (c->prec == GBC_TF32 || c->prec == GBC_BF16X3)
    return gbc_fail(c, GBC_EUNSUPPORTED,
                    "gbc_apply_h_noalloc: the tensor-core cell apply needs library scratch");
  GBC_CU(c, cudaSetDevice(c->dev));
  cudaStream_t s = (cudaStream_t)stream;
  if (c->prec == GBC_FP64) return apply_noalloc<double>(c, (const double2*)X, (double2*)Y, nvec, ldx, s);
  return apply_noalloc<float>(c, (const float2*)X, (float2*)Y, nvec, ldx, s);
}
