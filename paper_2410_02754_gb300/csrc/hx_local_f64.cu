// FP64 instantiations of the matrix-free cell apply (p = 2..7, nq = p + 2, one vector per CTA).
#include "hx_local.cuh"

cudaError_t launch_hx_local_group_f64(const HxJob* jobs, int n, int /*vb*/, cudaStream_t s) {
  return gbc::launch_hx_group<double, 1>(jobs, n, s);
}

cudaError_t launch_cell_gather_f64(const gbc_ctx* c, const double2* Ycell, double2* Y, int nvec,
                                   int ldx, cudaStream_t s) {
  const long long n = c->mesh.M * 2 * (long long)nvec;
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, 64LL * gbc_sm_count());
  gbc::k_cell_gather<double><<<grid, 256, 0, s>>>(Y, Ycell, c->mesh, nvec, ldx);
  return cudaGetLastError();
}

GBC_CHECK_WORD_ACCESSOR(gbc_check_word_hx64)
