// FP64 instantiations of the matrix-free cell-level apply (p = 2..7, nq = p + 2).
#include "hx_local.cuh"

cudaError_t launch_hx_local_f64(const gbc_ctx* c, const double2* X, double2* Y, int nvec, int ldx,
                                cudaStream_t s) {
  switch (c->mesh.p) {
    case 2: return gbc::launch_hx_local_p<double, 3, 1>(c, X, Y, nvec, ldx, s);
    case 3: return gbc::launch_hx_local_p<double, 4, 1>(c, X, Y, nvec, ldx, s);
    case 4: return gbc::launch_hx_local_p<double, 5, 1>(c, X, Y, nvec, ldx, s);
    case 5: return gbc::launch_hx_local_p<double, 6, 1>(c, X, Y, nvec, ldx, s);
    case 6: return gbc::launch_hx_local_p<double, 7, 1>(c, X, Y, nvec, ldx, s);
    case 7: return gbc::launch_hx_local_p<double, 8, 1>(c, X, Y, nvec, ldx, s);
    default: return cudaErrorInvalidValue;
  }
}
