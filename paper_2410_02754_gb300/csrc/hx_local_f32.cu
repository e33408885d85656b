// FP32 instantiations of the matrix-free cell-level apply (p = 2..7, nq = p + 2).
#include "hx_local.cuh"

cudaError_t launch_hx_local_f32(const gbc_ctx* c, const float2* X, float2* Y, int nvec, int ldx,
                                cudaStream_t s) {
  switch (c->mesh.p) {
    case 2: return gbc::launch_hx_local_p<float, 3, 2>(c, X, Y, nvec, ldx, s);
    case 3: return gbc::launch_hx_local_p<float, 4, 2>(c, X, Y, nvec, ldx, s);
    case 4: return gbc::launch_hx_local_p<float, 5, 2>(c, X, Y, nvec, ldx, s);
    case 5: return gbc::launch_hx_local_p<float, 6, 2>(c, X, Y, nvec, ldx, s);
    case 6: return gbc::launch_hx_local_p<float, 7, 2>(c, X, Y, nvec, ldx, s);
    case 7: return gbc::launch_hx_local_p<float, 8, 2>(c, X, Y, nvec, ldx, s);
    default: return cudaErrorInvalidValue;
  }
}
