// Instantiations of the quadrature-point gradient contraction (FP64: one vector
// per CTA, FP32: two).
#include "grad.cuh"

cudaError_t launch_quad_grad_f64(const gbc_ctx* c, const double2* A, const double2* B,
                                 const double* wv, double scale, int nvec, int ldx, double* g,
                                 int pointwise, cudaStream_t s) {
  return gbc::launch_quad_grad_t<double, 1>(c, A, B, wv, scale, nvec, ldx, g, pointwise, s);
}

cudaError_t launch_quad_grad_f32(const gbc_ctx* c, const float2* A, const float2* B,
                                 const double* wv, double scale, int nvec, int ldx, double* g,
                                 int pointwise, cudaStream_t s) {
  return gbc::launch_quad_grad_t<float, 2>(c, A, B, wv, scale, nvec, ldx, g, pointwise, s);
}
