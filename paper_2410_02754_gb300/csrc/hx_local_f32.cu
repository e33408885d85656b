// FP32 instantiations of the matrix-free cell apply, two vectors per CTA
// (p = 2..7, nq = p + 2).
#include "hx_local.cuh"

cudaError_t launch_hx_local_group_f32_vb2(const HxJob* jobs, int n, cudaStream_t s) {
  return gbc::launch_hx_group<float, 2>(jobs, n, s);
}
