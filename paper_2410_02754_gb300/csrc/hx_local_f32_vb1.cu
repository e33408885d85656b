// FP32 instantiations of the matrix-free cell apply, one vector per CTA
// (p = 2..7, nq = p + 2); the autotuner chooses between this tile and two
// vectors per CTA.
#include "hx_local.cuh"

cudaError_t launch_hx_local_group_f32_vb1(const HxJob* jobs, int n, cudaStream_t s) {
  return gbc::launch_hx_group<float, 1>(jobs, n, s);
}

cudaError_t launch_hx_local_group_f32(const HxJob* jobs, int n, int vb, cudaStream_t s) {
  return vb == 1 ? launch_hx_local_group_f32_vb1(jobs, n, s)
                 : launch_hx_local_group_f32_vb2(jobs, n, s);
}
