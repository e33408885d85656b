// FP64 instantiations of the matrix-free cell apply (p = 2..7, nq = p + 2, one vector per CTA).
#include "hx_local.cuh"

cudaError_t launch_hx_local_group_f64(const HxJob* jobs, int n, int /*vb*/, cudaStream_t s) {
  return gbc::launch_hx_group<double, 1>(jobs, n, s);
}

GBC_CHECK_WORD_ACCESSOR(gbc_check_word_hx64)
