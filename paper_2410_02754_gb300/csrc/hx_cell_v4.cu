// FP32 cell apply, variant 4: 4 vectors per CTA, 512 threads, registers sized
// for 2 CTAs per SM, scalar FP32 multiply-adds (p = 2..7, nq = p + 2).  The
// stages over n_p^2 pencils fill 12.25 of 16 warps (6.125 of 8 with 2 vectors)
// and the gather reads 32 contiguous bytes per node row and spin.
#include "hx_cell.cuh"

cudaError_t launch_cell_f32_v4(const CellJob* jobs, int n, cudaStream_t s) {
  return gbc::launch_cell_group<4, 512, 2, false>(jobs, n, s);
}

GBC_CHECK_WORD_ACCESSOR(gbc_check_word_cell4)
