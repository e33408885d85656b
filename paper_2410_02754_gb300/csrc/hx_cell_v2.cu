// FP32 cell apply, variant 2: 2 vectors per CTA, 256 threads, registers sized
// for 4 CTAs per SM, scalar FP32 multiply-adds (p = 2..7, nq = p + 2).
#include "hx_cell.cuh"

cudaError_t launch_cell_f32_v2(const CellJob* jobs, int n, cudaStream_t s) {
  return gbc::launch_cell_group<2, 256, 4, false>(jobs, n, s);
}

GBC_CHECK_WORD_ACCESSOR(gbc_check_word_cell2)
