// FP32 cell apply over systems of several orders in one persistent launch (the
// batched filter): 2 vectors x 256 threads per CTA, registers for 3 CTAs per SM,
// paired FP32 multiply-adds, every order p = 2..7 with and without k-terms.
#include "hx_cell.cuh"

cudaError_t launch_cell_multi_f32(const CellJob* jobs, int n, cudaStream_t s) {
  return gbc::launch_cell_multi<2, 256, 3, true>(jobs, n, s);
}
