// Dispatch of the FP32 cell apply over its compiled variants (chosen per
// context by the autotuner, gbc_tune).
#include "gbc_internal.h"

cudaError_t launch_cell_f32_v0(const CellJob* jobs, int n, cudaStream_t s);
cudaError_t launch_cell_f32_v1(const CellJob* jobs, int n, cudaStream_t s);
cudaError_t launch_cell_f32_v2(const CellJob* jobs, int n, cudaStream_t s);
cudaError_t launch_cell_f32_v3(const CellJob* jobs, int n, cudaStream_t s);
cudaError_t launch_cell_f32_v4(const CellJob* jobs, int n, cudaStream_t s);


CellVariant cell_variant(int v) {
  static const CellVariant tab[GBC_CELL_VARIANTS] = {{2, 256, 4, 1}, {2, 256, 3, 1},
                                                     {2, 256, 4, 0}, {2, 256, 3, 0},
                                                     {4, 512, 2, 0}};
  return tab[(v >= 0 && v < GBC_CELL_VARIANTS) ? v : 0];
}

cudaError_t launch_cell_f32(const CellJob* jobs, int n, int variant, cudaStream_t s) {
  switch (variant) {
    case 1: return launch_cell_f32_v1(jobs, n, s);
    case 2: return launch_cell_f32_v2(jobs, n, s);
    case 3: return launch_cell_f32_v3(jobs, n, s);
    case 4: return launch_cell_f32_v4(jobs, n, s);

    default: return launch_cell_f32_v0(jobs, n, s);
  }
}
