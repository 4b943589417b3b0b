// gs_loop32.cu -- the loop kernel of the float32 mixed-precision variant
// (GS_FP32_MIXED): float-float sums of float32 cell offsets, with float64
// rechecks of key decisions near cell faces, for d = 1 .. 8.
#include "gs_loop.cuh"

namespace gs {

int loop_grid_fp32(int d) { return loop_grid_t<true>(d); }

cudaError_t launch_loop_fp32(const LoopArgs& a, int grid, cudaStream_t s) {
  return launch_loop_t<true>(a, grid, s);
}

cudaError_t launch_modes_tail_fp32(const LoopArgs& a, uint32_t k, int T, cudaStream_t s) {
  return launch_modes_tail_t<true>(a, k, T, s);
}

cudaError_t launch_prep_sums_fp32(const LoopArgs& a, cudaStream_t s) {
  return launch_prep_sums_t<true>(a, s);
}

}  // namespace gs
