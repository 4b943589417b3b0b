// gs_loop64.cu -- the loop kernel with exact fixed-point sums rounded once to
// float64 (the GS_FP64 precision), for d = 1 .. 8.
#include "gs_loop.cuh"

namespace gs {

int loop_grid_fp64(int d) { return loop_grid_t<false>(d); }

cudaError_t launch_loop_fp64(const LoopArgs& a, int grid, cudaStream_t s) {
  return launch_loop_t<false>(a, grid, s);
}

cudaError_t launch_modes_tail_fp64(const LoopArgs& a, uint32_t k, int T, cudaStream_t s) {
  return launch_modes_tail_t<false>(a, k, T, s);
}

cudaError_t launch_prep_sums_fp64(const LoopArgs& a, cudaStream_t s) {
  return launch_prep_sums_t<false>(a, s);
}

// the precision-independent launches of step i's second pass and the labels
cudaError_t launch_prep_offsets(const LoopArgs& a, cudaStream_t s) {
  return launch_prep_offsets_t<false>(a, s);
}

cudaError_t launch_prep_scatter(const LoopArgs& a, cudaStream_t s) {
  return launch_prep_scatter_t<false>(a, s);
}

cudaError_t launch_labels_out(const LoopArgs& a, cudaStream_t s) {
  return launch_labels_out_t<false>(a, s);
}

}  // namespace gs
