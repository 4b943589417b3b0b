// gs_loop64s.cu -- the loop kernel of the sequential update (Sec. 2.2, Eq. 5)
// with exact fixed-point sums rounded once to float64 (GS_FP64, one point
// set), for d = 1 .. 8: each update is 2^d passes, one per parity colour.
// Only this translation unit instantiates k_loop<D, false, false, true>.
#include "gs_loop.cuh"

namespace gs {

namespace {

// Its own co-resident grid and launch.
template <int D>
int loop_grid_seq_d() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const int smem = (int)(kFilterWords * sizeof(uint32_t));
  if (cudaFuncSetAttribute(k_loop<D, false, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_loop<D, false, false, true>,
                                                    kLoopBlock, smem) != cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  if (per_sm > 2) per_sm = 2;
  const int g = sms * per_sm;
  return g < kMaxLoopGrid ? g : kMaxLoopGrid;
}

int loop_grid_seq_t(int d) {
  switch (d) {
    case 1: return loop_grid_seq_d<1>();
    case 2: return loop_grid_seq_d<2>();
    case 3: return loop_grid_seq_d<3>();
    case 4: return loop_grid_seq_d<4>();
    case 5: return loop_grid_seq_d<5>();
    case 6: return loop_grid_seq_d<6>();
    case 7: return loop_grid_seq_d<7>();
    case 8: return loop_grid_seq_d<8>();
  }
  return -1;
}

cudaError_t launch_loop_seq_t(const LoopArgs& a, int grid, cudaStream_t s) {
  LoopArgs args = a;
  void* params[] = {&args};
  const size_t smem = kFilterWords * sizeof(uint32_t);
  GS_DISPATCH_D(a.P.d, return cudaLaunchCooperativeKernel(
                           (const void*)k_loop<D, false, false, true>, dim3(grid),
                           dim3(kLoopBlock), params, smem, s));
  return cudaSuccess;
}

}  // namespace

int loop_grid_seq(int d) { return loop_grid_seq_t(d); }

cudaError_t launch_loop_seq(const LoopArgs& a, int grid, cudaStream_t s) {
  return launch_loop_seq_t(a, grid, s);
}

}  // namespace gs
