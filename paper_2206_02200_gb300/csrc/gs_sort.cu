// gs_sort.cu -- stable LSD radix sort of (uint64 key, uint32 value) pairs,
// 8 bits per pass.  Used to number the final cells by ascending packed key
// (lexicographic order of the integer cell keys, axis 0 first).
//
// Per pass: (1) every tile of kTile elements counts its digits; (2) one block
// turns the digit-major table of counts into exclusive offsets; (3) every tile
// scatters its elements, ranking equal digits in input order (warp by warp,
// chunk by chunk, lane by lane) so the pass is stable.
#include "gs_kernels.h"

namespace gs {

namespace {

constexpr int kSortThreads = 256;
constexpr int kWarps = kSortThreads / 32;
constexpr int kPerLane = 16;                    // chunks of 32 per warp
constexpr int kWarpSpan = 32 * kPerLane;        // elements per warp
constexpr int kTile = kWarps * kWarpSpan;       // elements per block
constexpr unsigned kAll = 0xFFFFFFFFu;

__global__ void __launch_bounds__(kSortThreads)
    k_hist(const uint64_t* __restrict__ keys, uint32_t n, int shift, uint32_t* __restrict__ hist,
           uint32_t nblocks) {
  __shared__ uint32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  uint32_t base = blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += blockDim.x) {
    uint32_t e = base + i;
    if (e < n) atomicAdd(&h[(keys[e] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[(size_t)i * nblocks + blockIdx.x] = h[i];
}

// Exclusive scan of hist[0 .. total) in place, one block.
__global__ void __launch_bounds__(1024) k_scan(uint32_t* hist, uint32_t total) {
  __shared__ uint32_t part[1024];
  uint32_t per = (total + blockDim.x - 1) / blockDim.x;
  uint32_t lo = threadIdx.x * per;
  uint32_t hi = lo + per < total ? lo + per : total;
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; ++i) s += hist[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (unsigned i = 0; i < blockDim.x; ++i) {
      uint32_t v = part[i];
      part[i] = run;
      run += v;
    }
  }
  __syncthreads();
  uint32_t run = part[threadIdx.x];
  for (uint32_t i = lo; i < hi; ++i) {
    uint32_t v = hist[i];
    hist[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(kSortThreads)
    k_scatter(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint32_t n,
              int shift, const uint32_t* __restrict__ offs, uint32_t nblocks,
              uint64_t* __restrict__ okeys, uint32_t* __restrict__ ovals) {
  __shared__ uint32_t cnt[kWarps][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kWarps * 256; i += blockDim.x) (&cnt[0][0])[i] = 0;
  __syncthreads();
  const uint32_t wbase = blockIdx.x * kTile + warp * kWarpSpan;
  uint32_t loc[kPerLane];
  uint32_t dig[kPerLane];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int c = 0; c < kPerLane; ++c) {
    uint32_t e = wbase + c * 32 + lane;
    bool valid = e < n;
    uint32_t g = valid ? (uint32_t)((keys[e] >> shift) & 0xFF) : 256u;
    unsigned peers = __match_any_sync(kAll, g);
    uint32_t before = valid ? cnt[warp][g] : 0u;
    __syncwarp();
    loc[c] = before + __popc(peers & lt);
    dig[c] = g;
    if (valid && (peers & lt) == 0) cnt[warp][g] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int g = threadIdx.x; g < 256; g += blockDim.x) {
    uint32_t run = offs[(size_t)g * nblocks + blockIdx.x];
    for (int w = 0; w < kWarps; ++w) {
      uint32_t v = cnt[w][g];
      cnt[w][g] = run;
      run += v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kPerLane; ++c) {
    uint32_t e = wbase + c * 32 + lane;
    if (e < n) {
      uint32_t dst = cnt[warp][dig[c]] + loc[c];
      okeys[dst] = keys[e];
      ovals[dst] = vals[e];
    }
  }
}

}  // namespace

size_t radix_hist_words(uint32_t n) {
  size_t nb = (n + kTile - 1) / kTile;
  if (nb == 0) nb = 1;
  return nb * 256;
}

int radix_sort_launches(uint32_t n, int nbits) {
  if (n <= 1 || nbits <= 0) return 0;
  return 3 * ((nbits + 7) / 8);
}

cudaError_t radix_sort(uint64_t* keys, uint32_t* vals, uint64_t* tkeys, uint32_t* tvals,
                       uint32_t* hist, uint32_t n, int nbits, cudaStream_t s) {
  if (n <= 1 || nbits <= 0) return cudaSuccess;
  uint32_t nblocks = (n + kTile - 1) / kTile;
  uint64_t* ik = keys;
  uint32_t* iv = vals;
  uint64_t* ok = tkeys;
  uint32_t* ov = tvals;
  int passes = (nbits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int shift = p * 8;
    k_hist<<<nblocks, kSortThreads, 0, s>>>(ik, n, shift, hist, nblocks);
    k_scan<<<1, 1024, 0, s>>>(hist, nblocks * 256);
    k_scatter<<<nblocks, kSortThreads, 0, s>>>(ik, iv, n, shift, hist, nblocks, ok, ov);
    uint64_t* tk = ik; ik = ok; ok = tk;
    uint32_t* tv = iv; iv = ov; ov = tv;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ik != keys) {
    e = cudaMemcpyAsync(keys, ik, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(vals, iv, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
  }
  return e;
}

}  // namespace gs
