// gs_track.cu -- the window step of GridShift-based object tracking (Sec. 2.3,
// Algorithm 2): the pixels R of a search window whose colour cell floor(c / h)
// lies in the reference set B, with the count, the exact position sums and
// extent of R, and which cells of B occur in R (the next B).
//
// One thread per window pixel: per channel, the exact cell key of its colour
// (floor of the exact quotient) decided by integer compares against a table
// of exact cell faces spanning B's keys on that channel (a colour outside
// that span cannot be in B), then a binary search in B sorted
// lexicographically, warp and block reductions and one set of global atomics
// per block.  No float64 arithmetic: the pass is bound by the read of the
// window's colours; B and the face table stay in L1/L2.
#include <cstdint>

#include "gs_common.cuh"

namespace gs {

namespace {

template <int D, typename T>
__global__ void __launch_bounds__(kBlock)
    k_track(const T* __restrict__ frame, int64_t width, int64_t x0, int64_t y0, int64_t ww,
            int64_t npix, TrackPlan tp, const int64_t* __restrict__ thr,
            const int64_t* __restrict__ bins, int64_t k, TrackAcc* acc,
            uint8_t* __restrict__ present) {
  __shared__ unsigned long long s_cnt, s_bad;
  __shared__ long long s_sx, s_sy, s_mnx, s_mxx, s_mny, s_mxy;
  if (threadIdx.x == 0) {
    s_cnt = 0;
    s_bad = 0;
    s_sx = s_sy = 0;
    s_mnx = s_mny = INT64_MAX;
    s_mxx = s_mxy = INT64_MIN;
  }
  __syncthreads();
  unsigned long long cnt = 0, bad = 0;
  long long sx = 0, sy = 0, mnx = INT64_MAX, mxx = INT64_MIN, mny = INT64_MAX, mxy = INT64_MIN;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride) {
    const int64_t x = x0 + p % ww, y = y0 + p / ww;
    const T* c = frame + (size_t)(y * width + x) * D;
    int64_t key[D];
    bool valid = true, inside = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const uint64_t b = load_bits<T>(c + a);
      // not finite, or |c| >= lim (4e15 h): no exact cell (counted invalid)
      valid = valid && (b & 0x7FFFFFFFFFFFFFFFull) < tp.lim_bits;
      const int64_t v = ord_of_bits(b);
      const int64_t* t = thr + tp.toff[a];
      // outside the faces of B's keys on this axis: not in B
      inside = inside && v >= __ldg(&t[0]) && v < __ldg(&t[tp.span[a]]);
      key[a] = inside ? tp.lo[a] + key_index(t, tp.span[a], tp.lo[a], tp.inv_h, b) : 0;
    }
    if (!valid) {
      ++bad;
      continue;
    }
    if (!inside) continue;
    // lexicographic binary search for the first bin >= key
    int64_t lo = 0, hi = k;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      int cmp = 0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int64_t b = __ldg(&bins[mid * D + a]);
        if (cmp == 0) cmp = b < key[a] ? -1 : (b > key[a] ? 1 : 0);
      }
      if (cmp < 0) lo = mid + 1; else hi = mid;
    }
    bool hit = lo < k;
#pragma unroll
    for (int a = 0; a < D; ++a) hit = hit && __ldg(&bins[lo * D + a]) == key[a];
    if (!hit) continue;
    if (!present[lo]) present[lo] = 1;
    ++cnt;
    sx += x;
    sy += y;
    mnx = x < mnx ? x : mnx;
    mxx = x > mxx ? x : mxx;
    mny = y < mny ? y : mny;
    mxy = y > mxy ? y : mxy;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(kFull, cnt, o);
    bad += __shfl_xor_sync(kFull, bad, o);
    sx += __shfl_xor_sync(kFull, sx, o);
    sy += __shfl_xor_sync(kFull, sy, o);
    mnx = min(mnx, __shfl_xor_sync(kFull, mnx, o));
    mxx = max(mxx, __shfl_xor_sync(kFull, mxx, o));
    mny = min(mny, __shfl_xor_sync(kFull, mny, o));
    mxy = max(mxy, __shfl_xor_sync(kFull, mxy, o));
  }
  if ((threadIdx.x & 31) == 0 && (cnt != 0 || bad != 0)) {
    atomicAdd(&s_cnt, cnt);
    atomicAdd(&s_bad, bad);
    atomicAdd((unsigned long long*)&s_sx, (unsigned long long)sx);
    atomicAdd((unsigned long long*)&s_sy, (unsigned long long)sy);
    atomicMin(&s_mnx, mnx);
    atomicMax(&s_mxx, mxx);
    atomicMin(&s_mny, mny);
    atomicMax(&s_mxy, mxy);
  }
  __syncthreads();
  if (threadIdx.x == 0 && (s_cnt != 0 || s_bad != 0)) {
    atomicAdd(&acc->count, s_cnt);
    atomicAdd(&acc->bad, s_bad);
    atomicAdd((unsigned long long*)&acc->sum_x, (unsigned long long)s_sx);
    atomicAdd((unsigned long long*)&acc->sum_y, (unsigned long long)s_sy);
    atomicMin(&acc->min_x, s_mnx);
    atomicMax(&acc->max_x, s_mxx);
    atomicMin(&acc->min_y, s_mny);
    atomicMax(&acc->max_y, s_mxy);
  }
}

}  // namespace

cudaError_t launch_track(const void* frame, bool f32, int d, int64_t width, int64_t x0,
                         int64_t y0, int64_t ww, int64_t wh, const TrackPlan& tp,
                         const int64_t* thr, const int64_t* bins, int64_t k, TrackAcc* acc,
                         uint8_t* present, cudaStream_t s) {
  const int64_t npix = ww * wh;
  if (npix <= 0) return cudaSuccess;
  const unsigned g = grid_for(npix, kBlock, 152u * 8u);
  if (f32) {
    GS_DISPATCH_D(d, k_track<D, float><<<g, kBlock, 0, s>>>((const float*)frame, width, x0, y0,
                                                            ww, npix, tp, thr, bins, k, acc,
                                                            present));
  } else {
    GS_DISPATCH_D(d, k_track<D, double><<<g, kBlock, 0, s>>>((const double*)frame, width, x0, y0,
                                                             ww, npix, tp, thr, bins, k, acc,
                                                             present));
  }
  return cudaGetLastError();
}

}  // namespace gs
