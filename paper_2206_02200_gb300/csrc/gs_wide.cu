// gs_wide.cu -- GridShift (Kumar et al., arXiv 2206.02200, Sec. 2.1, Algorithm
// 1, Eq. 1-4 in the parallel form of Eq. 6) for cell keys that the main
// pipeline's 63-bit packed key cannot hold: d up to 12, any number of cells
// along an axis (|x / h| < 4e15), key fields of any total width.
//
// A key is one biased int64 field per axis (k_a - kmin_a, kmin_a the data's
// smallest cell minus one), kept in structure-of-arrays form.  The cells of
// a level are stored in ascending lexicographic key order (axis 0 first),
// which is also the final numbering of the clusters:
//   binning     every point's key (floor of the exact quotient x / h), a
//               stable LSD radix sort of the points by key (one sort per
//               axis, last axis first), runs of equal keys -> cells, exact
//               cell sums by fixed-point atomics, rounded once;
//   update      one warp per cell walks the 3^d neighbour keys, each found
//               by binary search in the sorted cells; the exact sum over the
//               neighbours present divided by their count, rounded once; the
//               new key floor(centroid / h); the count-weighted centroid as an
//               exact fixed-point product; whether a neighbour v != 0 exists;
//   merge       a stable sort of the cells by new key, runs of equal keys ->
//               the next level's cells (counts and exact sums added, rounded
//               once), each old cell's parent recorded;
//   labels      every initial cell's chain of parents followed to its final
//               cell, whose index is its label; modes = sum / count.
// The host drives the levels (one synchronisation per update for the stop
// test, one per merge for the next cell count).  The fixed-point arithmetic
// is the main pipeline's (gs_device.cuh), so results are bit-identical to it
// and to the float64 oracle.
#include <cmath>
#include <cstring>
#include <vector>

#include "gs_common.cuh"
#include "gs_planner.cuh"
#include "gs_wide.h"

namespace gs {

namespace {

constexpr int kWB = 256;             // threads per block
constexpr int kScanTile = 4 * kWB;   // elements per block of the scan kernels

constexpr uint32_t kWideErrWindow = 1u;  // a value above the fixed-point window
constexpr uint32_t kWideErrBox = 2u;     // a key outside the widened key box

struct WideFlags {
  long long min_ord[kMaxWideD];
  long long max_ord[kMaxWideD];
  unsigned long long maxabs[kMaxWideD];
  unsigned long long bad;      // non-finite coordinates
  unsigned long long inexact;  // fixed-point truncations or unroundable centroids
  uint32_t err;                // kWideErr* bits
  uint32_t has_nb;             // some cell of the level has a neighbour v != 0
};

// Per-axis parameters of a run.
struct WidePlan {
  int d;
  int nprobe;                  // 3^d
  double h;
  int64_t kmin[kMaxWideD];     // the key box: biased keys 0 .. span - 1
  int64_t span[kMaxWideD];
  int L[kMaxWideD];            // fixed-point unit 2^L of each axis
};

__device__ __forceinline__ double as_double(uint64_t b) { return __longlong_as_double((long long)b); }

__device__ __forceinline__ u128 as_u128w(ulonglong2 v) { return (u128)v.x | ((u128)v.y << 64); }

__device__ __forceinline__ ulonglong2 pack_w(u128 v) {
  return make_ulonglong2((uint64_t)v, (uint64_t)(v >> 64));
}

// ---------------------------------------------------------------------------
// Key range and finiteness (any d <= kMaxWideD): per-axis extremes in
// registers, reduced per warp, published with one atomic per warp and axis.
template <typename T>
__global__ void __launch_bounds__(kWB) k_wide_range(const T* __restrict__ pts, int64_t n, int d,
                                                    WideFlags* fl) {
  long long mn[kMaxWideD], mx[kMaxWideD];
  unsigned long long ma[kMaxWideD];
#pragma unroll
  for (int a = 0; a < kMaxWideD; ++a) {
    mn[a] = INT64_MAX;
    mx[a] = INT64_MIN;
    ma[a] = 0;
  }
  unsigned long long bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
    for (int a = 0; a < kMaxWideD; ++a) {
      if (a >= d) continue;
      const uint64_t b = load_bits<T>(pts + (size_t)i * d + a);
      if (((b >> 52) & 0x7FF) == 0x7FF) {
        ++bad;
        continue;
      }
      const long long o = (long long)ord_of_bits(b);
      mn[a] = o < mn[a] ? o : mn[a];
      mx[a] = o > mx[a] ? o : mx[a];
      const unsigned long long ab = b & 0x7FFFFFFFFFFFFFFFull;
      ma[a] = ab > ma[a] ? ab : ma[a];
    }
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int a = 0; a < kMaxWideD; ++a) {
    if (a >= d) continue;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long x = __shfl_xor_sync(kFull, mn[a], o);
      const long long y = __shfl_xor_sync(kFull, mx[a], o);
      const unsigned long long z = __shfl_xor_sync(kFull, ma[a], o);
      mn[a] = x < mn[a] ? x : mn[a];
      mx[a] = y > mx[a] ? y : mx[a];
      ma[a] = z > ma[a] ? z : ma[a];
    }
    if (lane == 0 && mn[a] != INT64_MAX) {
      atomicMin(&fl->min_ord[a], mn[a]);
      atomicMax(&fl->max_ord[a], mx[a]);
      atomicMax(&fl->maxabs[a], ma[a]);
    }
  }
  if (bad) atomicAdd(&fl->bad, bad);
}

// Biased cell key of every point along every axis (keys[a * n + i]) and the
// identity permutation.
template <typename T>
__global__ void __launch_bounds__(kWB) k_wide_keys(const T* __restrict__ pts, int64_t n, WidePlan P,
                                                   uint64_t* __restrict__ keys,
                                                   uint32_t* __restrict__ vals, WideFlags* fl) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    vals[i] = (uint32_t)i;
    for (int a = 0; a < P.d; ++a) {
      const double x = as_double(load_bits<T>(pts + (size_t)i * P.d + a));
      int64_t q = plan_floor_div(x, P.h) - P.kmin[a];
      if (q < 0 || q >= P.span[a]) {
        atomicOr(&fl->err, kWideErrBox);
        q = 0;
      }
      keys[(size_t)a * n + i] = (uint64_t)q;
    }
  }
}

__global__ void k_wide_iota(uint32_t* __restrict__ v, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v[i] = i;
}

// dst[i] = src[idx[i]]: one axis of the keys in the current sorted order.
__global__ void k_wide_gather(const uint64_t* __restrict__ src, const uint32_t* __restrict__ idx,
                              uint64_t* __restrict__ dst, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

// flag[i] = 1 where the key of element vals[i] differs from that of
// vals[i - 1] (a run of equal keys starts), keys[a * ld + e] per axis.
__global__ void k_wide_heads(const uint64_t* __restrict__ keys, size_t ld, int d,
                             const uint32_t* __restrict__ vals, uint32_t n,
                             uint32_t* __restrict__ flag) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t h = i == 0 ? 1u : 0u;
    if (i > 0) {
      const uint32_t e = vals[i], f = vals[i - 1];
      for (int a = 0; a < d && !h; ++a) h = keys[a * ld + e] != keys[a * ld + f] ? 1u : 0u;
    }
    flag[i] = h;
  }
}

// Inclusive scan of 32-bit counts in three launches: tile sums, an exclusive
// scan of the tile sums in one block, then each tile scanned from its offset.
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t* s_w, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  uint32_t before = 0, all = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
    before += q < w ? s_w[q] : 0u;
    all += s_w[q];
  }
  __syncthreads();
  if (total) *total = all;
  return before + x;
}

__global__ void __launch_bounds__(kWB) k_scan_tiles(const uint32_t* __restrict__ in, uint32_t n,
                                                    uint32_t* __restrict__ sums) {
  __shared__ uint32_t s_w[kWB / 32];
  const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * 4;
  uint32_t v = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) v += base + k < n ? in[base + k] : 0u;
  uint32_t total = 0;
  block_incl_scan(v, s_w, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kWB) k_scan_sums(uint32_t* sums, uint32_t nt) {
  __shared__ uint32_t s_w[kWB / 32];
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t c0 = 0; c0 < nt; c0 += blockDim.x) {
    const uint32_t i = c0 + threadIdx.x;
    const uint32_t v = i < nt ? sums[i] : 0u;
    uint32_t total = 0;
    const uint32_t incl = block_incl_scan(v, s_w, &total);
    if (i < nt) sums[i] = s_carry + incl - v;  // exclusive
    __syncthreads();
    if (threadIdx.x == 0) s_carry += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kWB) k_scan_apply(const uint32_t* __restrict__ in, uint32_t n,
                                                    const uint32_t* __restrict__ sums,
                                                    uint32_t* __restrict__ out) {
  __shared__ uint32_t s_w[kWB / 32];
  const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * 4;
  uint32_t v[4], t = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = base + k < n ? in[base + k] : 0u;
    t += v[k];
  }
  const uint32_t incl = block_incl_scan(t, s_w, nullptr);
  uint32_t run = sums[blockIdx.x] + incl - t;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    run += v[k];
    if (base + k < n) out[base + k] = run;
  }
}

// Cells from the sorted points: position i (point vals[i]) belongs to cell
// ids[i] - 1; the first position of a run writes the cell's key; counts and
// exact coordinate sums are added with atomics (acc: m x d limb quadruples,
// zero before).
template <typename T>
__global__ void __launch_bounds__(kWB) k_wide_bin_cells(const T* __restrict__ pts, int64_t n,
                                                        WidePlan P, const uint64_t* __restrict__ pkeys,
                                                        const uint32_t* __restrict__ vals,
                                                        const uint32_t* __restrict__ ids,
                                                        uint32_t* __restrict__ cell0,
                                                        uint64_t* __restrict__ ckey, size_t ld,
                                                        uint32_t* __restrict__ cnt,
                                                        uint64_t* __restrict__ acc, WideFlags* fl) {
  unsigned inexact = 0, werr = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (uint32_t)n;
       i += gridDim.x * blockDim.x) {
    const uint32_t e = vals[i];
    const uint32_t c = ids[i] - 1;
    cell0[e] = c;
    atomicAdd(&cnt[c], 1u);
    const bool head = i == 0 || ids[i - 1] != ids[i];
    for (int a = 0; a < P.d; ++a) {
      if (head) ckey[a * ld + c] = pkeys[(size_t)a * n + e];
      const u128 V = to_fixed(load_bits<T>(pts + (size_t)e * P.d + a), P.L[a], inexact, werr);
      atomic_add_fixed(acc + ((size_t)c * P.d + a) * 4, V);
    }
  }
  if (inexact) atomicAdd(&fl->inexact, 1ull);
  if (werr) atomicOr(&fl->err, kWideErrWindow);
}

// The exact sums of m cells rounded once to float64 (kept in fixed point);
// the accumulators are cleared.
__global__ void k_wide_settle(uint64_t* __restrict__ acc, uint32_t m, WidePlan P,
                              ulonglong2* __restrict__ csum, WideFlags* fl) {
  unsigned werr = 0;
  const size_t total = (size_t)m * P.d;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total;
       w += (size_t)gridDim.x * blockDim.x) {
    uint64_t* q = acc + w * 4;
    const int a = (int)(w % P.d);
    csum[w] = pack_w(round_to_double(limbs_value(q), P.L[a], werr));
    q[0] = q[1] = q[2] = q[3] = 0;
  }
  if (werr) atomicOr(&fl->err, kWideErrWindow);
}

// Index of the cell with biased key nk among m cells sorted by key, or -1.
__device__ __forceinline__ int64_t wide_find(const uint64_t* __restrict__ ckey, size_t ld, int d,
                                             uint32_t m, const int64_t (&nk)[kMaxWideD]) {
  uint32_t lo = 0, hi = m;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    int c = 0;
#pragma unroll
    for (int a = 0; a < kMaxWideD; ++a) {
      if (a >= d || c != 0) continue;
      const int64_t k = (int64_t)__ldg(&ckey[a * ld + mid]);
      c = k < nk[a] ? -1 : (k > nk[a] ? 1 : 0);
    }
    if (c == 0) return mid;
    if (c < 0) lo = mid + 1; else hi = mid;
  }
  return -1;
}

// One update step (Eq. 1-2, parallel form Eq. 6; steps ii-iii and the
// neighbour test of step v) for the m cells of a level, one warp per cell:
// the lanes share the 3^d neighbour offsets (axis 0 the slowest digit),
// find each neighbour key by binary search and add its count and exact sum;
// lane a < d then forms coordinate a of the centroid, its new key and the
// cell's count-weighted centroid C(j) S'(j) (exact product).
__global__ void __launch_bounds__(kWB) k_wide_update(WidePlan P, uint32_t m,
                                                     const uint64_t* __restrict__ ckey, size_t ld,
                                                     const uint32_t* __restrict__ cnt,
                                                     const ulonglong2* __restrict__ csum,
                                                     uint64_t* __restrict__ wkey,
                                                     ulonglong2* __restrict__ wval, WideFlags* fl) {
  unsigned inexact = 0, werr = 0, box = 0;
  const int lane = threadIdx.x & 31;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const int d = P.d;
  bool any_nb = false;
  for (uint32_t j = gwarp; j < m; j += nwarps) {
    int64_t kj[kMaxWideD];
#pragma unroll
    for (int a = 0; a < kMaxWideD; ++a) kj[a] = a < d ? (int64_t)ckey[a * ld + j] : 0;
    uint32_t Dc = 0;
    u128 N[kMaxWideD];
#pragma unroll
    for (int a = 0; a < kMaxWideD; ++a) N[a] = 0;
    bool nb = false;
    for (int p = lane; p < P.nprobe; p += 32) {
      int64_t nk[kMaxWideD];
      bool ok = true, nz = false;
      int rest = p;
#pragma unroll
      for (int a = kMaxWideD - 1; a >= 0; --a) {
        nk[a] = 0;
        if (a >= d) continue;
        const int v = rest % 3 - 1;
        rest /= 3;
        nk[a] = kj[a] + v;
        nz = nz || v != 0;
        ok = ok && nk[a] >= 0 && nk[a] < P.span[a];
      }
      if (!ok) continue;
      const int64_t q = wide_find(ckey, ld, d, m, nk);
      if (q < 0) continue;
      Dc += cnt[q];
      nb = nb || nz;
#pragma unroll
      for (int a = 0; a < kMaxWideD; ++a)
        if (a < d) N[a] += as_u128w(csum[(size_t)q * d + a]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Dc += __shfl_xor_sync(kFull, Dc, o);
#pragma unroll
      for (int a = 0; a < kMaxWideD; ++a) {
        if (a >= d) continue;
        const uint64_t lo = __shfl_xor_sync(kFull, (uint64_t)N[a], o);
        const uint64_t hi = __shfl_xor_sync(kFull, (uint64_t)(N[a] >> 64), o);
        N[a] += (u128)lo | ((u128)hi << 64);
      }
    }
    nb = __any_sync(kFull, nb);
    any_nb = any_nb || nb;
    if (lane < d) {
      u128 Na = 0;
      int La = 0;
      int64_t kmin = 0, span = 0;
#pragma unroll
      for (int a = 0; a < kMaxWideD; ++a)
        if (a == lane) {
          Na = N[a];
          La = P.L[a];
          kmin = P.kmin[a];
          span = P.span[a];
        }
      const double sv = div_round(Na, Dc, La, inexact);
      int64_t q = plan_floor_div(sv, P.h) - kmin;
      if (q < 0 || q >= span) {
        box = 1;
        q = 0;
      }
      wkey[lane * ld + j] = (uint64_t)q;
      const u128 V = to_fixed((uint64_t)__double_as_longlong(sv), La, inexact, werr);
      wval[(size_t)j * d + lane] = pack_w(V * (u128)cnt[j]);
    }
  }
  if (__any_sync(kFull, any_nb) && lane == 0) atomicOr(&fl->has_nb, 1u);
  if (inexact) atomicAdd(&fl->inexact, 1ull);
  if (werr) atomicOr(&fl->err, kWideErrWindow);
  if (box) atomicOr(&fl->err, kWideErrBox);
}

// The merge (Eq. 3-4): sorted position i holds old cell j = vals[i], which
// joins new cell ids[i] - 1 (its parent); the new cell adds the old count and
// the exact count-weighted centroid; the first position of a run writes the
// new cell's key.
__global__ void __launch_bounds__(kWB) k_wide_merge(WidePlan P, uint32_t m,
                                                    const uint32_t* __restrict__ vals,
                                                    const uint32_t* __restrict__ ids,
                                                    const uint64_t* __restrict__ wkey, size_t ld,
                                                    const ulonglong2* __restrict__ wval,
                                                    const uint32_t* __restrict__ cnt,
                                                    uint64_t* __restrict__ nkey,
                                                    uint32_t* __restrict__ ncnt,
                                                    uint64_t* __restrict__ acc,
                                                    uint32_t* __restrict__ parent) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const uint32_t j = vals[i];
    const uint32_t c = ids[i] - 1;
    parent[j] = c;
    atomicAdd(&ncnt[c], cnt[j]);
    const bool head = i == 0 || ids[i - 1] != ids[i];
    for (int a = 0; a < P.d; ++a) {
      if (head) nkey[a * ld + c] = wkey[a * ld + j];
      atomic_add_fixed(acc + ((size_t)c * P.d + a) * 4, as_u128w(wval[(size_t)j * P.d + a]));
    }
  }
}

// Final cell (= label) of every initial cell: its chain of T parents, level
// t's parents at forest[t * m0 .. t * m0 + m_t).
__global__ void k_wide_roots(const uint32_t* __restrict__ forest, uint32_t m0, int T,
                             uint32_t* __restrict__ root) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m0; c += gridDim.x * blockDim.x) {
    uint32_t v = c;
    for (int t = 0; t < T; ++t) v = forest[(size_t)t * m0 + v];
    root[c] = v;
  }
}

__global__ void k_wide_labels(const uint32_t* __restrict__ cell0, const uint32_t* __restrict__ root,
                              int32_t* __restrict__ labels, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    labels[i] = (int32_t)root[cell0[i]];
}

// Mode of final cell r: its sum rounded to float64 divided by its count.
__global__ void k_wide_modes(const ulonglong2* __restrict__ csum, const uint32_t* __restrict__ cnt,
                             uint32_t k, WidePlan P, double* __restrict__ modes, WideFlags* fl) {
  unsigned inexact = 0;
  const size_t total = (size_t)k * P.d;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total;
       w += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(w % P.d);
    modes[w] = round_fixed(as_u128w(csum[w]), P.L[a], inexact) / (double)cnt[w / P.d];
  }
  if (inexact) atomicAdd(&fl->inexact, 1ull);
}

// A growable device buffer of the wide workspace.
template <typename T>
struct WBuf {
  T* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = n + n / 4 + 64;
    cudaError_t e = cudaMalloc((void**)&p, want * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    cap = want;
    return cudaSuccess;
  }
  // keeps the first `keep` elements
  cudaError_t grow(size_t n, size_t keep, cudaStream_t s) {
    if (n <= cap && p) return cudaSuccess;
    const size_t want = n + n / 2 + 64;
    T* q = nullptr;
    cudaError_t e = cudaMalloc((void**)&q, want * sizeof(T));
    if (e != cudaSuccess) return e;
    if (p && keep) {
      e = cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        cudaFree(q);
        return e;
      }
    }
    if (p) cudaFree(p);
    p = q;
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

}  // namespace

struct WideWorkspace {
  WBuf<WideFlags> flags;
  WideFlags* h_flags = nullptr;  // pinned
  uint32_t* h_word = nullptr;    // pinned: one count read back
  WBuf<uint64_t> pkeys, skey, tkey;
  WBuf<uint32_t> vals, tvals, hist, flag, ids, sums, cell0, root;
  WBuf<uint64_t> ckey[2], wkey, acc;
  WBuf<uint32_t> cnt[2], forest;
  WBuf<ulonglong2> csum[2], wval;
  void release() {
    flags.release();
    pkeys.release(); skey.release(); tkey.release();
    vals.release(); tvals.release(); hist.release(); flag.release(); ids.release();
    sums.release(); cell0.release(); root.release();
    for (int i = 0; i < 2; ++i) {
      ckey[i].release();
      cnt[i].release();
      csum[i].release();
    }
    wkey.release(); acc.release(); forest.release(); wval.release();
    if (h_flags) cudaFreeHost(h_flags);
    if (h_word) cudaFreeHost(h_word);
    h_flags = nullptr;
    h_word = nullptr;
  }
};

WideWorkspace* wide_workspace_new() { return new (std::nothrow) WideWorkspace(); }

void wide_workspace_free(WideWorkspace* w) {
  if (!w) return;
  w->release();
  delete w;
}

namespace {

gs_status wfail(std::string* err, gs_status s, const std::string& msg) {
  if (err) *err = msg;
  return s;
}

gs_status wcuda(std::string* err, cudaError_t e, const char* where) {
  if (err) *err = std::string(where) + ": " + cudaGetErrorName(e);
  return e == cudaErrorMemoryAllocation ? GS_E_NOMEM : GS_E_CUDA;
}

}  // namespace

#define W_CU(call, where)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return wcuda(err, e_, where);   \
  } while (0)
#define W_LAUNCH(call, where, nk)                               \
  do {                                                          \
    call;                                                       \
    W_CU(cudaGetLastError(), where);                            \
    info->launches += (nk);                                     \
  } while (0)

gs_status wide_fit(WideWorkspace* w, const FitArgs& a, int64_t* k_out, gs_fit_info* info,
                   std::string* err) {
  if (!w) return wfail(err, GS_E_NOMEM, "no wide workspace");
  if (a.B != 1 || a.mixed || a.sequential || a.d < 1 || a.d > kMaxWideD || a.n < 1)
    return wfail(err, GS_E_INVALID,
                 "keys wider than the packed key: plain GS_FP64 runs with the parallel update");
  const int d = a.d;
  const int64_t n = a.n;
  const cudaStream_t s = a.stream;
  const uint32_t un = (uint32_t)n;
  if (!w->h_flags) W_CU(cudaMallocHost((void**)&w->h_flags, sizeof(WideFlags)), "pinned flags");
  if (!w->h_word) W_CU(cudaMallocHost((void**)&w->h_word, sizeof(uint32_t)), "pinned word");
  W_CU(w->flags.ensure(1), "alloc flags");
  WideFlags* hf = w->h_flags;
  WideFlags* fl = w->flags.p;
  std::memset(hf, 0, sizeof(WideFlags));
  for (int i = 0; i < kMaxWideD; ++i) {
    hf->min_ord[i] = INT64_MAX;
    hf->max_ord[i] = INT64_MIN;
  }
  W_CU(cudaMemcpyAsync(fl, hf, sizeof(WideFlags), cudaMemcpyHostToDevice, s), "H2D flags");
  const unsigned gp = grid_for(n, kWB, 152u * 8u);
  if (a.f32)
    W_LAUNCH((k_wide_range<float><<<gp, kWB, 0, s>>>((const float*)a.points, n, d, fl)),
             "k_wide_range", 1);
  else
    W_LAUNCH((k_wide_range<double><<<gp, kWB, 0, s>>>((const double*)a.points, n, d, fl)),
             "k_wide_range", 1);
  W_CU(cudaMemcpyAsync(hf, fl, sizeof(WideFlags), cudaMemcpyDeviceToHost, s), "D2H flags");
  W_CU(cudaStreamSynchronize(s), "sync key range");
  if (hf->bad) return wfail(err, GS_E_INVALID, "non-finite input coordinate");

  // the plan: per axis the data's key box widened by one cell each side
  // (centroids are convex combinations, Eq. 1 and 3) and the fixed-point unit
  WidePlan P;
  std::memset(&P, 0, sizeof(P));
  P.d = d;
  P.h = a.h;
  P.nprobe = 1;
  for (int i = 0; i < d; ++i) P.nprobe *= 3;
  int clog2n = 0;
  while ((1ll << clog2n) < n) ++clog2n;
  int bits[kMaxWideD] = {};
  for (int ax = 0; ax < d; ++ax) {
    const double lo = plan_from_ord(hf->min_ord[ax]), hi = plan_from_ord(hf->max_ord[ax]);
    if (!(std::fabs(lo / a.h) < 4.0e15) || !(std::fabs(hi / a.h) < 4.0e15))
      return wfail(err, GS_E_KEYRANGE, "a coordinate divided by h exceeds 2^52");
    P.kmin[ax] = plan_floor_div(lo, a.h) - 1;
    P.span[ax] = plan_floor_div(hi, a.h) + 1 - P.kmin[ax] + 1;
    bits[ax] = plan_bitlen((uint64_t)P.span[ax]);
    double ma;
    const uint64_t mb = hf->maxabs[ax];
    std::memcpy(&ma, &mb, 8);
    int e = 0;
    if (ma > 0) std::frexp(ma, &e);
    P.L[ax] = e + clog2n - 126;
  }

  // binning: keys, the points sorted by key, runs -> cells
  W_CU(w->pkeys.ensure((size_t)d * un), "alloc keys");
  W_CU(w->skey.ensure(un), "alloc sort");
  W_CU(w->tkey.ensure(un), "alloc sort");
  W_CU(w->vals.ensure(un), "alloc sort");
  W_CU(w->tvals.ensure(un), "alloc sort");
  W_CU(w->hist.ensure(radix_hist_words(un)), "alloc sort");
  W_CU(w->flag.ensure(un), "alloc flags");
  W_CU(w->ids.ensure(un), "alloc ids");
  W_CU(w->sums.ensure((un + kScanTile - 1) / kScanTile + 1), "alloc scan");
  W_CU(w->cell0.ensure(un), "alloc cell0");
  if (a.f32)
    W_LAUNCH((k_wide_keys<float><<<gp, kWB, 0, s>>>((const float*)a.points, n, P, w->pkeys.p,
                                                    w->vals.p, fl)), "k_wide_keys", 1);
  else
    W_LAUNCH((k_wide_keys<double><<<gp, kWB, 0, s>>>((const double*)a.points, n, P, w->pkeys.p,
                                                     w->vals.p, fl)), "k_wide_keys", 1);

  // stable sort of the elements vals[0 .. cnt) by the keys keys[a * ld + e],
  // one radix sort per axis, the last axis first; then the run ids (1-based)
  auto sort_and_number = [&](const uint64_t* keys, size_t ld, uint32_t count,
                             uint32_t* m_out) -> gs_status {
    const unsigned g = grid_for(count, kWB);
    for (int ax = d - 1; ax >= 0; --ax) {
      W_LAUNCH((k_wide_gather<<<g, kWB, 0, s>>>(keys + (size_t)ax * ld, w->vals.p, w->skey.p,
                                                count)), "k_wide_gather", 1);
      W_CU(radix_sort(w->skey.p, w->vals.p, w->tkey.p, w->tvals.p, w->hist.p, count, bits[ax], s),
           "radix_sort");
      info->launches += radix_sort_launches(count, bits[ax]);
    }
    W_LAUNCH((k_wide_heads<<<g, kWB, 0, s>>>(keys, ld, d, w->vals.p, count, w->flag.p)),
             "k_wide_heads", 1);
    const uint32_t nt = (count + kScanTile - 1) / kScanTile;
    W_LAUNCH((k_scan_tiles<<<nt, kWB, 0, s>>>(w->flag.p, count, w->sums.p)), "k_scan_tiles", 1);
    W_LAUNCH((k_scan_sums<<<1, kWB, 0, s>>>(w->sums.p, nt)), "k_scan_sums", 1);
    W_LAUNCH((k_scan_apply<<<nt, kWB, 0, s>>>(w->flag.p, count, w->sums.p, w->ids.p)),
             "k_scan_apply", 1);
    W_CU(cudaMemcpyAsync(w->h_word, w->ids.p + (count - 1), sizeof(uint32_t),
                         cudaMemcpyDeviceToHost, s), "D2H cell count");
    W_CU(cudaStreamSynchronize(s), "sync cell count");
    *m_out = *w->h_word;
    return GS_OK;
  };

  uint32_t m0 = 0;
  {
    const gs_status st = sort_and_number(w->pkeys.p, (size_t)un, un, &m0);
    if (st != GS_OK) return st;
  }
  info->m0 = m0;
  const size_t ld = m0;  // stride of the per-axis key arrays of the cell levels
  for (int i = 0; i < 2; ++i) {
    W_CU(w->ckey[i].ensure((size_t)d * m0), "alloc cell keys");
    W_CU(w->cnt[i].ensure(m0), "alloc counts");
    W_CU(w->csum[i].ensure((size_t)m0 * d), "alloc sums");
  }
  W_CU(w->wkey.ensure((size_t)d * m0), "alloc new keys");
  W_CU(w->wval.ensure((size_t)m0 * d), "alloc new sums");
  W_CU(w->acc.ensure((size_t)m0 * d * 4), "alloc accumulators");
  W_CU(w->root.ensure(m0), "alloc roots");
  W_CU(w->forest.ensure((size_t)m0 * 4), "alloc forest");
  W_CU(cudaMemsetAsync(w->acc.p, 0, sizeof(uint64_t) * (size_t)m0 * d * 4, s), "memset acc");
  W_CU(cudaMemsetAsync(w->cnt[0].p, 0, sizeof(uint32_t) * m0, s), "memset counts");
  if (a.f32)
    W_LAUNCH((k_wide_bin_cells<float><<<grid_for(n, kWB), kWB, 0, s>>>(
                 (const float*)a.points, n, P, w->pkeys.p, w->vals.p, w->ids.p, w->cell0.p,
                 w->ckey[0].p, ld, w->cnt[0].p, w->acc.p, fl)), "k_wide_bin_cells", 1);
  else
    W_LAUNCH((k_wide_bin_cells<double><<<grid_for(n, kWB), kWB, 0, s>>>(
                 (const double*)a.points, n, P, w->pkeys.p, w->vals.p, w->ids.p, w->cell0.p,
                 w->ckey[0].p, ld, w->cnt[0].p, w->acc.p, fl)), "k_wide_bin_cells", 1);
  W_LAUNCH((k_wide_settle<<<grid_for((int64_t)m0 * d, kWB), kWB, 0, s>>>(w->acc.p, m0, P,
                                                                          w->csum[0].p, fl)),
           "k_wide_settle", 1);

  // the update steps
  int t = 0, cur = 0;
  uint32_t m = m0;
  bool converged = false;
  int64_t cell_iters = 0;
  const unsigned gw = grid_for((int64_t)m0 * 32, kWB, 152u * 16u);
  for (;;) {
    W_CU(cudaMemsetAsync(&fl->has_nb, 0, sizeof(uint32_t), s), "memset has_nb");
    W_LAUNCH((k_wide_update<<<gw, kWB, 0, s>>>(P, m, w->ckey[cur].p, ld, w->cnt[cur].p,
                                               w->csum[cur].p, w->wkey.p, w->wval.p, fl)),
             "k_wide_update", 1);
    W_CU(cudaMemcpyAsync(hf, fl, sizeof(WideFlags), cudaMemcpyDeviceToHost, s), "D2H flags");
    W_CU(cudaStreamSynchronize(s), "sync update");
    if (hf->err) break;
    if (!hf->has_nb) {
      converged = true;
      break;
    }
    if (t == a.max_iter) break;
    // the merge into level t + 1: cells sorted by new key (stable: members
    // in ascending old key), runs -> cells, parents of level t
    W_CU(w->forest.grow((size_t)(t + 1) * m0, (size_t)t * m0, s), "alloc forest");
    W_LAUNCH((k_wide_iota<<<grid_for(m, kWB), kWB, 0, s>>>(w->vals.p, m)), "k_wide_iota", 1);
    uint32_t m1 = 0;
    {
      const gs_status st = sort_and_number(w->wkey.p, ld, m, &m1);
      if (st != GS_OK) return st;
    }
    const int nx = cur ^ 1;
    W_CU(cudaMemsetAsync(w->cnt[nx].p, 0, sizeof(uint32_t) * m1, s), "memset counts");
    W_LAUNCH((k_wide_merge<<<grid_for(m, kWB), kWB, 0, s>>>(
                 P, m, w->vals.p, w->ids.p, w->wkey.p, ld, w->wval.p, w->cnt[cur].p,
                 w->ckey[nx].p, w->cnt[nx].p, w->acc.p, w->forest.p + (size_t)t * m0)),
             "k_wide_merge", 1);
    W_LAUNCH((k_wide_settle<<<grid_for((int64_t)m1 * d, kWB), kWB, 0, s>>>(w->acc.p, m1, P,
                                                                            w->csum[nx].p, fl)),
             "k_wide_settle", 1);
    cell_iters += m;
    m = m1;
    cur = nx;
    ++t;
  }
  if (hf->err & kWideErrWindow)
    return wfail(err, GS_E_INTERNAL, "a value above the fixed-point window");
  if (hf->err & kWideErrBox) return wfail(err, GS_E_INTERNAL, "a cell key left the key box");
  const uint32_t k = m;
  // labels: every initial cell's final cell is its label (cells are in key order)
  W_LAUNCH((k_wide_roots<<<grid_for(m0, kWB), kWB, 0, s>>>(w->forest.p, m0, t, w->root.p)),
           "k_wide_roots", 1);
  W_LAUNCH((k_wide_labels<<<grid_for(n, kWB), kWB, 0, s>>>(w->cell0.p, w->root.p, a.labels, n)),
           "k_wide_labels", 1);
  if ((int64_t)k <= a.modes_cap)
    W_LAUNCH((k_wide_modes<<<grid_for((int64_t)k * d, kWB), kWB, 0, s>>>(
                 w->csum[cur].p, w->cnt[cur].p, k, P, a.modes, fl)), "k_wide_modes", 1);
  W_CU(cudaMemcpyAsync(hf, fl, sizeof(WideFlags), cudaMemcpyDeviceToHost, s), "D2H flags");
  W_CU(cudaStreamSynchronize(s), "sync labels");
  info->iterations = t;
  info->converged = converged ? 1 : 0;
  info->k = k;
  info->inexact = (int64_t)hf->inexact;
  info->cell_iters = cell_iters;
  *k_out = k;
  if ((int64_t)k > a.modes_cap) return wfail(err, GS_E_CAPACITY, "modes_cap < number of clusters");
  return GS_OK;
}

}  // namespace gs
