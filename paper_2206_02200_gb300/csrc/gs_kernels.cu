// gs_kernels.cu -- the GridShift hot path on sm_103a.
//
// Steps (Kumar et al., arXiv 2206.02200, Sec. 2.1 and Algorithm 1):
//   k_range  key range, fixed-point window and finiteness of the input
//   k_bin    step i: cell key of every point, per-cell count and exact sum
//   k_loop   one cooperative launch for everything after binning:
//              level 0 (the initial cells and their lookup table), then per
//              update step t:
//                gather   steps ii-iii: Eq. 1-2 over the 3^d neighbours in the
//                         parallel form (Eq. 6), centroid rounded once, new key,
//                         and the neighbour test of step v
//                merge    step iv: cells sharing a new key add their counts and
//                         count-weighted centroids (Eq. 3-4) exactly
//                compact  the next level's cells and lookup table
//              then the forest of merges (the union of resident sets of Eq. 4)
//              is resolved by pointer jumping, the final cells are numbered by
//              ascending key, and every point gets its label.
//            Phases are separated by a software grid barrier whose waits are
//            bounded in time.
#include <cstdio>

#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kLoopBlock = 512;  // threads per block of the loop kernel

inline unsigned grid_for(int64_t work, int per_block = kBlock, unsigned cap = 152u * 32u) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > (int64_t)cap) g = cap;
  return (unsigned)g;
}

#define GS_DISPATCH_D(dval, ...)                  \
  switch (dval) {                                 \
    case 1: { constexpr int D = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int D = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int D = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int D = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int D = 5; __VA_ARGS__; } break; \
    case 6: { constexpr int D = 6; __VA_ARGS__; } break; \
    case 7: { constexpr int D = 7; __VA_ARGS__; } break; \
    case 8: { constexpr int D = 8; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;        \
  }

// ---------------------------------------------------------------------------
// Key range and finiteness

// The point array is read as one flat stream of n*D values in words of W
// values (W = 16 bytes / sizeof(T) when the array is 16-byte aligned, else 1):
// thread t reads the words t, t + S, t + 2S, ... with S a multiple of D, so
// the j-th value of every word a thread reads has the same coordinate
// (t*W + j) mod D, and consecutive threads read consecutive words
// (coalesced).  Four words per thread are in flight at once.  Per-coordinate
// extremes are reduced in shared memory and published with one global atomic
// per block and coordinate.
template <int W, typename T>
struct Word;
template <>
struct Word<1, double> {
  static __device__ __forceinline__ void load(const double* p, uint64_t (&b)[1]) {
    b[0] = (uint64_t)__double_as_longlong(__ldg(p));
  }
};
template <>
struct Word<1, float> {
  static __device__ __forceinline__ void load(const float* p, uint64_t (&b)[1]) {
    b[0] = f32_bits_to_f64_bits(__float_as_uint(__ldg(p)));
  }
};
template <>
struct Word<2, double> {
  static __device__ __forceinline__ void load(const double* p, uint64_t (&b)[2]) {
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p));
    b[0] = v.x;
    b[1] = v.y;
  }
};
template <>
struct Word<4, float> {
  static __device__ __forceinline__ void load(const float* p, uint64_t (&b)[4]) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    b[0] = f32_bits_to_f64_bits(v.x);
    b[1] = f32_bits_to_f64_bits(v.y);
    b[2] = f32_bits_to_f64_bits(v.z);
    b[3] = f32_bits_to_f64_bits(v.w);
  }
};

struct RangeAcc {
  int64_t mn = INT64_MAX, mx = INT64_MIN;
  uint64_t ma = 0;
  __device__ __forceinline__ void add(uint64_t b, unsigned long long& bad) {
    if (((b >> 52) & 0x7FF) == 0x7FF) {
      ++bad;
      return;
    }
    const int64_t o = ord_of_bits(b);
    mn = o < mn ? o : mn;
    mx = o > mx ? o : mx;
    const uint64_t ab = b & 0x7FFFFFFFFFFFFFFFull;
    ma = ab > ma ? ab : ma;
  }
};

template <int D, typename T, int W>
__global__ void __launch_bounds__(kBlock) k_range(const T* __restrict__ pts, int64_t n,
                                                  DevFlags* fl) {
  constexpr int U = 4;  // words in flight per thread
  __shared__ long long s_mn[D], s_mx[D];
  __shared__ unsigned long long s_ma[D], s_bad;
  if (threadIdx.x < D) {
    s_mn[threadIdx.x] = INT64_MAX;
    s_mx[threadIdx.x] = INT64_MIN;
    s_ma[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  const int64_t total = n * D;
  const int64_t words = total / W;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t S = nthreads - nthreads % D;  // stride in words, a multiple of D
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  RangeAcc acc[W];
  unsigned long long bad = 0;
  if (t < S) {
    int64_t q = t;
    for (; q + (U - 1) * S < words; q += U * S) {
      uint64_t b[U][W];
#pragma unroll
      for (int u = 0; u < U; ++u) Word<W, T>::load(pts + (q + u * S) * W, b[u]);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < W; ++j) acc[j].add(b[u][j], bad);
    }
    for (; q < words; q += S) {
      uint64_t b[W];
      Word<W, T>::load(pts + q * W, b);
#pragma unroll
      for (int j = 0; j < W; ++j) acc[j].add(b[j], bad);
    }
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const int a = (int)((t * W + j) % D);
      if (acc[j].mn != INT64_MAX) {
        atomicMin(&s_mn[a], (long long)acc[j].mn);
        atomicMax(&s_mx[a], (long long)acc[j].mx);
        atomicMax(&s_ma[a], (unsigned long long)acc[j].ma);
      }
    }
  }
  if (t == 0) {
    // values after the last whole word
    for (int64_t e = words * W; e < total; ++e) {
      uint64_t b[1];
      Word<1, T>::load(pts + e, b);
      RangeAcc r;
      r.add(b[0], bad);
      const int a = (int)(e % D);
      if (r.mn != INT64_MAX) {
        atomicMin(&s_mn[a], (long long)r.mn);
        atomicMax(&s_mx[a], (long long)r.mx);
        atomicMax(&s_ma[a], (unsigned long long)r.ma);
      }
    }
  }
  if (bad) atomicAdd(&s_bad, bad);
  __syncthreads();
  if (threadIdx.x < D && s_mn[threadIdx.x] != INT64_MAX) {
    atomicMin(&fl->min_ord[threadIdx.x], s_mn[threadIdx.x]);
    atomicMax(&fl->max_ord[threadIdx.x], s_mx[threadIdx.x]);
    atomicMax(&fl->maxabs[threadIdx.x], s_ma[threadIdx.x]);
  }
  if (threadIdx.x == 0 && s_bad) atomicAdd(&fl->bad, s_bad);
}

// ---------------------------------------------------------------------------
// Step i: binning, first pass (cell keys and counts)
//
// A warp takes 32 consecutive points at a time.  It copies their d
// coordinates (one contiguous run of 32*d values) into shared memory with
// 16-byte loads, so the global reads are coalesced.  Lanes holding the same
// cell key (__match_any_sync) are counted together: only the lowest such lane
// touches the global table, with one insert and one count add per distinct
// key per warp.  The exact cell sums are formed later (k_loop, after a
// counting sort of the points by cell), without per-point atomics.

template <typename T>
__device__ __forceinline__ void stage_points(const T* __restrict__ src, int count,
                                             T* __restrict__ dst, bool vec_ok, int lane) {
  // src: first value of the run, count values; dst: shared memory
  int done = 0;
  if (vec_ok) {
    const int nvec = (int)((size_t)count * sizeof(T) / 16);
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (int v = lane; v < nvec; v += 32) d4[v] = __ldg(&s4[v]);
    done = (int)((size_t)nvec * 16 / sizeof(T));
  }
  for (int e = done + lane; e < count; e += 32) dst[e] = __ldg(&src[e]);
}

__device__ __forceinline__ uint64_t bits_of(double v) { return (uint64_t)__double_as_longlong(v); }
__device__ __forceinline__ uint64_t bits_of(float v) {
  return f32_bits_to_f64_bits((uint32_t)__float_as_uint(v));
}

// Instance of point i in a batched run: the b with offsets[b] <= i < offsets[b + 1].
__device__ __forceinline__ uint32_t instance_of(const int64_t* __restrict__ offsets, int B,
                                                int64_t i) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&offsets[mid]) <= i) lo = mid; else hi = mid - 1;
  }
  return (uint32_t)lo;
}

template <int D, typename T>
__global__ void __launch_bounds__(kBlock)
    k_bin(const T* __restrict__ pts, int64_t n, Plan P, const int64_t* __restrict__ thr,
          BinTable T0, uint32_t mask0, uint32_t maxcells, uint32_t* __restrict__ slot0,
          DevFlags* fl, bool vec_ok, const int64_t* __restrict__ offsets, int B) {
  __shared__ __align__(16) T s_pts[kWarps][32 * D];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = gwarp * 32; base < n; base += nwarps * 32) {
    const int cnt = n - base < 32 ? (int)(n - base) : 32;
    stage_points<T>(pts + base * D, cnt * D, s_pts[w], vec_ok, lane);
    __syncwarp();
    const bool valid = lane < cnt;
    uint64_t key = kEmpty;
    if (valid) {
      key = B > 1 ? (uint64_t)instance_of(offsets, B, base + lane) << P.inst_off : 0ull;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const uint64_t b = bits_of(s_pts[w][lane * D + a]);
        const int idx = key_index(thr + P.thr_off[a], P.span[a], P.kmin[a], P.inv_h, b);
        key |= (uint64_t)(idx + 1) << P.off[a];
      }
    }
    __syncwarp();
    const unsigned peers = __match_any_sync(kFull, key);
    const int leader = __ffs(peers) - 1;
    uint32_t s = kNone;
    if (valid && lane == leader) {
      bool won;
      s = table_insert(T0.key, mask0, key, won, &fl->err);
      if (s != kNone) {
        if (won) {
          const uint32_t id = atomicAdd(&fl->m0, 1u);
          if (id < maxcells) T0.list[id] = s; else atomicOr(&fl->err, kErrOverflow);
        }
        atomicAdd(&T0.cnt[s], (uint32_t)__popc(peers));
      }
    }
    s = __shfl_sync(kFull, s, leader);
    if (valid) slot0[base + lane] = s;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Software grid barrier for the cooperative loop kernel.  All blocks are
// co-resident (cooperative launch).  Block leaders arrive on a counter; the
// last one, after every block's writes of the phase, reads the error flags,
// records whether the kernel must stop, resets the counter and advances the
// generation the others wait on.  Every block therefore takes the same stop
// decision at the same barrier.  A wait gives up after kBarrierNs of global
// time, sets kErrBarrier and makes the kernel return.

constexpr unsigned long long kBarrierNs = 10ull * 1000ull * 1000ull * 1000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_sync(GridBar* bar, DevFlags* fl) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = &bar->gen;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar->count, 0u);
      *(volatile unsigned int*)&bar->stop = *(volatile uint32_t*)&fl->err != 0u ? 1u : 0u;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*vgen == g) {
        __nanosleep(64);
        if (global_ns() - t0 > kBarrierNs) {
          atomicOr(&fl->err, kErrBarrier);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok && *(volatile unsigned int*)&bar->stop == 0u;
  }
  __syncthreads();
  return s_ok != 0;
}

// Device-clock split of the loop kernel, kept by thread 0 of block 0.
struct SegClock {
  unsigned long long last = 0;
  unsigned long long ns[kLoopPhases] = {};
  bool on = false;
  __device__ void start() {
    on = blockIdx.x == 0 && threadIdx.x == 0;
    if (on) last = global_ns();
  }
  __device__ void lap(int seg) {
    if (!on) return;
    const unsigned long long now = global_ns();
    ns[seg] += now - last;
    last = now;
  }
};

enum {
  kSegOffsets = 0,
  kSegScatter = 1,
  kSegSums = 2,
  kSegLevel0 = 3,
  kSegUpdateFirst = 4,
  kSegUpdateRest = 5,
  kSegCompact = 6,
  kSegLabels = 7
};

__device__ __forceinline__ u128 as_u128(ulonglong2 v) { return (u128)v.x | ((u128)v.y << 64); }

__device__ __forceinline__ ulonglong2 pack(u128 v) {
  return make_ulonglong2((uint64_t)v, (uint64_t)(v >> 64));
}

// The cell sum of one axis as the float64 value of Sec. 2.1 (the exact sum in
// the limb accumulators rounded once), held as the fixed-point integer it
// equals; clears the accumulators.
__device__ __forceinline__ ulonglong2 settle_sum(uint64_t* acc, int L, unsigned& inexact,
                                                 unsigned& werr) {
  const double v = round_fixed(limbs_value(acc), L, inexact);
  acc[0] = acc[1] = acc[2] = acc[3] = 0;
  return pack(to_fixed(bits_of(v), L, inexact, werr));
}

// ---------------------------------------------------------------------------
// Occupancy filter of a level: one bit per hashed key (a Bloom filter with
// one hash function), 2^B bits with 2^B >= 32 m (at most kFilterBits).  A
// neighbour probe whose bit is clear cannot hit and never leaves the SM: the
// update phase copies the level's filter into shared memory first.
constexpr uint32_t kFilterBits = 1u << kFilterLog2Max;

__device__ __forceinline__ int filter_log2(uint32_t m) {
  int b = 10;
  while (b < kFilterLog2Max && (1u << b) < 32u * m) ++b;
  return b;
}

__device__ __forceinline__ uint32_t filter_bit(uint64_t key, int lg) {
  return (uint32_t)((key * 0xD6E8FEB86659FD93ull) >> (64 - lg));
}

__device__ __forceinline__ void filter_set(uint32_t* f, uint64_t key, int lg) {
  const uint32_t b = filter_bit(key, lg);
  atomicOr(&f[b >> 5], 1u << (b & 31));
}

// Lanes given to one cell in the update: a power of two, at least d and at
// least GatherLanes<D>::min.  Few lanes per cell put several cells in flight
// per warp, which hides the latency of their dependent table loads when a
// level has many cells; a level with few cells gets 32 lanes per cell, which
// shortens each cell's chain of probes.
template <int D>
struct GatherLanes {
  static constexpr int min = D <= 3 ? 4 : D <= 5 ? 8 : D == 6 ? 16 : 32;
};

constexpr int pow3(int d) { return d == 0 ? 1 : 3 * pow3(d - 1); }

// Probes each lane has in flight at once: min(4, its probes per cell).
template <int D, int GS>
struct ProbeBatch {
  static constexpr int probes = pow3(D);
  static constexpr int per_lane = (probes + GS - 1) / GS;
  static constexpr int value = per_lane < 4 ? per_lane : 4;
};

// ---------------------------------------------------------------------------
// Step i, second pass: the exact sum of every cell, by a counting sort of the
// points by cell.  Offsets follow the cells' list order; a cell's points then
// occupy one contiguous run of perm[], and a warp reading 32 consecutive
// entries adds each run of equal cells with a segmented shuffle reduction, so
// the sum accumulators receive a few atomic adds per run instead of d per
// point.  Exact integer sums make the order irrelevant.

// Per-block totals of the counts of cells [b * chunk, (b + 1) * chunk).
__device__ void phase_count_totals(const LoopArgs& A, uint32_t m0) {
  __shared__ uint32_t s_part[kLoopBlock / 32];
  const uint32_t chunk = (m0 + gridDim.x - 1) / gridDim.x;
  const uint32_t lo = blockIdx.x * chunk;
  const uint32_t hi = lo + chunk < m0 ? lo + chunk : m0;
  uint32_t sum = 0;
  for (uint32_t id = lo + threadIdx.x; id < hi; id += blockDim.x) sum += A.T0.cnt[A.T0.list[id]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
    A.blocksum[blockIdx.x] = t;
  }
}

// Start offset of every cell's run: T0.off[slot] = points of all earlier cells.
__device__ void phase_offsets(const LoopArgs& A, uint32_t m0) {
  __shared__ uint32_t s_warp[kLoopBlock / 32];
  __shared__ uint32_t s_base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (w == 0) {
    uint32_t t = 0;
    for (uint32_t b = lane; b < blockIdx.x; b += 32) t += A.blocksum[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    if (lane == 0) s_base = t;
  }
  __syncthreads();
  const uint32_t chunk = (m0 + gridDim.x - 1) / gridDim.x;
  const uint32_t lo = blockIdx.x * chunk;
  const uint32_t hi = lo + chunk < m0 ? lo + chunk : m0;
  uint32_t run = s_base;
  for (uint32_t c0 = lo; c0 < hi; c0 += blockDim.x) {
    const uint32_t id = c0 + threadIdx.x;
    const uint32_t slot = id < hi ? A.T0.list[id] : 0u;
    const uint32_t v = id < hi ? A.T0.cnt[slot] : 0u;
    uint32_t x = v;  // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int q = 0; q < nw; ++q) {
      const uint32_t t = s_warp[q];
      before += q < w ? t : 0u;
      total += t;
    }
    if (id < hi) A.T0.off[slot] = run + before + x - v;
    run += total;
    __syncthreads();
  }
}

// perm[off[cell] + rank] = point: each point claims a position in its cell's
// run (equal cells within a warp claim theirs with one atomic add).  A warp
// handles kScatterBatch chunks of 32 points at once, so their loads and
// atomics are in flight together.
constexpr int kScatterBatch = 4;

__device__ void phase_scatter(const LoopArgs& A) {
  constexpr int B = kScatterBatch;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = gwarp * 32 * B; base < A.n; base += nwarps * 32 * B) {
    uint32_t s[B], pos[B];
    unsigned peers[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int64_t i = base + b * 32 + lane;
      s[b] = i < A.n ? A.slot0[i] : kNone;
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      peers[b] = __match_any_sync(kFull, s[b]);
      pos[b] = 0;
      if (lane == __ffs(peers[b]) - 1 && s[b] != kNone)
        pos[b] = atomicAdd(&A.T0.off[s[b]], (uint32_t)__popc(peers[b]));
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const uint32_t p = __shfl_sync(kFull, pos[b], __ffs(peers[b]) - 1);
      if (s[b] != kNone) A.perm[p + __popc(peers[b] & below)] = (uint32_t)(base + b * 32 + lane);
    }
  }
}

// Exact sums of the cells: sums of the fixed-point values of their points.
// Lane l of a warp takes kSumRun consecutive entries of perm[] (one 16-byte
// load) and adds the runs of equal cells among them in registers; every run
// but its last is added into the cell's limb accumulators at once.  The
// lanes' last runs are contiguous in cell order across the warp, so a
// segmented shuffle reduction combines them and the first lane of each
// segment adds the segment's sum.
constexpr int kSumRun = 4;

template <int D>
__device__ __forceinline__ void add_cell_sum(const LoopArgs& A, uint32_t s, const u128 (&V)[D]) {
#pragma unroll
  for (int a = 0; a < D; ++a) atomic_add_fixed(A.T0.acc + ((size_t)s * D + a) * 4, V[a]);
}

template <int D, typename T>
__device__ void phase_cell_sums(const LoopArgs& A, unsigned& inexact, unsigned& werr) {
  constexpr int E = kSumRun;
  const T* __restrict__ pts = static_cast<const T*>(A.pts);
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = gwarp * 32 * E; base < A.n; base += nwarps * 32 * E) {
    const int64_t p0 = base + (int64_t)lane * E;
    uint32_t idx[E], s[E];
    if (p0 + E <= A.n) {
      const uint4 q = *reinterpret_cast<const uint4*>(A.perm + p0);
      idx[0] = q.x;
      idx[1] = q.y;
      idx[2] = q.z;
      idx[3] = q.w;
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) idx[e] = p0 + e < A.n ? A.perm[p0 + e] : kNone;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) s[e] = idx[e] != kNone ? A.slot0[idx[e]] : kNone;
    uint64_t raw[E][D];
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int a = 0; a < D; ++a)
        raw[e][a] = idx[e] != kNone ? load_bits<T>(pts + (size_t)idx[e] * D + a) : 0ull;
    // runs within the lane
    uint32_t cur = s[0];
    u128 V[D];
#pragma unroll
    for (int a = 0; a < D; ++a) V[a] = to_fixed(raw[0][a], A.P.L[a], inexact, werr);
#pragma unroll
    for (int e = 1; e < E; ++e) {
      if (s[e] != cur) {
        if (cur != kNone) add_cell_sum<D>(A, cur, V);
        cur = s[e];
#pragma unroll
        for (int a = 0; a < D; ++a) V[a] = 0;
      }
#pragma unroll
      for (int a = 0; a < D; ++a) V[a] += to_fixed(raw[e][a], A.P.L[a], inexact, werr);
    }
    // the lanes' last runs: lane l ends with the sum of [l, end of its segment)
    const uint32_t prev = __shfl_up_sync(kFull, cur, 1);
    const bool head = lane == 0 || prev != cur;
    const unsigned heads = __ballot_sync(kFull, head);
    const unsigned after = lane == 31 ? 0u : heads & ~((2u << lane) - 1u);
    const int end = after ? __ffs(after) - 1 : 32;
    if (__any_sync(kFull, end - lane > 1)) {
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const uint64_t lo = __shfl_down_sync(kFull, (uint64_t)V[a], o);
          const uint64_t hi = __shfl_down_sync(kFull, (uint64_t)(V[a] >> 64), o);
          if (lane + o < end) V[a] += (u128)lo | ((u128)hi << 64);
        }
      }
    }
    if (head && cur != kNone) add_cell_sum<D>(A, cur, V);
  }
}

// Level 0: the cells binning created (in arrival order), their sums rounded
// once, in the level table tab[0].  Resets the binning table's slots.
template <int D>
__device__ void phase_level0(const LoopArgs& A, uint32_t m0, uint32_t maskA, unsigned& inexact,
                             unsigned& werr) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nth = gridDim.x * blockDim.x;
  const BinTable T0 = A.T0;
  const LevelTable G = A.tab[0];
  const Cells c = A.cells[0];
  const int lg0 = filter_log2(m0);
  for (uint32_t id = tid; id < m0; id += nth) {
    const uint32_t s = T0.list[id];
    const uint64_t key = T0.key[s];
    const uint32_t cnt = T0.cnt[s];
    bool won;
    const uint32_t sa = table_insert(G.key, maskA, key, won, &A.fl->err);
    if (sa != kNone) {
      ulonglong2* r = G.row + (size_t)sa * (D + 1);
      r[0] = make_ulonglong2((uint64_t)cnt, 0ull);
#pragma unroll
      for (int a = 0; a < D; ++a)
        r[1 + a] = settle_sum(T0.acc + ((size_t)s * D + a) * 4, A.P.L[a], inexact, werr);
      G.id[sa] = id;
      G.list[id] = sa;
    }
    filter_set(A.filter[0], key, lg0);
    c.key[id] = key;
    c.cnt[id] = cnt;
    T0.cnt[s] = 0;
    T0.key[s] = kEmpty;
  }
}

// One update step t for every cell of level t (table tab[t % 3]):
//   ii)  D = sum of the counts and N = sum of the coordinate sums over the
//        3^d neighbours present (Eq. 1-2, all cells reading level t: Eq. 6),
//        centroid N / D rounded once, and whether a neighbour v != 0 is
//        present (step v);
//   iii) new key floor(centroid / h);
//   iv)  the cell's count and count-weighted centroid (Eq. 3-4) added exactly
//        into the slot of its new key in tab[(t + 1) % 3].
// The merge is applied before the stop test is known; when the test stops
// the run, the merge table is cleared instead of used.
// For t > 0 the same phase links every cell of level t-1 to its cell of level
// t (the union of resident sets of Eq. 4) and clears level t-1's table.
template <int D, int GS, bool BT>
__device__ void phase_update(const LoopArgs& A, int t, uint32_t m, uint32_t mask, uint32_t maskM,
                             uint32_t m_prev, uint32_t base_prev, uint32_t base, bool& any_nb,
                             unsigned& inexact, unsigned& werr) {
  constexpr int U = ProbeBatch<D, GS>::value;
  const int lane = threadIdx.x & 31;
  const int glane = lane & (GS - 1);
  const unsigned gmask = GS == 32 ? kFull : (((1u << GS) - 1u) << (lane & ~(GS - 1)));
  const uint32_t group = (blockIdx.x * blockDim.x + threadIdx.x) / GS;
  const uint32_t ngroups = (gridDim.x * blockDim.x) / GS;
  const LevelTable G = A.tab[t % 3];
  const LevelTable M = A.tab[(t + 1) % 3];
  const Cells c = A.cells[t & 1];
  uint32_t* pslot = A.pslot[t & 1];
  const int nprobe = A.P.nprobe, center = A.P.center;
  // the level's occupancy filter, into shared memory; the filter of level
  // t-1 is cleared for level t+1
  extern __shared__ uint4 s_dyn[];
  uint32_t* s_filter = reinterpret_cast<uint32_t*>(s_dyn);
  const int lg = filter_log2(m);
  {
    const uint4* src = reinterpret_cast<const uint4*>(A.filter[t & 1]);
    uint4* dst = reinterpret_cast<uint4*>(s_filter);
    const uint32_t n4 = (1u << lg) / 128;
    for (uint32_t w = threadIdx.x; w < n4; w += blockDim.x) dst[w] = __ldcg(src + w);
    if (t > 0) {
      uint4* old = reinterpret_cast<uint4*>(A.filter[(t + 1) & 1]);
      const uint32_t o4 = (1u << filter_log2(m_prev)) / 128;
      const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
      for (uint32_t w = tid; w < o4; w += gridDim.x * blockDim.x) old[w] = make_uint4(0, 0, 0, 0);
    }
    if (BT) {
      // per-instance flags of the next step start clear
      const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
      for (uint32_t b = tid; b < (uint32_t)A.B; b += gridDim.x * blockDim.x) {
        A.I.nbf[(t + 1) & 1][b] = 0;
        A.I.mt[(t + 1) & 1][b] = 0;
      }
    }
    __syncthreads();
  }
  for (uint32_t j = group; j < m; j += ngroups) {
    const uint64_t key = c.key[j];
    const uint32_t cj = c.cnt[j];
    // batched runs: a cell of an instance that has stopped is carried to the
    // next level unchanged (same key, its own exact sum)
    uint32_t inst = 0;
    bool live = true;
    if (BT) {
      inst = (uint32_t)(key >> A.P.inst_off);
      live = A.I.done[t & 1][inst] == 0;
    }
    uint32_t Dc = 0;
    bool nbc = false;
    u128 N[D];
#pragma unroll
    for (int a = 0; a < D; ++a) N[a] = 0;
    for (int p0 = glane; live && p0 < nprobe; p0 += GS * U) {
      uint64_t q[U];
      bool v[U];
      uint32_t sl[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = p0 + u * GS;
        q[u] = key + (p < nprobe ? __ldg(&A.dtab[p]) : 0ull);
        const uint32_t fb = filter_bit(q[u], lg);
        v[u] = p < nprobe && ((s_filter[fb >> 5] >> (fb & 31)) & 1u);
      }
      table_find_many<U>(G.key, mask, q, v, sl);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (sl[u] == kNone) continue;
        const ulonglong2* r = G.row + (size_t)sl[u] * (D + 1);
        Dc += (uint32_t)r[0].x;
#pragma unroll
        for (int a = 0; a < D; ++a) N[a] += as_u128(r[1 + a]);
        if (p0 + u * GS != center) nbc = true;
      }
    }
    any_nb = any_nb || nbc;
#pragma unroll
    for (int o = GS / 2; o > 0; o >>= 1) {
      Dc += __shfl_xor_sync(gmask, Dc, o);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        uint64_t lo = (uint64_t)N[a], hi = (uint64_t)(N[a] >> 64);
        lo = __shfl_xor_sync(gmask, lo, o);
        hi = __shfl_xor_sync(gmask, hi, o);
        N[a] += (u128)lo | ((u128)hi << 64);
      }
    }
    // lane a < d: coordinate a of the centroid, its key field, its fixed value
    uint64_t field = 0;
    u128 V = 0;
    int La = 0;
    uint32_t mult = cj;
    if (BT && !live) {
      field = key;
      mult = 1;
      if (glane < D) V = as_u128(G.row[(size_t)G.list[j] * (D + 1) + 1 + glane]);
    } else if (glane < D) {
      u128 Na = 0;
      int off = 0, span = 1, toff = 0;
      int64_t kmin = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a == glane) {
          Na = N[a];
          La = A.P.L[a];
          off = A.P.off[a];
          span = A.P.span[a];
          toff = A.P.thr_off[a];
          kmin = A.P.kmin[a];
        }
      const double sv = div_round(Na, Dc, La, inexact);
      const int idx = key_index(A.thr + toff, span, kmin, A.P.inv_h, bits_of(sv));
      field = (uint64_t)(idx + 1) << off;
      V = to_fixed(bits_of(sv), La, inexact, werr);
    }
    if (!BT || live) {
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1) field |= __shfl_xor_sync(gmask, field, o);
      if (BT) field |= (key >> A.P.inst_off) << A.P.inst_off;  // the instance field
    }
    const bool nbg = BT && (__ballot_sync(gmask, nbc) & gmask) != 0u;
    // iv: merge into the slot of the new key
    uint32_t ms = kNone;
    if (glane == 0) {
      bool won;
      ms = table_insert(M.key, maskM, field, won, &A.fl->err);
      if (ms != kNone) {
        if (won) {
          const uint32_t id = atomicAdd(&A.st[t + 1].m, 1u);
          M.list[id] = ms;
          if (BT) M.id[ms] = j;  // a member, to restore an instance that stops here
        }
        atomicAdd((unsigned long long*)&M.row[(size_t)ms * (D + 1)].x, (unsigned long long)cj);
      }
      pslot[j] = ms;
      if (BT && live) {
        if (nbg && !A.I.nbf[t & 1][inst]) atomicOr(&A.I.nbf[t & 1][inst], 1u);
        atomicAdd(&A.I.mt[t & 1][inst], 1u);
      }
    }
    ms = __shfl_sync(gmask, ms, 0, GS);
    if (glane < D && ms != kNone)
      atomic_add_fixed(M.acc + ((size_t)ms * D + glane) * 4, V * (u128)mult);
  }
  if (t > 0) {
    // level t-1: parent links, then its table is released
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nth = gridDim.x * blockDim.x;
    const LevelTable Lp = A.tab[(t + 2) % 3];
    const uint32_t* pp = A.pslot[(t - 1) & 1];
    for (uint32_t i = tid; i < m_prev; i += nth) {
      A.forest[base_prev + i] = base + G.id[pp[i]];
      const uint32_t s = Lp.list[i];
      Lp.key[s] = kEmpty;
      Lp.row[(size_t)s * (D + 1)].x = 0;
    }
  }
}

// The cells of level t+1 from the merge table: sums rounded once.
// Batched runs: a cell of an instance that stops at step t (it had no
// neighbour) is restored from its single member (no merges happen in such an
// instance), since the update of step t is not applied to it.
template <int D, bool BT>
__device__ void phase_compact(const LoopArgs& A, int t, uint32_t m1, unsigned& inexact,
                              unsigned& werr) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nth = gridDim.x * blockDim.x;
  const LevelTable G = A.tab[t % 3];
  const LevelTable M = A.tab[(t + 1) % 3];
  const Cells cur = A.cells[t & 1];
  const Cells nx = A.cells[(t + 1) & 1];
  uint32_t* f = A.filter[(t + 1) & 1];
  const int lg = filter_log2(m1);
  for (uint32_t id = tid; id < m1; id += nth) {
    const uint32_t s = M.list[id];
    ulonglong2* r = M.row + (size_t)s * (D + 1);
    uint64_t key = M.key[s];
    bool restored = false;
    if (BT) {
      const uint32_t inst = (uint32_t)(key >> A.P.inst_off);
      if (!A.I.done[t & 1][inst] && !A.I.nbf[t & 1][inst]) {
        const uint32_t j = M.id[s];
        const ulonglong2* o = G.row + (size_t)G.list[j] * (D + 1);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          r[1 + a] = o[1 + a];
          uint64_t* acc = M.acc + ((size_t)s * D + a) * 4;
          acc[0] = acc[1] = acc[2] = acc[3] = 0;
        }
        key = cur.key[j];
        restored = true;
      }
    }
    if (!restored) {
#pragma unroll
      for (int a = 0; a < D; ++a)
        r[1 + a] = settle_sum(M.acc + ((size_t)s * D + a) * 4, A.P.L[a], inexact, werr);
    }
    nx.key[id] = key;
    nx.cnt[id] = (uint32_t)r[0].x;
    M.id[s] = id;
    filter_set(f, key, lg);
  }
  if (BT) {
    for (uint32_t b = tid; b < (uint32_t)A.B; b += nth) {
      const bool act = A.I.done[t & 1][b] == 0, nb = A.I.nbf[t & 1][b] != 0;
      A.I.done[(t + 1) & 1][b] = act && nb ? 0u : 1u;
      if (act && nb) A.I.cell_iters[b] += A.I.mt[t & 1][b];
      if (act && !nb) {
        A.I.iters[b] = t;
        A.I.conv[b] = 1;
      }
    }
  }
}

// Mode of final cell r (row of its table slot) written to its label's row,
// then the slot is released.
template <int D>
__device__ __forceinline__ void mode_and_release(const LevelTable& G, const Plan& P, uint32_t r,
                                                 uint32_t label, double* modes, bool write,
                                                 unsigned& inexact) {
  const uint32_t s = G.list[r];
  ulonglong2* row = G.row + (size_t)s * (D + 1);
  if (write) {
    const double cnt = (double)row[0].x;
#pragma unroll
    for (int a = 0; a < D; ++a)
      modes[(size_t)label * D + a] = round_fixed(as_u128(row[1 + a]), P.L[a], inexact) / cnt;
  }
  row[0].x = 0;
  G.key[s] = kEmpty;
}

template <int D, bool BT>
__global__ void __launch_bounds__(kLoopBlock, 1) k_loop(LoopArgs A) {
  unsigned inexact = 0, werr = 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nth = gridDim.x * blockDim.x;
  volatile IterState* vst = A.st;
  SegClock clk;
  clk.start();

  // step i, second pass: exact cell sums
  const uint32_t m0 = *(volatile uint32_t*)&A.fl->m0;
  phase_count_totals(A, m0);
  if (!grid_sync(A.bar, A.fl)) return;
  phase_offsets(A, m0);
  if (!grid_sync(A.bar, A.fl)) return;
  clk.lap(kSegOffsets);
  phase_scatter(A);
  if (!grid_sync(A.bar, A.fl)) return;
  clk.lap(kSegScatter);
  if (A.f32)
    phase_cell_sums<D, float>(A, inexact, werr);
  else
    phase_cell_sums<D, double>(A, inexact, werr);
  if (!grid_sync(A.bar, A.fl)) return;
  clk.lap(kSegSums);

  // level 0
  const uint32_t maskA = mask_for(m0, A.capAB);
  if (tid == 0) {
    A.st[0].m = m0;
    A.st[0].mask = maskA;
    A.st[0].base = 0;
  }
  phase_level0<D>(A, m0, maskA, inexact, werr);
  if (BT) {
    for (uint32_t id = tid; id < m0; id += nth)
      atomicAdd(&A.I.m0[(uint32_t)(A.cells[0].key[id] >> A.P.inst_off)], 1u);
  }
  if (!grid_sync(A.bar, A.fl)) return;
  clk.lap(kSegLevel0);

  int t = 0;
  uint32_t m = m0, mask = maskA, base = 0, m_prev = 0, base_prev = 0;
  unsigned long long cell_iters = 0;
  bool converged = false;
  for (;;) {
    bool any_nb = false;
    const uint32_t maskM = mask_for(m, A.capAB);
    // lanes per cell: the fewest (most cells in flight) while the level has
    // more cells than warps, else 32
    constexpr int GSmin = GatherLanes<D>::min;
    if (GSmin < 32 && m > (nth >> 5))
      phase_update<D, GSmin, BT>(A, t, m, mask, maskM, m_prev, base_prev, base, any_nb, inexact,
                                 werr);
    else
      phase_update<D, 32, BT>(A, t, m, mask, maskM, m_prev, base_prev, base, any_nb, inexact,
                              werr);
    if (__any_sync(kFull, any_nb) && (threadIdx.x & 31) == 0) atomicOr(&A.st[t].has_nb, 1u);
    if (!grid_sync(A.bar, A.fl)) return;
    clk.lap(t == 0 ? kSegUpdateFirst : kSegUpdateRest);
    if (!vst[t].has_nb) {
      converged = true;
      break;
    }
    if (t == A.max_iter) break;
    const uint32_t m1 = vst[t + 1].m;
    phase_compact<D, BT>(A, t, m1, inexact, werr);
    if (tid == 0) {
      A.st[t + 1].mask = maskM;
      A.st[t + 1].base = base + m;
    }
    if (!grid_sync(A.bar, A.fl)) return;
    clk.lap(kSegCompact);
    cell_iters += m;
    m_prev = m;
    base_prev = base;
    base += m;
    m = m1;
    mask = maskM;
    ++t;
  }
  const int T = t;
  const uint32_t k = m;

  // the update of step T is not applied: clear its merge table; every final
  // cell is its own root
  {
    const LevelTable Ms = A.tab[(T + 1) % 3];
    const uint32_t ms = vst[T + 1].m;
    for (uint32_t id = tid; id < ms; id += nth) {
      const uint32_t s = Ms.list[id];
      Ms.key[s] = kEmpty;
      Ms.row[(size_t)s * (D + 1)].x = 0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        uint64_t* acc = Ms.acc + ((size_t)s * D + a) * 4;
        acc[0] = acc[1] = acc[2] = acc[3] = 0;
      }
    }
    for (uint32_t j = tid; j < k; j += nth) A.forest[base + j] = base + j;
    if (BT) {
      // instances still updating stop at step T (converged unless the step
      // limit stopped them with a neighbour present); final cells per instance
      for (uint32_t b = tid; b < (uint32_t)A.B; b += nth) {
        if (!A.I.done[T & 1][b]) {
          A.I.iters[b] = T;
          A.I.conv[b] = A.I.nbf[T & 1][b] ? 0 : 1;
        }
      }
      const Cells c = A.cells[T & 1];
      for (uint32_t j = tid; j < k; j += nth)
        atomicAdd(&A.I.k[(uint32_t)(c.key[j] >> A.P.inst_off)], 1u);
    }
  }
  if (!grid_sync(A.bar, A.fl)) return;
  if (BT && tid == 0) {
    // labels of instance b start at 0: subtract the final cells of earlier ones
    uint32_t run = 0;
    for (int b = 0; b < A.B; ++b) {
      A.I.koff[b] = run;
      run += A.I.k[b];
    }
  }

  // pointer jumping over the forest of merges: after r rounds every node
  // points 2^r levels up (or to its root)
  const uint32_t nodes = base + k;
  uint32_t* in = A.forest;
  uint32_t* out = A.forest2;
  for (int hop = 1; hop < T; hop <<= 1) {
    for (uint32_t v = tid; v < nodes; v += nth) out[v] = in[in[v]];
    if (!grid_sync(A.bar, A.fl)) return;
    uint32_t* tmp = in;
    in = out;
    out = tmp;
  }
  if (in != A.forest) {
    for (uint32_t v = tid; v < m0; v += nth) A.forest[v] = in[v];
    if (!grid_sync(A.bar, A.fl)) return;
  }

  const bool numbered = k <= A.rank_max;
  if (numbered) {
    // label of a final cell = number of final keys below its key (keys are
    // unique), i.e. ascending lexicographic order of the integer keys
    const Cells c = A.cells[T & 1];
    const uint32_t warp = tid >> 5, nwarps = nth >> 5;
    const int lane = threadIdx.x & 31;
    for (uint32_t r = warp; r < k; r += nwarps) {
      const uint64_t kr = c.key[r];
      uint32_t below = 0;
      for (uint32_t q = lane; q < k; q += 32) below += c.key[q] < kr ? 1u : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(kFull, below, o);
      if (lane == 0) A.rank[r] = below;
    }
    if (!grid_sync(A.bar, A.fl)) return;
    for (uint32_t cc = tid; cc < m0; cc += nth) {
      const uint32_t r = A.forest[cc] - base;
      uint32_t label = A.rank[r];
      if (BT) label -= A.I.koff[(uint32_t)(c.key[r] >> A.P.inst_off)];
      A.labslot[A.T0.list[cc]] = label;
    }
    if (!grid_sync(A.bar, A.fl)) return;
    for (int64_t i = tid; i < A.n; i += nth) A.labels[i] = (int32_t)A.labslot[A.slot0[i]];
    const LevelTable G = A.tab[T % 3];
    const bool write = (int64_t)k <= A.modes_cap;
    for (uint32_t r = tid; r < k; r += nth)
      mode_and_release<D>(G, A.P, r, A.rank[r], A.modes, write, inexact);
  }
  clk.lap(kSegLabels);
  if (tid == 0) {
    A.res->iterations = T;
    A.res->converged = converged ? 1 : 0;
    A.res->k = k;
    A.res->base = base;
    A.res->need_sort = numbered ? 0u : 1u;
    A.res->cell_iters = cell_iters;
#pragma unroll
    for (int i = 0; i < kLoopPhases; ++i) A.res->ns[i] = clk.ns[i];
  }
  if (inexact) atomicAdd(&A.fl->inexact, 1ull);
  if (werr) atomicOr(&A.fl->err, kErrWindow);
}

// Labels and modes when the final cells were too many to number inside
// k_loop (after a radix sort of their keys has filled rank[]).
// Batched runs (koff != null) number each instance's clusters from 0.
__global__ void k_labslot_tail(const uint32_t* __restrict__ list0,
                               const uint32_t* __restrict__ root,
                               const uint32_t* __restrict__ rank, uint32_t baseT,
                               uint32_t* __restrict__ labslot, uint32_t m0,
                               const uint64_t* __restrict__ fkey,
                               const uint32_t* __restrict__ koff, int inst_off) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m0; c += gridDim.x * blockDim.x) {
    const uint32_t r = root[c] - baseT;
    uint32_t label = rank[r];
    if (koff) label -= koff[(uint32_t)(fkey[r] >> inst_off)];
    labslot[list0[c]] = label;
  }
}

__global__ void k_labels_tail(const uint32_t* __restrict__ slot0,
                              const uint32_t* __restrict__ labslot, int32_t* __restrict__ labels,
                              int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    labels[i] = (int32_t)labslot[slot0[i]];
}

template <int D>
__global__ void k_modes_tail(LevelTable G, Plan P, const uint32_t* __restrict__ rank,
                             double* __restrict__ modes, uint32_t k, bool write) {
  unsigned inexact = 0;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x)
    mode_and_release<D>(G, P, r, rank[r], modes, write, inexact);
}

__global__ void k_iota_keys(Cells c, uint64_t* keys, uint32_t* vals, uint32_t k) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x) {
    keys[r] = c.key[r];
    vals[r] = r;
  }
}

__global__ void k_rank(const uint32_t* __restrict__ sorted_vals, uint32_t* __restrict__ rank,
                       uint32_t k) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
    rank[sorted_vals[p]] = p;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers

cudaError_t launch_range(const void* pts, bool f32, int64_t n, int d, DevFlags* fl,
                         cudaStream_t s) {
  const bool vec = ((uintptr_t)pts & 15u) == 0;
  const int W = vec ? (f32 ? 4 : 2) : 1;
  const unsigned g = grid_for(n * d / W, kBlock * 4, 152u * 8u);
  if (f32) {
    if (vec) {
      GS_DISPATCH_D(d, k_range<D, float, 4><<<g, kBlock, 0, s>>>((const float*)pts, n, fl));
    } else {
      GS_DISPATCH_D(d, k_range<D, float, 1><<<g, kBlock, 0, s>>>((const float*)pts, n, fl));
    }
  } else {
    if (vec) {
      GS_DISPATCH_D(d, k_range<D, double, 2><<<g, kBlock, 0, s>>>((const double*)pts, n, fl));
    } else {
      GS_DISPATCH_D(d, k_range<D, double, 1><<<g, kBlock, 0, s>>>((const double*)pts, n, fl));
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_bin(const void* pts, bool f32, int64_t n, const Plan& P, const int64_t* thr,
                       BinTable T0, uint32_t mask0, uint32_t maxcells, uint32_t* slot0,
                       DevFlags* fl, const int64_t* offsets, int B, cudaStream_t s) {
  const unsigned g = grid_for((n + 31) / 32 * 32, kBlock, 152u * 6u);
  const bool vec_ok = ((uintptr_t)pts & 15u) == 0;
  if (f32) {
    GS_DISPATCH_D(P.d, k_bin<D, float><<<g, kBlock, 0, s>>>((const float*)pts, n, P, thr, T0,
                                                            mask0, maxcells, slot0, fl, vec_ok,
                                                            offsets, B));
  } else {
    GS_DISPATCH_D(P.d, k_bin<D, double><<<g, kBlock, 0, s>>>((const double*)pts, n, P, thr, T0,
                                                             mask0, maxcells, slot0, fl, vec_ok,
                                                             offsets, B));
  }
  return cudaGetLastError();
}

namespace {
template <int D>
int loop_grid_d() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const int smem = (int)(kFilterWords * sizeof(uint32_t));
  if (cudaFuncSetAttribute(k_loop<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_loop<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
          cudaSuccess)
    return -1;
  int per_sm_b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_loop<D, true>, kLoopBlock, smem) !=
      cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_loop<D, false>, kLoopBlock, smem) !=
      cudaSuccess)
    return -1;
  if (per_sm_b < per_sm) per_sm = per_sm_b;  // one grid size serves both variants
  if (per_sm < 1) return -1;
  if (per_sm > 2) per_sm = 2;  // fewer blocks make the grid barriers cheaper
  const int g = sms * per_sm;
  return g < kMaxLoopGrid ? g : kMaxLoopGrid;
}
}  // namespace

int loop_grid(int d) {
  switch (d) {
    case 1: return loop_grid_d<1>();
    case 2: return loop_grid_d<2>();
    case 3: return loop_grid_d<3>();
    case 4: return loop_grid_d<4>();
    case 5: return loop_grid_d<5>();
    case 6: return loop_grid_d<6>();
    case 7: return loop_grid_d<7>();
    case 8: return loop_grid_d<8>();
  }
  return -1;
}

cudaError_t launch_loop(const LoopArgs& a, int grid, cudaStream_t s) {
  LoopArgs args = a;
  void* params[] = {&args};
  const size_t smem = kFilterWords * sizeof(uint32_t);
  if (a.B > 1) {
    GS_DISPATCH_D(a.P.d, return cudaLaunchCooperativeKernel((const void*)k_loop<D, true>,
                                                            dim3(grid), dim3(kLoopBlock), params,
                                                            smem, s));
  }
  GS_DISPATCH_D(a.P.d, return cudaLaunchCooperativeKernel((const void*)k_loop<D, false>, dim3(grid),
                                                          dim3(kLoopBlock), params, smem, s));
  return cudaSuccess;
}

cudaError_t launch_iota_keys(Cells c, uint64_t* keys, uint32_t* vals, uint32_t k,
                             cudaStream_t s) {
  k_iota_keys<<<grid_for(k), kBlock, 0, s>>>(c, keys, vals, k);
  return cudaGetLastError();
}

cudaError_t launch_rank(const uint32_t* sorted_vals, uint32_t* rank, uint32_t k,
                        cudaStream_t s) {
  k_rank<<<grid_for(k), kBlock, 0, s>>>(sorted_vals, rank, k);
  return cudaGetLastError();
}

cudaError_t launch_label_tail(const LoopArgs& a, uint32_t m0, uint32_t k, uint32_t baseT, int T,
                              cudaStream_t s) {
  const bool bt = a.B > 1;
  k_labslot_tail<<<grid_for(m0), kBlock, 0, s>>>(a.T0.list, a.forest, a.rank, baseT, a.labslot,
                                                 m0, a.cells[T & 1].key,
                                                 bt ? a.I.koff : nullptr, a.P.inst_off);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_labels_tail<<<grid_for(a.n), kBlock, 0, s>>>(a.slot0, a.labslot, a.labels, a.n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // modes (if they fit) and release of the final level's table
  const bool write = (int64_t)k <= a.modes_cap;
  GS_DISPATCH_D(a.P.d, k_modes_tail<D><<<grid_for(k), kBlock, 0, s>>>(a.tab[T % 3], a.P, a.rank,
                                                                       a.modes, k, write));
  return cudaGetLastError();
}

}  // namespace gs
