// gs_loop.cuh -- the loop kernel of the GridShift hot path (Kumar et al.,
// arXiv 2206.02200, Sec. 2.1 and Algorithm 1): one cooperative launch for
// everything between the first binning pass and the labels:
//   binning, second pass: exact cell sums through a counting sort of the
//            points by cell (step i)
//   level 0: the initial cells and their table
//   per update step t:
//     update   steps ii-iv: Eq. 1-2 over the 3^d neighbours in the parallel
//              form (Eq. 6), centroid, new key, and the neighbour test of
//              step v; the count-weighted centroid merged (Eq. 3-4) into the
//              slot of the new key
//     compact  the next level's cells and sums
//   then the forest of merges (the union of resident sets of Eq. 4) is
//   resolved by pointer jumping, the final cells are numbered by ascending
//   key, and every point gets its label.
// Phases are separated by a software grid barrier whose waits are bounded in
// time.  Included by gs_loop64.cu (exact sums rounded once to float64) and
// gs_loop32.cu (the float32 mixed-precision variant), which instantiate it.
#pragma once

#include "gs_common.cuh"

namespace gs {

namespace {

// The plan of the call (DevFlags::plan), copied into shared memory by every
// block of the loop kernel at its start.
__shared__ Plan g_plan;

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

// Device-clock split of the loop kernel, kept by thread 0 of block 0.
struct SegClock {
  unsigned long long last = 0;
  unsigned long long ns[kLoopPhases] = {};
  bool on = false;
  __device__ void start() {
    on = blockIdx.x == 0 && threadIdx.x == 0;
    if (on) last = global_ns();
  }
  __device__ void lap(int seg) { lap_step(seg, -1, nullptr); }
  // also records the lap in step[t] (update steps t < kClockSteps; col 0 the
  // update phase, col 1 the compaction)
  __device__ void lap_step(int seg, int t, LoopResult* res) {
    if (!on) return;
    const unsigned long long now = global_ns();
    ns[seg] += now - last;
    if (res && t >= 0 && t < kClockSteps) res->step_ns[t][seg == kSegCompact ? 1 : 0] = now - last;
    last = now;
  }
};


// This thread's first item of a grid-stride loop over `items` items.  With
// at least as many items as threads, consecutive threads take consecutive
// items (coalesced); with fewer, consecutive items go to consecutive blocks
// (so to different SMs) and the loop spreads over the whole grid instead of
// filling the first blocks.  Either way a bijection of the grid's threads.
__device__ __forceinline__ uint32_t item_tid(uint32_t items) {
  return items >= gridDim.x * blockDim.x ? blockIdx.x * blockDim.x + threadIdx.x
                                         : threadIdx.x * gridDim.x + blockIdx.x;
}

// The same for groups of GS consecutive lanes of a warp.
template <int GS>
__device__ __forceinline__ uint32_t item_group(uint32_t items) {
  return items >= gridDim.x * (blockDim.x / GS) ? (blockIdx.x * blockDim.x + threadIdx.x) / GS
                                                : (threadIdx.x / GS) * gridDim.x + blockIdx.x;
}

__device__ __forceinline__ u128 as_u128(ulonglong2 v) { return (u128)v.x | ((u128)v.y << 64); }

__device__ __forceinline__ ulonglong2 pack(u128 v) {
  return make_ulonglong2((uint64_t)v, (uint64_t)(v >> 64));
}

// The cell sum of one axis as the float64 value of Sec. 2.1 (the exact sum in
// the limb accumulators rounded once), held as the fixed-point integer it
// equals; clears the accumulators.
__device__ __forceinline__ ulonglong2 settle_sum(uint64_t* acc, int L, unsigned& inexact,
                                                 unsigned& werr) {
  (void)inexact;
  const u128 v = round_to_double(limbs_value(acc), L, werr);
  acc[0] = acc[1] = acc[2] = acc[3] = 0;
  return pack(v);
}

// ---------------------------------------------------------------------------
// Occupancy filter of a level: one bit per hashed key (a Bloom filter with
// one hash function), 2^B bits with 2^B >= 32 m (at most 2^kFilterLog2Max).  A
// neighbour probe whose bit is clear cannot hit and never leaves the SM: the
// update phase copies the level's filter into shared memory first.

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

// Capacity mask of a level table that receives at most m distinct keys, at
// load <= 2^-shift where cap_max allows.
__device__ __forceinline__ uint32_t level_mask(uint32_t m, uint32_t cap_max, uint32_t shift) {
  uint64_t c = 64;
  while (c < ((uint64_t)m << shift) && c < cap_max) c <<= 1;
  return (uint32_t)c - 1u;
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
    if (id < hi) {
      A.T0.off[slot] = run + before + x - v;
      A.T0.id[slot] = id;
    }
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

// Adds V into the sum accumulators of the cell of id `id` (they are indexed
// by the cell's id, so the initial cells' sums are dense).
template <int D>
__device__ __forceinline__ void add_cell_sum(const LoopArgs& A, uint32_t id, const u128 (&V)[D]) {
#pragma unroll
  for (int a = 0; a < D; ++a) atomic_add_fixed(A.T0.acc + ((size_t)id * D + a) * 4, V[a]);
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
    // the row of each point (a bandwidth sweep's instances share the points)
    uint32_t src[E];
#pragma unroll
    for (int e = 0; e < E; ++e) src[e] = A.n0 && idx[e] != kNone ? idx[e] % A.n0 : idx[e];
    uint64_t raw[E][D];
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int a = 0; a < D; ++a)
        raw[e][a] = idx[e] != kNone ? load_bits<T>(pts + (size_t)src[e] * D + a) : 0ull;
    // the cells' ids, loaded while the coordinates are in flight
    uint32_t cid[E];
#pragma unroll
    for (int e = 0; e < E; ++e) cid[e] = s[e] != kNone ? A.T0.id[s[e]] : 0u;
    // runs within the lane
    uint32_t cur = s[0], curid = cid[0];
    u128 V[D];
#pragma unroll
    for (int a = 0; a < D; ++a) V[a] = to_fixed(raw[0][a], g_plan.L[a], inexact, werr);
#pragma unroll
    for (int e = 1; e < E; ++e) {
      if (s[e] != cur) {
        if (cur != kNone) add_cell_sum<D>(A, curid, V);
        cur = s[e];
        curid = cid[e];
#pragma unroll
        for (int a = 0; a < D; ++a) V[a] = 0;
      }
#pragma unroll
      for (int a = 0; a < D; ++a) V[a] += to_fixed(raw[e][a], g_plan.L[a], inexact, werr);
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
    if (head && cur != kNone) add_cell_sum<D>(A, curid, V);
  }
}

// Level 0: the cells binning created (in arrival order), their sums rounded
// once, in the level table tab[0].  Resets the binning table's slots.
template <int D>
__device__ void phase_level0(const LoopArgs& A, uint32_t m0, uint32_t maskA, unsigned& inexact,
                             unsigned& werr) {
  const uint32_t tid = item_tid(m0);
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
        r[1 + a] = settle_sum(T0.acc + ((size_t)id * D + a) * 4, g_plan.L[a], inexact, werr);
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

// ---------------------------------------------------------------------------
// The pencil form of the first update step.  The 3^d-neighbour sums of Eq. 1
// are sums over v_0 in {-1,0,1} inside sums over the other d - 1 axes, so
// they are taken in two passes: first, for every position q of the level-0
// cells dilated by one cell along axis 0 (the pencil set Q), the count and
// the coordinate sums of the up to three cells q - e_0, q, q + e_0; then, per
// cell, the sum of those over its 3^(d-1) offsets with v_0 = 0.  The sums are
// exact integers, so the result is the direct sum's, in about a third of the
// probes.  Q lives in tab[2] (free during step 0) with its slots listed in
// qlist, and its keys join the level-0 occupancy filter.

// The least level-0 cells for the pencil form is Tuning::pencil_min (by
// default 4096: below it the two extra grid barriers cost more than the
// probes they save).

// Field of axis a of a packed key (plain runs: nothing above axis 0).
__device__ __forceinline__ int64_t key_field(uint64_t key, int a) {
  const int w = (a == 0 ? 64 : g_plan.off[a - 1]) - g_plan.off[a];
  const uint64_t f = key >> g_plan.off[a];
  return (int64_t)(w >= 64 ? f : (f & ((1ull << w) - 1ull)));
}

// Keys of a pencil set: every key of the source (n keys: skey[i], or
// skey[via[i]]) and its two neighbours along `axis`, where that axis's field
// stays in [1, span] (the only positions the update probes); each new key is
// listed in dlist (count in *dcount) and joins the level-0 filter.
__device__ __forceinline__ void pencil_keys_into(const LoopArgs& A, int axis, const uint64_t* skey,
                                                 const uint32_t* via, uint32_t n, uint64_t* dkey,
                                                 uint32_t dmask, uint32_t* dlist, uint32_t* dcount,
                                                 int lg0) {
  const uint32_t tid = item_tid(3 * n);
  const uint32_t nth = gridDim.x * blockDim.x;
  const uint64_t e = 1ull << g_plan.off[axis];
  for (uint32_t w = tid; w < 3 * n; w += nth) {
    const uint32_t i = w / 3;
    const uint32_t u = w - 3 * i;  // 0, 1, 2: offsets -1, 0, +1
    const uint64_t key = via ? skey[via[i]] : skey[i];
    const int64_t f = key_field(key, axis) + (int64_t)u - 1;
    if (f < 1 || f > g_plan.span[axis]) continue;
    const uint64_t q = key + (u == 0 ? (uint64_t)0 - e : u == 2 ? e : 0ull);
    bool won;
    const uint32_t sl = table_insert(dkey, dmask, q, won, &A.fl->err);
    if (sl != kNone && won) {
      dlist[atomicAdd(dcount, 1u)] = sl;
      if (u != 1) filter_set(A.filter[0], q, lg0);
    }
  }
}

// Stage 1: Q (tab[2], listed in qlist) from the level-0 cells along axis 0.
template <int D>
__device__ void phase_pencil_keys(const LoopArgs& A, uint32_t m0, uint32_t maskQ) {
  pencil_keys_into(A, 0, A.cells[0].key, nullptr, m0, A.tab[2].key, maskQ, A.qlist, &A.st[0].qn,
                   filter_log2(m0));
}

// Stage 2: Q2 (ptab, listed in ptab.list) from Q along axis 1.
template <int D>
__device__ void phase_pencil_keys2(const LoopArgs& A, uint32_t qn, uint32_t m0, uint32_t maskQ2) {
  pencil_keys_into(A, 1, A.tab[2].key, A.qlist, qn, A.ptab.key, maskQ2, A.ptab.list,
                   &A.st[0].qn2, filter_log2(m0));
}

// Count and coordinate sums of the three entries q - e, q, q + e (e along
// `axis`) of the source table, for every q listed in dlist, into the row of q
// in the destination table (the layout of a level row).
template <int D>
__device__ void pencil_sums_into(int axis, const uint32_t* dlist, uint32_t n, const LevelTable& dst,
                                 const LevelTable& src, uint32_t smask) {
  const uint32_t tid = item_tid(n);
  const uint32_t nth = gridDim.x * blockDim.x;
  const uint64_t e = 1ull << g_plan.off[axis];
  for (uint32_t j = tid; j < n; j += nth) {
    const uint32_t sl0 = dlist[j];
    const uint64_t q = dst.key[sl0];
    // the field stays in [1, span] (the key arithmetic then never borrows
    // or carries out of it)
    const int64_t f = key_field(q, axis);
    const uint64_t keys[3] = {q - e, q, q + e};
    const bool valid[3] = {f >= 2, f >= 1 && f <= g_plan.span[axis], f + 1 <= g_plan.span[axis]};
    uint32_t sl[3];
    table_find_many<3>(src.key, smask, keys, valid, sl);
    uint64_t cnt = 0;
    u128 N[D];
#pragma unroll
    for (int a = 0; a < D; ++a) N[a] = 0;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (sl[u] == kNone) continue;
      const ulonglong2* r = src.row + (size_t)sl[u] * (D + 1);
      cnt += r[0].x;
#pragma unroll
      for (int a = 0; a < D; ++a) N[a] += as_u128(r[1 + a]);
    }
    ulonglong2* r = dst.row + (size_t)sl0 * (D + 1);
    r[0] = make_ulonglong2(cnt, 0ull);
#pragma unroll
    for (int a = 0; a < D; ++a) r[1 + a] = pack(N[a]);
  }
}

template <int D>
__device__ void phase_pencil_sums(const LoopArgs& A, uint32_t qn, uint32_t maskA) {
  pencil_sums_into<D>(0, A.qlist, qn, A.tab[2], A.tab[0], maskA);
}

template <int D>
__device__ void phase_pencil_sums2(const LoopArgs& A, uint32_t qn2, uint32_t maskQ) {
  pencil_sums_into<D>(1, A.ptab.list, qn2, A.ptab, A.tab[2], maskQ);
}

// A pencil table back to clean (keys empty, counts zero) once step 0 has
// read it.
template <int D>
__device__ void pencil_release(const LevelTable& Q, const uint32_t* list, uint32_t n) {
  const uint32_t tid = item_tid(n);
  const uint32_t nth = gridDim.x * blockDim.x;
  // four list entries loaded before any store, so their loads overlap
  for (uint32_t j = tid; j < n; j += 4 * nth) {
    uint32_t sl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) sl[k] = j + k * nth < n ? list[j + k * nth] : kNone;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (sl[k] == kNone) continue;
      Q.key[sl[k]] = kEmpty;
      Q.row[(size_t)sl[k] * (D + 1)].x = 0;
    }
  }
}

// Parity colour of a packed key (the sequential update's sweep order):
// bit D-1-a is k_a mod 2, where the field of axis a holds k_a - kmin_a + 1.
template <int D>
__device__ __forceinline__ uint32_t key_colour(uint64_t key) {
  uint32_t c = 0;
#pragma unroll
  for (int a = 0; a < D; ++a)
    c = 2u * c + (uint32_t)((key_field(key, a) - 1 + g_plan.kmin[a]) & 1);
  return c;
}

// Whether the neighbour at probe p (offset digits v_a + 1 in base 3, axis
// D-1 the fastest) of a cell of colour col has a lower colour: its parity
// differs from the cell's exactly on the axes with v_a != 0.
template <int D>
__device__ __forceinline__ bool colour_before(int p, uint32_t col) {
  uint32_t nz = 0;
#pragma unroll
  for (int a = D - 1; a >= 0; --a) {
    nz |= (uint32_t)(p % 3 != 1) << (D - 1 - a);
    p /= 3;
  }
  return (col ^ nz) < col;
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
// With pen = 1 (step 0 only) the sums over the 3^d neighbours are taken as
// sums over the 3^(d-1) offsets with v_0 = 0 of the pencil table tab[2]
// (mask `mask`), each entry of which already holds the three cells along
// axis 0; with pen = 2 over the 3^(d-2) offsets with v_0 = v_1 = 0 of the
// second pencil table (nine cells per entry).  A neighbour v != 0 is present
// iff D exceeds the cell's own count.
// With SEQ (the sequential update of Eq. 5, plain FP64 runs, pen = 0) the
// phase is the pass of parity colour col: only the cells of that colour
// are updated, a neighbour of a lower colour (updated in an earlier pass of
// this step) contributes its count times its new centroid from A.srow, and
// each updated cell leaves that product in A.srow at its slot of level t.
// The filter load and the links of level t-1 happen in the step's first pass
// only (first).
template <int D, int GS, bool BT, bool SEQ = false>
__device__ void phase_update(const LoopArgs& A, int t, uint32_t m, uint32_t mask, uint32_t maskM,
                             uint32_t m_prev, uint32_t base_prev, uint32_t base, bool& any_nb,
                             unsigned& inexact, unsigned& werr, int pen = 0, int col = 0,
                             const uint32_t* sel = nullptr, uint32_t nsel = 0,
                             bool first = true) {
  static_assert(!(SEQ && BT), "the sequential update runs on plain runs only");
  constexpr int U = ProbeBatch<D, GS>::value > 2 ? 2 : ProbeBatch<D, GS>::value;
  const int lane = threadIdx.x & 31;
  const int glane = lane & (GS - 1);
  const unsigned gmask = GS == 32 ? kFull : (((1u << GS) - 1u) << (lane & ~(GS - 1)));
  // sequential passes update the nsel cells of colour col listed in sel
  const uint32_t items = SEQ ? nsel : m;
  const uint32_t group = item_group<GS>(items);
  const uint32_t ngroups = (gridDim.x * blockDim.x) / GS;
  const LevelTable G = A.tab[t % 3];
  const LevelTable P = pen == 2 ? A.ptab : A.tab[pen == 1 ? 2 : t % 3];  // the table probed
  const LevelTable M = A.tab[(t + 1) % 3];
  const Cells c = A.cells[t & 1];
  uint32_t* pslot = A.pslot[t & 1];
  // probes pbase .. pbase + np - 1 of the offset table (axes 0, 1 the slowest
  // digits: v_0 = 0 is its middle third, v_0 = v_1 = 0 that third's middle)
  const int np = g_plan.nprobe / (pen == 2 ? 9 : pen == 1 ? 3 : 1);
  const int pbase = pen == 2 ? 4 * np : pen == 1 ? np : 0;
  // the level's occupancy filter, into shared memory; the filter of level
  // t-1 is cleared for level t+1
  extern __shared__ uint4 s_dyn[];
  uint32_t* s_filter = reinterpret_cast<uint32_t*>(s_dyn);
  const int lg = filter_log2(m);
  if (!SEQ || first) {
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
  for (uint32_t q = group; q < items; q += ngroups) {
    const uint32_t j = SEQ ? sel[q] : q;
    const uint64_t key = c.key[j];
    const uint32_t cj = c.cnt[j];
    // batched runs: a cell of an instance that has stopped is carried to the
    // next level unchanged (same key, its own exact sum)
    uint32_t inst = 0;
    bool live = true;
    if (BT) {
      inst = (uint32_t)(key >> g_plan.inst_off);
      live = A.I.done[t & 1][inst] == 0;
    }
    uint32_t Dc = 0;
    u128 N[D];
#pragma unroll
    for (int a = 0; a < D; ++a) N[a] = 0;
    for (int p0 = glane; live && p0 < np; p0 += GS * U) {
      uint64_t q[U];
      bool v[U];
      uint32_t sl[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = p0 + u * GS;
        q[u] = key + (p < np ? __ldg(&A.dtab[pbase + p]) : 0ull);
        const uint32_t fb = filter_bit(q[u], lg);
        v[u] = p < np && (!A.tune.filter || ((s_filter[fb >> 5] >> (fb & 31)) & 1u));
      }
      table_find_many<U>(P.key, mask, q, v, sl);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (sl[u] == kNone) continue;
        const ulonglong2* r = P.row + (size_t)sl[u] * (D + 1);
        Dc += (uint32_t)r[0].x;
        // sequential passes: a neighbour of a lower colour has its new value
        const ulonglong2* src = r + 1;
        if (SEQ && col > 0 && colour_before<D>(p0 + u * GS, (uint32_t)col))
          src = A.srow + (size_t)sl[u] * D;
#pragma unroll
        for (int a = 0; a < D; ++a) N[a] += as_u128(src[a]);
      }
    }
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
    // a neighbour other than the cell itself (counts are at least 1)
    const bool nbc = live && Dc > cj;
    any_nb = any_nb || nbc;
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
      float inv_h = g_plan.inv_h;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a == glane) {
          Na = N[a];
          La = g_plan.L[a];
          off = g_plan.off[a];
          span = g_plan.span[a];
          toff = g_plan.thr_off[a];
          kmin = g_plan.kmin[a];
        }
      if (BT && A.sweep) {
        // bandwidth sweep: the cell decision of this instance's h
        const SweepPlan* S = A.sweep + inst;
        span = __ldg(&S->span[glane]);
        toff = __ldg(&S->thr_off[glane]);
        kmin = __ldg(&S->kmin[glane]);
        inv_h = __ldg(&S->inv_h);
      }
      const double sv = div_round(Na, Dc, La, inexact);
      const int idx = key_index(A.thr + toff, span, kmin, inv_h, bits_of(sv));
      field = (uint64_t)(idx + 1) << off;
      V = to_fixed(bits_of(sv), La, inexact, werr);
    }
    if (!BT || live) {
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1) field |= __shfl_xor_sync(gmask, field, o);
      if (BT) field |= (key >> g_plan.inst_off) << g_plan.inst_off;  // the instance field
    }
    const bool nbg = BT && nbc;
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
    // sequential passes: what the later colours read for this cell
    if (SEQ && glane < D) A.srow[(size_t)G.list[j] * D + glane] = pack(V * (u128)mult);
  }
  if (t > 0 && (!SEQ || first)) {
    // level t-1: parent links, then its table is released
    const uint32_t tid = item_tid(m_prev);
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
  const uint32_t tid = item_tid(m1);
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
      const uint32_t inst = (uint32_t)(key >> g_plan.inst_off);
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
        r[1 + a] = settle_sum(M.acc + ((size_t)s * D + a) * 4, g_plan.L[a], inexact, werr);
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

// ---------------------------------------------------------------------------
// The float32 mixed-precision variant (GS_FP32_MIXED).  A cell row holds the
// resident count and, per axis, the mean offset of its residents from the
// cell's lower face (count-normalised, float32):
//   row32[s * (d + 1)]      count (uint32)
//   row32[s * (d + 1) + 1 + a]  float32 bits of the mean offset along axis a
// Sums are kept as float-float pairs (hi + lo, compensated additions);
// merges and binning add their partial sums with float32 atomics.  A
// centroid that falls within kFaceBand * h of a face of its cell is
// recomputed from the same float32 state in float64 and its key decided
// against the face table, since that decision sets merges and labels; a
// recomputed centroid less than kTieBand * h below a face counts as a tie and
// goes to the upper cell, as an exact tie does in the exact path.

constexpr float kFaceBand = 1e-5f;
constexpr float kTieBand = 4e-6f;  // below the state error bound of the float32 path

// Float-float number hi + lo with |lo| <= ulp(hi) / 2.
struct FF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float b) {  // Knuth's TwoSum, then renormalise
    const float s = hi + b;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (b - bb);
    const float l = lo + err;
    hi = s + l;
    lo = l - (hi - s);
  }
  __device__ __forceinline__ void add(const FF& o) {
    const float s = hi + o.hi;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (o.hi - bb);
    const float l = lo + o.lo + err;
    hi = s + l;
    lo = l - (hi - s);
  }
  __device__ __forceinline__ float value() const { return hi + lo; }
};

// Kahan-compensated sum: s holds the sum, c the (negated) low part lost so far.
struct KS {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ FF ff() const {
    FF r;
    r.hi = s;
    r.lo = 0.f;
    r.add(-c);
    return r;
  }
};

__device__ __forceinline__ FF shfl_xor_ff(unsigned mask, const FF& v, int o) {
  FF r;
  r.hi = __shfl_xor_sync(mask, v.hi, o);
  r.lo = __shfl_xor_sync(mask, v.lo, o);
  return r;
}

// Lower face (least double >= q h) of the cell with packed key `key` along
// axis a, from the face table.
__device__ __forceinline__ double face_of(const Plan& P, const int64_t* __restrict__ thr,
                                          uint64_t key, int a) {
  const int top = a == 0 ? P.inst_off : P.off[a - 1];
  const uint64_t fmask = (1ull << (top - P.off[a])) - 1ull;
  const int idx = (int)((key >> P.off[a]) & fmask) - 1;
  const int64_t o = __ldg(&thr[P.thr_off[a] + idx]);
  return __longlong_as_double((long long)(o ^ ((o >> 63) & 0x7FFFFFFFFFFFFFFFll)));
}

// ---------------------------------------------------------------------------
// Float32 level tables keep the key inside the row: a probe reads the whole
// row (key, count, offsets) with one load and checks the key afterwards.
// Row words: [key low, key high, count, offset of axis 0, ...], padded to
// RowW<D> words (16, 32 or 64 bytes, so a row never straddles more sectors
// than it must).  A free row has key 0 (packed keys are never 0: every field
// is at least 1).  Linear probing from the key's home slot.

template <int D>
struct RowW {
  static constexpr int value = D + 3 <= 4 ? 4 : (D + 3 <= 8 ? 8 : 16);
  static constexpr int loads = (D + 3 + 3) / 4;  // 16-byte words holding key, count, offsets
};

constexpr uint32_t kMaxRowProbe = 4 * kMaxProbeBuckets;  // slots

__device__ __forceinline__ uint64_t row_key(uint4 w0) {
  return (uint64_t)w0.x | ((uint64_t)w0.y << 32);
}

// Word i (a constant after unrolling) of a row held as 16-byte words.
template <int N>
__device__ __forceinline__ uint32_t row_word(const uint4 (&w)[N], int i) {
  const uint4 v = w[i >> 2];
  const int j = i & 3;
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// Slot of key in the rows (mask = slots - 1), inserting it if absent; won is
// set for the inserting thread.  kNone (and kErrTableFull) when no free row
// lies within kMaxRowProbe slots.
template <int W>
__device__ __forceinline__ uint32_t row_insert(uint32_t* rows, uint32_t mask, uint64_t key,
                                               bool& won, uint32_t* err) {
  uint32_t s = home_bucket(key, mask);
  won = false;
  const uint32_t lim = mask < kMaxRowProbe ? mask + 1 : kMaxRowProbe;
  for (uint32_t i = 0; i < lim; ++i) {
    unsigned long long* kp = reinterpret_cast<unsigned long long*>(rows + (size_t)s * W);
    const uint64_t k = __ldcg(kp);
    if (k == key) return s;
    if (k == 0) {
      const uint64_t prev = atomicCAS(kp, 0ull, (unsigned long long)key);
      if (prev == 0) {
        won = true;
        return s;
      }
      if (prev == key) return s;
    }
    s = (s + 1) & mask;
  }
  atomicOr(err, kErrTableFull);
  return kNone;
}

// Lookups of U keys at once: the home rows of all of them are loaded before
// any is examined; dat receives the row of each key found.
template <int D, int U>
__device__ __forceinline__ void row_find_many(const uint32_t* rows, uint32_t mask,
                                              const uint64_t (&key)[U], const bool (&valid)[U],
                                              uint32_t (&slot)[U],
                                              uint4 (&dat)[U][RowW<D>::loads]) {
  constexpr int W = RowW<D>::value, NL = RowW<D>::loads;
  uint32_t s[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    s[u] = home_bucket(key[u], mask);
    if (valid[u]) {
      const uint4* r = reinterpret_cast<const uint4*>(rows + (size_t)s[u] * W);
#pragma unroll
      for (int i = 0; i < NL; ++i) dat[u][i] = r[i];
    }
  }
  const uint32_t lim = mask < kMaxRowProbe ? mask + 1 : kMaxRowProbe;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    slot[u] = kNone;
    if (!valid[u]) continue;
    uint64_t k = row_key(dat[u][0]);
    uint32_t sl = s[u];
    for (uint32_t i = 1; k != key[u] && k != 0 && i < lim; ++i) {
      sl = (sl + 1) & mask;
      const uint4* r = reinterpret_cast<const uint4*>(rows + (size_t)sl * W);
#pragma unroll
      for (int j = 0; j < NL; ++j) dat[u][j] = r[j];
      k = row_key(dat[u][0]);
    }
    if (k == key[u]) slot[u] = sl;
  }
}

// Slot of key (single lookup), or kNone.
template <int D>
__device__ __forceinline__ uint32_t row_find(const uint32_t* rows, uint32_t mask, uint64_t key) {
  constexpr int W = RowW<D>::value;
  uint32_t s = home_bucket(key, mask);
  const uint32_t lim = mask < kMaxRowProbe ? mask + 1 : kMaxRowProbe;
  for (uint32_t i = 0; i < lim; ++i) {
    const uint64_t k = *reinterpret_cast<const unsigned long long*>(rows + (size_t)s * W);
    if (k == key) return s;
    if (k == 0) return kNone;
    s = (s + 1) & mask;
  }
  return kNone;
}

__device__ __forceinline__ void row_release(uint32_t* r) {
  *reinterpret_cast<unsigned long long*>(r) = 0ull;
  r[2] = 0;
}

// Binning, second pass (float32): each cell's sum of offsets from its lower
// face, over the runs of the counting sort (as phase_cell_sums).
template <int D, typename T>
__device__ void phase_cell_sums32(const LoopArgs& A) {
  constexpr int E = kSumRun;
  const T* __restrict__ pts = static_cast<const T*>(A.pts);
  float* __restrict__ tacc = reinterpret_cast<float*>(A.T0.acc);
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
    float x[E][D];
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int a = 0; a < D; ++a)
        x[e][a] = idx[e] != kNone ? (float)__ldg(pts + (size_t)idx[e] * D + a) : 0.f;
    // the cells' ids and keys, loaded while the coordinates are in flight
    uint32_t cid[E];
    uint64_t ckey[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      cid[e] = s[e] != kNone ? A.T0.id[s[e]] : 0u;
      ckey[e] = s[e] != kNone ? A.T0.key[s[e]] : 0ull;
    }
    uint32_t cur = kNone, curid = 0;
    float org[D];
    FF V[D];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (s[e] != cur) {
        if (cur != kNone) {
#pragma unroll
          for (int a = 0; a < D; ++a) atomicAdd(&tacc[(size_t)curid * D + a], V[a].value());
        }
        cur = s[e];
        curid = cid[e];
        if (cur != kNone) {
#pragma unroll
          for (int a = 0; a < D; ++a) org[a] = (float)face_of(g_plan, A.thr, ckey[e], a);
        }
#pragma unroll
        for (int a = 0; a < D; ++a) V[a] = FF();
      }
      if (cur != kNone) {
#pragma unroll
        for (int a = 0; a < D; ++a) V[a].add(x[e][a] - org[a]);
      }
    }
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
          FF w;
          w.hi = __shfl_down_sync(kFull, V[a].hi, o);
          w.lo = __shfl_down_sync(kFull, V[a].lo, o);
          if (lane + o < end) V[a].add(w);
        }
      }
    }
    if (head && cur != kNone) {
#pragma unroll
      for (int a = 0; a < D; ++a) atomicAdd(&tacc[(size_t)curid * D + a], V[a].value());
    }
  }
}

// Level 0 (float32): mean offsets of the initial cells; resets the binning
// table's slots.
template <int D>
__device__ void phase_level0_32(const LoopArgs& A, uint32_t m0, uint32_t maskA) {
  const uint32_t tid = item_tid(m0);
  const uint32_t nth = gridDim.x * blockDim.x;
  const BinTable T0 = A.T0;
  float* tacc = reinterpret_cast<float*>(T0.acc);
  const LevelTable G = A.tab[0];
  uint32_t* row = reinterpret_cast<uint32_t*>(G.row);
  constexpr int W = RowW<D>::value;
  const Cells c = A.cells[0];
  const int lg0 = filter_log2(m0);
  for (uint32_t id = tid; id < m0; id += nth) {
    const uint32_t s = T0.list[id];
    const uint64_t key = T0.key[s];
    const uint32_t cnt = T0.cnt[s];
    bool won;
    const uint32_t sa = row_insert<W>(row, maskA, key, won, &A.fl->err);
    if (sa != kNone) {
      uint32_t* r = row + (size_t)sa * W;
      r[2] = cnt;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        r[3 + a] = __float_as_uint(tacc[(size_t)id * D + a] / (float)cnt);
        tacc[(size_t)id * D + a] = 0.f;
      }
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

// The pencil form of step 0 in float32 (as phase_pencil_keys and
// phase_pencil_sums): Q's rows hold the key, the count of the up to three
// cells q - e_0, q, q + e_0, and their count-weighted mean offset from q's
// lower face.
template <int D>
__device__ __forceinline__ void pencil_keys_into32(const LoopArgs& A, int axis,
                                                   const uint32_t* srows, const uint64_t* skey,
                                                   const uint32_t* via, uint32_t n,
                                                   uint32_t* drows, uint32_t dmask,
                                                   uint32_t* dlist, uint32_t* dcount, int lg0) {
  constexpr int W = RowW<D>::value;
  const uint32_t tid = item_tid(3 * n);
  const uint32_t nth = gridDim.x * blockDim.x;
  const uint64_t e = 1ull << g_plan.off[axis];
  for (uint32_t w = tid; w < 3 * n; w += nth) {
    const uint32_t i = w / 3;
    const uint32_t u = w - 3 * i;  // 0, 1, 2: offsets -1, 0, +1
    const uint64_t key =
        srows ? *reinterpret_cast<const unsigned long long*>(srows + (size_t)via[i] * W) : skey[i];
    const int64_t f = key_field(key, axis) + (int64_t)u - 1;
    if (f < 1 || f > g_plan.span[axis]) continue;
    const uint64_t q = key + (u == 0 ? (uint64_t)0 - e : u == 2 ? e : 0ull);
    bool won;
    const uint32_t sl = row_insert<W>(drows, dmask, q, won, &A.fl->err);
    if (sl != kNone && won) {
      dlist[atomicAdd(dcount, 1u)] = sl;
      if (u != 1) filter_set(A.filter[0], q, lg0);
    }
  }
}

template <int D>
__device__ void phase_pencil_keys32(const LoopArgs& A, uint32_t m0, uint32_t maskQ) {
  pencil_keys_into32<D>(A, 0, nullptr, A.cells[0].key, nullptr, m0,
                        reinterpret_cast<uint32_t*>(A.tab[2].row), maskQ, A.qlist, &A.st[0].qn,
                        filter_log2(m0));
}

template <int D>
__device__ void phase_pencil_keys2_32(const LoopArgs& A, uint32_t qn, uint32_t m0, uint32_t maskQ2) {
  pencil_keys_into32<D>(A, 1, reinterpret_cast<const uint32_t*>(A.tab[2].row), nullptr, A.qlist,
                        qn, reinterpret_cast<uint32_t*>(A.ptab.row), maskQ2, A.ptab.list,
                        &A.st[0].qn2, filter_log2(m0));
}

// The count of the three entries q - e, q, q + e of the source rows and their
// count-weighted mean offset from q's lower face.
template <int D>
__device__ void pencil_sums_into32(int axis, const uint32_t* dlist, uint32_t n, uint32_t* drows,
                                   const uint32_t* srows, uint32_t smask) {
  constexpr int W = RowW<D>::value, NL = RowW<D>::loads;
  const uint32_t tid = item_tid(n);
  const uint32_t nth = gridDim.x * blockDim.x;
  const uint64_t e = 1ull << g_plan.off[axis];
  const float h = g_plan.h32;
  for (uint32_t j = tid; j < n; j += nth) {
    uint32_t* r = drows + (size_t)dlist[j] * W;
    const uint64_t q = *reinterpret_cast<const unsigned long long*>(r);
    const int64_t f = key_field(q, axis);
    const uint64_t keys[3] = {q - e, q, q + e};
    const bool valid[3] = {f >= 2, f >= 1 && f <= g_plan.span[axis], f + 1 <= g_plan.span[axis]};
    uint32_t sl[3];
    uint4 dat[3][NL];
    row_find_many<D, 3>(srows, smask, keys, valid, sl, dat);
    uint32_t cnt = 0;
    KS S[D];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (sl[u] == kNone) continue;
      const uint32_t cn = row_word(dat[u], 2);
      const float fc = (float)cn;
      cnt += cn;
#pragma unroll
      for (int a = 0; a < D; ++a)
        S[a].add(fc * (__uint_as_float(row_word(dat[u], 3 + a)) +
                       (a == axis ? (float)((int)u - 1) * h : 0.f)));
    }
    const float fC = (float)cnt;
    r[2] = cnt;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const FF v = S[a].ff();
      r[3 + a] = __float_as_uint(v.hi / fC + v.lo / fC);
    }
  }
}

template <int D>
__device__ void phase_pencil_sums32(const LoopArgs& A, uint32_t qn, uint32_t maskA) {
  pencil_sums_into32<D>(0, A.qlist, qn, reinterpret_cast<uint32_t*>(A.tab[2].row),
                        reinterpret_cast<const uint32_t*>(A.tab[0].row), maskA);
}

template <int D>
__device__ void phase_pencil_sums2_32(const LoopArgs& A, uint32_t qn2, uint32_t maskQ) {
  pencil_sums_into32<D>(1, A.ptab.list, qn2, reinterpret_cast<uint32_t*>(A.ptab.row),
                        reinterpret_cast<const uint32_t*>(A.tab[2].row), maskQ);
}

template <int D>
__device__ void pencil_release32(const LevelTable& Q, const uint32_t* list, uint32_t n) {
  constexpr int W = RowW<D>::value;
  const uint32_t tid = item_tid(n);
  const uint32_t nth = gridDim.x * blockDim.x;
  uint32_t* qrow = reinterpret_cast<uint32_t*>(Q.row);
  for (uint32_t j = tid; j < n; j += 4 * nth) {
    uint32_t sl[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) sl[k] = j + k * nth < n ? list[j + k * nth] : kNone;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (sl[k] != kNone) row_release(qrow + (size_t)sl[k] * W);
  }
}

// One update step t (float32), as phase_update: Eq. 1-2 over the neighbours
// in float-float, centroid relative to the cell's lower face, new key, and
// the count-weighted centroid merged (Eq. 3-4) relative to the new cell's
// lower face.  A centroid within kFaceBand * h of a face is recomputed in
// float64 from the same neighbours and its key decided exactly.  With pen
// (step 0 only) the neighbour sums come from the pencil rows of tab[2] (mask
// maskQ) over the 3^(d-1) offsets with v_0 = 0; the float64 recheck still
// reads the level's own rows.
template <int D, int GS, bool BT>
__device__ void phase_update32(const LoopArgs& A, int t, uint32_t m, uint32_t mask,
                               uint32_t maskM, uint32_t m_prev, uint32_t base_prev,
                               uint32_t base, bool& any_nb, int pen = 0,
                               uint32_t maskQ = 0) {
  constexpr int U = ProbeBatch<D, GS>::value > 2 ? 2 : ProbeBatch<D, GS>::value;
  constexpr int W = RowW<D>::value, NL = RowW<D>::loads;
  const int lane = threadIdx.x & 31;
  const int glane = lane & (GS - 1);
  const unsigned gmask = GS == 32 ? kFull : (((1u << GS) - 1u) << (lane & ~(GS - 1)));
  const uint32_t group = item_group<GS>(m);
  const uint32_t ngroups = (gridDim.x * blockDim.x) / GS;
  const LevelTable G = A.tab[t % 3];
  const LevelTable M = A.tab[(t + 1) % 3];
  const uint32_t* grow = reinterpret_cast<const uint32_t*>(G.row);
  // the rows the neighbour sums read: the level's, or the pencil rows
  const uint32_t* prow = reinterpret_cast<const uint32_t*>(
      (pen == 2 ? A.ptab : A.tab[pen == 1 ? 2 : t % 3]).row);
  const uint32_t maskP = pen ? maskQ : mask;
  uint32_t* mrow = reinterpret_cast<uint32_t*>(M.row);  // rows with the key inside (RowW)
  float* macc = reinterpret_cast<float*>(M.acc);
  const Cells c = A.cells[t & 1];
  uint32_t* pslot = A.pslot[t & 1];
  const int nprobe = g_plan.nprobe;
  // probes pbase .. pbase + np - 1 of the offset table (as phase_update)
  const int np = nprobe / (pen == 2 ? 9 : pen == 1 ? 3 : 1);
  const int pbase = pen == 2 ? 4 * np : pen == 1 ? np : 0;
  const float h = g_plan.h32;
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
    uint32_t inst = 0;
    bool live = true;
    if (BT) {
      inst = (uint32_t)(key >> g_plan.inst_off);
      live = A.I.done[t & 1][inst] == 0;
    }
    uint32_t Dc = 0;
    KS Nk[D];
    for (int p0 = glane; live && p0 < np; p0 += GS * U) {
      uint64_t q[U];
      bool v[U];
      uint32_t sl[U];
      uint4 dat[U][NL];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = p0 + u * GS;
        q[u] = key + (p < np ? __ldg(&A.dtab[pbase + p]) : 0ull);
        const uint32_t fb = filter_bit(q[u], lg);
        v[u] = p < np && (!A.tune.filter || ((s_filter[fb >> 5] >> (fb & 31)) & 1u));
      }
      row_find_many<D, U>(prow, maskP, q, v, sl, dat);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (sl[u] == kNone) continue;
        const int p = p0 + u * GS;
        const uint32_t cn = row_word(dat[u], 2);
        const float fc = (float)cn;
        Dc += cn;
        // the probe's offset v in {-1, 0, 1}^d: 2 bits per axis, v_a + 1
        const uint32_t vp = __ldg(&A.vpack[pbase + p]);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const float dv = (float)((int)((vp >> (2 * a)) & 3u) - 1);
          Nk[a].add(fc * (__uint_as_float(row_word(dat[u], 3 + a)) + dv * h));
        }
      }
    }
    FF N[D];
#pragma unroll
    for (int a = 0; a < D; ++a) N[a] = Nk[a].ff();
#pragma unroll
    for (int o = GS / 2; o > 0; o >>= 1) {
      Dc += __shfl_xor_sync(gmask, Dc, o);
#pragma unroll
      for (int a = 0; a < D; ++a) N[a].add(shfl_xor_ff(gmask, N[a], o));
    }
    // float-float additions are not symmetric in their low parts: every lane
    // of the group takes the first lane's sums, so all take the same decisions
#pragma unroll
    for (int a = 0; a < D; ++a) {
      N[a].hi = __shfl_sync(gmask, N[a].hi, 0, GS);
      N[a].lo = __shfl_sync(gmask, N[a].lo, 0, GS);
    }
    // a neighbour other than the cell itself (counts are at least 1)
    const bool nbc = live && Dc > cj;
    any_nb = any_nb || nbc;
    // centroid relative to the lower face; move q_a in {-1, 0, 1} per axis
    uint64_t field = 0;
    float rel[D];
    bool near = false;
    if (BT && !live) {
      field = key;
#pragma unroll
      for (int a = 0; a < D; ++a) rel[a] = 0.f;
    } else {
      const float fD = (float)Dc;
      uint64_t nk = key;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        rel[a] = N[a].hi / fD + N[a].lo / fD;
        const int qa = rel[a] < 0.f ? -1 : (rel[a] >= h ? 1 : 0);
        near = near || fabsf(rel[a]) < kFaceBand * h || fabsf(rel[a] - h) < kFaceBand * h;
        nk += (uint64_t)(int64_t)qa << g_plan.off[a];
      }
      field = nk;
    }
    if (near) {
      // float64 recheck: the same neighbours, upcast, summed in float64 about
      // the cell's lower face; the key of N / D decided on the face table
      double N64[D];
#pragma unroll
      for (int a = 0; a < D; ++a) N64[a] = 0.0;
      double org[D];
#pragma unroll
      for (int a = 0; a < D; ++a) org[a] = (double)(float)face_of(g_plan, A.thr, key, a);
      for (int p = glane; p < nprobe; p += GS) {
        const uint64_t qk = key + __ldg(&A.dtab[p]);
        const uint32_t sl = row_find<D>(grow, mask, qk);
        if (sl == kNone) continue;
        const uint32_t* r = grow + (size_t)sl * W;
        const double cn = (double)r[2];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const double of = (double)(float)face_of(g_plan, A.thr, qk, a);
          N64[a] += cn * ((of - org[a]) + (double)__uint_as_float(r[3 + a]));
        }
      }
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < D; ++a) N64[a] += __shfl_xor_sync(gmask, N64[a], o);
      uint64_t nk = (key >> g_plan.inst_off) << g_plan.inst_off;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const double xa = org[a] + N64[a] / (double)Dc;
        const int64_t* thr = A.thr + g_plan.thr_off[a];
        int idx = key_index(thr, g_plan.span[a], g_plan.kmin[a], g_plan.inv_h,
                            (uint64_t)__double_as_longlong(xa));
        // a centroid this close below a face is taken to lie on it: the
        // float32 state cannot tell such a value from an exact tie, which the
        // exact path assigns to the upper cell
        if (idx + 1 < g_plan.span[a]) {
          const int64_t o = __ldg(&thr[idx + 1]);
          const double fnext =
              __longlong_as_double((long long)(o ^ ((o >> 63) & 0x7FFFFFFFFFFFFFFFll)));
          if (fnext - xa < (double)kTieBand * (double)h) ++idx;
        }
        nk |= (uint64_t)(idx + 1) << g_plan.off[a];
        // the centroid relative to its own cell's lower face, in float32
        rel[a] = (float)(xa - org[a]);
      }
      field = nk;
      if (glane == 0) atomicAdd(&A.fl->rechecks, 1ull);
    }
    const bool nbg = BT && nbc;
    uint32_t ms = kNone;
    if (glane == 0) {
      bool won;
      ms = row_insert<W>(mrow, maskM, field, won, &A.fl->err);
      if (ms != kNone) {
        if (won) {
          const uint32_t id = atomicAdd(&A.st[t + 1].m, 1u);
          M.list[id] = ms;
          if (BT) M.id[ms] = j;
        }
        atomicAdd(&mrow[(size_t)ms * W + 2], cj);
      }
      pslot[j] = ms;
      if (BT && live) {
        if (nbg && !A.I.nbf[t & 1][inst]) atomicOr(&A.I.nbf[t & 1][inst], 1u);
        atomicAdd(&A.I.mt[t & 1][inst], 1u);
      }
    }
    ms = __shfl_sync(gmask, ms, 0, GS);
    if (glane < D && ms != kNone) {
      // this cell's count-weighted centroid about the new cell's lower face
      float contrib = 0.f;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (a != glane) continue;
        if (BT && !live) {
          contrib = (float)cj * __uint_as_float(grow[(size_t)G.list[j] * W + 3 + a]);
        } else {
          const int top = a == 0 ? g_plan.inst_off : g_plan.off[a - 1];
          const uint64_t fm = (1ull << (top - g_plan.off[a])) - 1ull;
          const int qa = (int)((field >> g_plan.off[a]) & fm) - (int)((key >> g_plan.off[a]) & fm);
          contrib = (float)cj * (rel[a] - (float)qa * h);
        }
      }
      atomicAdd(&macc[(size_t)ms * D + glane], contrib);
    }
  }
  if (t > 0) {
    const uint32_t tid = item_tid(m_prev);
    const uint32_t nth = gridDim.x * blockDim.x;
    const LevelTable Lp = A.tab[(t + 2) % 3];
    uint32_t* prow = reinterpret_cast<uint32_t*>(Lp.row);
    const uint32_t* pp = A.pslot[(t - 1) & 1];
    for (uint32_t i = tid; i < m_prev; i += nth) {
      A.forest[base_prev + i] = base + G.id[pp[i]];
      row_release(prow + (size_t)Lp.list[i] * W);
    }
  }
}

// The cells of level t+1 (float32): mean offsets = merged sums / counts.
template <int D, bool BT>
__device__ void phase_compact32(const LoopArgs& A, int t, uint32_t m1) {
  const uint32_t tid = item_tid(m1);
  const uint32_t nth = gridDim.x * blockDim.x;
  const LevelTable G = A.tab[t % 3];
  const LevelTable M = A.tab[(t + 1) % 3];
  constexpr int W = RowW<D>::value;
  const uint32_t* grow = reinterpret_cast<const uint32_t*>(G.row);
  uint32_t* mrow = reinterpret_cast<uint32_t*>(M.row);
  float* macc = reinterpret_cast<float*>(M.acc);
  const Cells cur = A.cells[t & 1];
  const Cells nx = A.cells[(t + 1) & 1];
  uint32_t* f = A.filter[(t + 1) & 1];
  const int lg = filter_log2(m1);
  for (uint32_t id = tid; id < m1; id += nth) {
    const uint32_t s = M.list[id];
    uint32_t* r = mrow + (size_t)s * W;
    uint64_t key = *reinterpret_cast<const unsigned long long*>(r);
    const uint32_t cnt = r[2];
    bool restored = false;
    if (BT) {
      const uint32_t inst = (uint32_t)(key >> g_plan.inst_off);
      if (!A.I.done[t & 1][inst] && !A.I.nbf[t & 1][inst]) {
        const uint32_t j = M.id[s];
        const uint32_t* o = grow + (size_t)G.list[j] * W;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          r[3 + a] = o[3 + a];
          macc[(size_t)s * D + a] = 0.f;
        }
        key = cur.key[j];
        restored = true;
      }
    }
    if (!restored) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        r[3 + a] = __float_as_uint(macc[(size_t)s * D + a] / (float)cnt);
        macc[(size_t)s * D + a] = 0.f;
      }
    }
    nx.key[id] = key;
    nx.cnt[id] = cnt;
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

// Mode of final cell r (float32 state): its lower face plus its mean offset,
// in float64; then the slot is released.
template <int D>
__device__ __forceinline__ void mode_and_release32(const LevelTable& G, const Plan& P,
                                                   const int64_t* thr, const uint64_t* keys,
                                                   uint32_t r, uint32_t label, double* modes,
                                                   bool write) {
  const uint32_t s = G.list[r];
  uint32_t* row = reinterpret_cast<uint32_t*>(G.row) + (size_t)s * RowW<D>::value;
  if (write) {
    const uint64_t key = keys[r];
#pragma unroll
    for (int a = 0; a < D; ++a)
      modes[(size_t)label * D + a] =
          (double)(float)face_of(P, thr, key, a) + (double)__uint_as_float(row[3 + a]);
  }
  row_release(row);
}

// ---------------------------------------------------------------------------
// The tail of the update loop in one block (plain runs).  Once a
// level has at most Tuning::tail_enter cells, block 0 copies it into shared memory
// and runs the remaining update steps alone, with block barriers, while the
// other blocks wait at one grid barrier.  With so few cells, neighbours are
// found by comparing every pair of cells (|k_i - k_j| <= 1 on every axis is
// the same test as k_i = k_j + v for some v in {-1,0,1}^d, Eq. 1), and the
// cells sharing a new key by comparing new keys, so no hash table is needed.
// The arithmetic is that of phase_update and phase_compact (exact sums
// rounded once); a merged cell's sum is added over its members.

// Longest run whose labels walk the chain of merges directly (one dependent
// load per step) instead of pointer jumping (one grid barrier per round).
constexpr int kWalkMax = 16;

// Largest level handed to the one-block tail: Tuning::tail_enter.  A tail
// step makes m^2 pair tests on one SM; measured on GB300 (d = 3 and 5), it
// beats a multi-block step (grid barriers, dependent L2 loads) up to about
// 110 cells and loses from about 150 (14 against 20 us at 107 cells, 31
// against 21 us at 149): 128 by default.
constexpr int kTailMax = (int)kTailMaxCells;  // cells the tail's shared memory holds
constexpr int kTailLanes = 8;  // lanes comparing one cell against the level

constexpr size_t tail_bytes(int d, int mx) {
  return (size_t)mx * d * 16 * 3   // sums of two levels; neighbour sums, then centroids
         + (size_t)mx * 8 * 3      // keys of two levels, new keys
         + (size_t)mx * 4 * 3      // counts of two levels, neighbour counts
         + (size_t)mx * d * 4      // key fields of the level (axis-major)
         + (size_t)mx * 2 * 4;     // first member, member count, new id, member of a new id
}

// Shared-memory layout of the tail.  The two levels' arrays are reached by
// offset arithmetic (no runtime-indexed pointer array), so every access stays
// a shared-memory access.
template <int D>
struct TailMem {
  static constexpr int Mx = kTailMax;
  static constexpr size_t kSum = (size_t)Mx * D * 16, kKey = (size_t)Mx * 8,
                          kCnt = (size_t)Mx * 4;
  char* p;
  __device__ explicit TailMem(void* base) : p(static_cast<char*>(base)) {}
  // level c (0 or 1): sums, keys, counts
  __device__ ulonglong2* sum(int c) const { return reinterpret_cast<ulonglong2*>(p + c * kSum); }
  __device__ uint64_t* key(int c) const {
    return reinterpret_cast<uint64_t*>(p + 3 * kSum + c * kKey);
  }
  __device__ uint32_t* cnt(int c) const {
    return reinterpret_cast<uint32_t*>(p + 3 * kSum + 3 * kKey + c * kCnt);
  }
  // neighbour sums, then centroids; new keys; neighbour counts; key fields
  __device__ ulonglong2* V() const { return reinterpret_cast<ulonglong2*>(p + 2 * kSum); }
  __device__ uint64_t* nk() const { return reinterpret_cast<uint64_t*>(p + 3 * kSum + 2 * kKey); }
  __device__ uint32_t* dc() const {
    return reinterpret_cast<uint32_t*>(p + 3 * kSum + 3 * kKey + 2 * kCnt);
  }
  __device__ int32_t* F() const {
    return reinterpret_cast<int32_t*>(p + 3 * kSum + 3 * kKey + 3 * kCnt);
  }
  // first member, member count, new id, first member of a new id
  __device__ uint16_t* u16(int which) const {
    return reinterpret_cast<uint16_t*>(p + 3 * kSum + 3 * kKey + 3 * kCnt + (size_t)Mx * D * 4 +
                                       (size_t)which * Mx * 2);
  }
};
static_assert(kDefaultTuning.tail_enter <= kTailMaxCells &&
                  tail_bytes(kMaxD, kTailMax) <= (size_t)kFilterWords * 4,
              "the tail's shared memory must fit in the filter's");

// Width of axis a's key field (axis 0 most significant).
__device__ __forceinline__ int field_width(const Plan& P, int a) {
  return (a == 0 ? 64 : P.off[a - 1]) - P.off[a];
}

// Result of the tail, published by block 0 for the other blocks.
struct TailOut {
  int t;
  uint32_t m, base;
  int converged;
  unsigned long long cell_iters;
};

// Block 0 only.  Level t (m cells, in table tab[t % 3] and cells[t & 1]) is
// the first level of the tail.  On return level t (the final level) is back
// in tab[t % 3] and cells[t & 1], and the forest holds the parent links of
// every level before it.
template <int D>
__device__ void run_tail(const LoopArgs& A, int t, uint32_t m, uint32_t m_prev,
                         uint32_t base_prev, uint32_t base, unsigned long long cell_iters,
                         SegClock& clk, unsigned& inexact, unsigned& werr, TailOut& out) {
  constexpr int Mx = TailMem<D>::Mx;
  constexpr int GS = kTailLanes;
  extern __shared__ uint4 s_dyn[];
  const TailMem<D> S(s_dyn);
  ulonglong2* const V = S.V();
  uint64_t* const nk = S.nk();
  uint32_t* const dc = S.dc();
  int32_t* const F = S.F();
  uint16_t* const lead = S.u16(0);
  uint16_t* const mcnt = S.u16(1);
  uint16_t* const nid = S.u16(2);
  uint16_t* const lidx = S.u16(3);
  __shared__ uint32_t s_nb, s_wc[kLoopBlock / 32];
  const uint32_t tid = threadIdx.x, nth = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int glane = lane & (GS - 1);
  const uint32_t group = threadIdx.x / GS, ngroups = blockDim.x / GS;

  // parent links of level t-1 and release of its table (the update phase of
  // step t does this in the multi-block path)
  {
    const LevelTable G = A.tab[t % 3];
    if (t > 0) {
      const LevelTable Lp = A.tab[(t + 2) % 3];
      const uint32_t* pp = A.pslot[(t - 1) & 1];
      for (uint32_t i = tid; i < m_prev; i += nth) {
        A.forest[base_prev + i] = base + G.id[pp[i]];
        const uint32_t s = Lp.list[i];
        Lp.key[s] = kEmpty;
        Lp.row[(size_t)s * (D + 1)].x = 0;
      }
    }
    // level t into shared memory; its table is released
    const Cells c = A.cells[t & 1];
    for (uint32_t i = tid; i < m; i += nth) {
      const uint32_t s = G.list[i];
      S.key(0)[i] = c.key[i];
      S.cnt(0)[i] = c.cnt[i];
#pragma unroll
      for (int a = 0; a < D; ++a) S.sum(0)[(size_t)i * D + a] = G.row[(size_t)s * (D + 1) + 1 + a];
      G.key[s] = kEmpty;
      G.row[(size_t)s * (D + 1)].x = 0;
    }
  }
  __syncthreads();

  int cur = 0;
  bool converged = false;
  for (;;) {
    const uint64_t* key = S.key(cur);
    const uint32_t* cnt = S.cnt(cur);
    const ulonglong2* sum = S.sum(cur);
    // the key fields of the level, axis-major
    for (uint32_t i = tid; i < m; i += nth) {
      const uint64_t k = key[i];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int w = field_width(g_plan, a);
        const uint64_t f = k >> g_plan.off[a];
        F[a * Mx + i] = (int32_t)(w >= 64 ? f : (f & ((1ull << w) - 1ull)));
      }
      nk[i] = 0;
    }
    if (tid == 0) s_nb = 0;
    __syncthreads();
    // ii: D and N over the cells within one cell on every axis (Eq. 1-2);
    // GS lanes per cell, each comparing a share of the level
    for (uint32_t j0 = 0; j0 < m; j0 += ngroups) {
      const uint32_t j = j0 + group;
      const bool live = j < m;
      int32_t fj[D];
#pragma unroll
      for (int a = 0; a < D; ++a) fj[a] = live ? F[a * Mx + j] : 0;
      uint32_t Dc = 0;
      bool nb = false;
      u128 N[D];
#pragma unroll
      for (int a = 0; a < D; ++a) N[a] = 0;
      for (uint32_t i = glane; live && i < m; i += GS) {
        bool adj = true;
#pragma unroll
        for (int a = 0; a < D; ++a) adj &= (uint32_t)(F[a * Mx + i] - fj[a] + 1) <= 2u;
        if (adj) {
          Dc += cnt[i];
#pragma unroll
          for (int a = 0; a < D; ++a) N[a] += as_u128(sum[(size_t)i * D + a]);
          if (i != j) nb = true;
        }
      }
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1) {
        Dc += __shfl_xor_sync(kFull, Dc, o);
#pragma unroll
        for (int a = 0; a < D; ++a) N[a] += shfl_xor_u128(N[a], o);
      }
      if (live) {
        if (glane == 0) dc[j] = Dc;
#pragma unroll
        for (int a = 0; a < D; ++a)
          if (a == glane) V[(size_t)j * D + a] = pack(N[a]);
      }
      if (__any_sync(kFull, nb) && lane == 0) s_nb = 1u;
    }
    __syncthreads();
    // ii-iii: one thread per (cell, axis): centroid N / D rounded once, its
    // key field, its fixed-point value
    for (uint32_t w = tid; w < m * D; w += nth) {
      const uint32_t j = w / D;
      const int ax = (int)(w - j * D);
      int La = 0, off = 0, span = 1, toff = 0;
      int64_t kmin = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a == ax) {
          La = g_plan.L[a];
          off = g_plan.off[a];
          span = g_plan.span[a];
          toff = g_plan.thr_off[a];
          kmin = g_plan.kmin[a];
        }
      const double sv = div_round(as_u128(V[w]), dc[j], La, inexact);
      const int idx = key_index(A.thr + toff, span, kmin, g_plan.inv_h, bits_of(sv));
      atomicOr((unsigned long long*)&nk[j], (unsigned long long)(idx + 1) << off);
      V[w] = pack(to_fixed(bits_of(sv), La, inexact, werr));
    }
    __syncthreads();
    clk.lap_step(kSegUpdateRest, t, A.res);
    if (!s_nb) {
      converged = true;
      break;
    }
    if (t == A.max_iter) break;
    // iv: merge.  A cell's first member is the lowest-indexed cell with its
    // new key; new cells are numbered in the order of their first members.
    // GS lanes per cell compare its new key with a share of the level's.
    for (uint32_t j0 = 0; j0 < m; j0 += ngroups) {
      const uint32_t i = j0 + group;
      const bool live = i < m;
      const uint64_t k = live ? nk[i] : 0ull;
      uint32_t l = kNone, c = 0;
      for (uint32_t q = glane; live && q < m; q += GS) {
        if (nk[q] == k) {
          l = min(l, q);
          ++c;
        }
      }
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1) {
        l = min(l, __shfl_xor_sync(kFull, l, o));
        c += __shfl_xor_sync(kFull, c, o);
      }
      if (live && glane == 0) {
        lead[i] = (uint16_t)l;
        mcnt[i] = (uint16_t)c;
      }
    }
    __syncthreads();
    uint32_t m1 = 0;
    {
      uint32_t base_w = 0;
      for (uint32_t i0 = 0; i0 < m; i0 += nth) {
        const uint32_t i = i0 + tid;
        const bool first = i < m && lead[i] == i;
        const unsigned bal = __ballot_sync(kFull, first);
        if (lane == 0) s_wc[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = base_w;
        for (int w = 0; w < warp; ++w) before += s_wc[w];
        if (first) {
          const uint32_t id = before + __popc(bal & ((1u << lane) - 1u));
          nid[i] = (uint16_t)id;
          lidx[id] = (uint16_t)i;
        }
        for (int w = 0; w < (int)(nth >> 5); ++w) base_w += s_wc[w];
        __syncthreads();
      }
      m1 = base_w;
    }
    const int nxtb = cur ^ 1;
    // GS lanes per new cell: the count-weighted sum of its members'
    // centroids (Eq. 3-4), exact, rounded once; a cell alone under its new
    // key is its only member
    for (uint32_t id0 = 0; id0 < m1; id0 += ngroups) {
      const uint32_t id = id0 + group;
      const bool live = id < m1;
      const uint32_t l = live ? lidx[id] : 0u;
      const bool many = live && mcnt[l] > 1;
      uint32_t c1 = 0;
      u128 Sx[D];
#pragma unroll
      for (int a = 0; a < D; ++a) Sx[a] = 0;
      for (uint32_t i = l + glane; live && i < m && (many || i == l); i += GS) {
        if (lead[i] != l) continue;
        const uint32_t ci = cnt[i];
        c1 += ci;
#pragma unroll
        for (int a = 0; a < D; ++a) Sx[a] += as_u128(V[(size_t)i * D + a]) * (u128)ci;
      }
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1) {
        c1 += __shfl_xor_sync(kFull, c1, o);
#pragma unroll
        for (int a = 0; a < D; ++a) Sx[a] += shfl_xor_u128(Sx[a], o);
      }
      if (live && glane < D) {
        u128 Sa = 0;
        int La = 0;
#pragma unroll
        for (int a = 0; a < D; ++a)
          if (a == glane) {
            Sa = Sx[a];
            La = g_plan.L[a];
          }
        S.sum(nxtb)[(size_t)id * D + glane] = pack(round_to_double(Sa, La, werr));
      }
      if (live) {
        if (glane == 0) {
          S.key(nxtb)[id] = nk[l];
          S.cnt(nxtb)[id] = c1;
        }
      }
    }
    for (uint32_t i = tid; i < m; i += nth) A.forest[base + i] = base + m + nid[lead[i]];
    __syncthreads();
    clk.lap_step(kSegCompact, t, A.res);
    cell_iters += m;
    base += m;
    m = m1;
    cur = nxtb;
    ++t;
  }

  // the final level back into its global table and cell list
  {
    const LevelTable G = A.tab[t % 3];
    const Cells c = A.cells[t & 1];
    const uint32_t maskT = level_mask(m, A.capAB, A.tune.load_shift);
    for (uint32_t i = tid; i < m; i += nth) {
      bool won;
      const uint64_t k = S.key(cur)[i];
      const uint32_t s = table_insert(G.key, maskT, k, won, &A.fl->err);
      c.key[i] = k;
      c.cnt[i] = S.cnt(cur)[i];
      if (s == kNone) continue;
      ulonglong2* r = G.row + (size_t)s * (D + 1);
      r[0] = make_ulonglong2((uint64_t)S.cnt(cur)[i], 0ull);
#pragma unroll
      for (int a = 0; a < D; ++a) r[1 + a] = S.sum(cur)[(size_t)i * D + a];
      G.id[s] = i;
      G.list[i] = s;
    }
    if (tid == 0) {
      A.st[t].m = m;
      A.st[t].mask = maskT;
      A.st[t].base = base;
    }
  }
  out.t = t;
  out.m = m;
  out.base = base;
  out.converged = converged ? 1 : 0;
  out.cell_iters = cell_iters;
}

// The one-block tail in float32 (GS_FP32_MIXED, plain runs): run_tail's
// steps with the arithmetic of phase_update32 and phase_compact32.  A cell's
// state is its count and its mean offset from its lower face; neighbour sums
// are Kahan sums of cnt (o + v h) per lane combined as float-float; a centroid
// within kFaceBand * h of a face is recomputed in float64 from the same
// neighbours.  A merged cell's mean is the sum over its members, in member
// order, of cnt (rel - q h), divided by its count.
constexpr size_t tail32_bytes(int d, int mx) {
  return (size_t)mx * d * 4 * 3    // means of two levels, merge contributions
         + (size_t)mx * 8 * 3      // keys of two levels, new keys
         + (size_t)mx * 4 * 2      // counts of two levels
         + (size_t)mx * d * 4      // key fields of the level (axis-major)
         + (size_t)mx * 2 * 4;     // first member, member count, new id, member of a new id
}

template <int D>
struct TailMem32 {
  static constexpr int Mx = kTailMax;
  static constexpr size_t kMean = (size_t)Mx * D * 4, kKey = (size_t)Mx * 8,
                          kCnt = (size_t)Mx * 4;
  char* p;
  __device__ explicit TailMem32(void* base) : p(static_cast<char*>(base)) {}
  __device__ float* mean(int c) const { return reinterpret_cast<float*>(p + c * kMean); }
  __device__ float* contrib() const { return reinterpret_cast<float*>(p + 2 * kMean); }
  __device__ uint64_t* key(int c) const {
    return reinterpret_cast<uint64_t*>(p + 3 * kMean + c * kKey);
  }
  __device__ uint64_t* nk() const { return reinterpret_cast<uint64_t*>(p + 3 * kMean + 2 * kKey); }
  __device__ uint32_t* cnt(int c) const {
    return reinterpret_cast<uint32_t*>(p + 3 * kMean + 3 * kKey + c * kCnt);
  }
  __device__ int32_t* F() const {
    return reinterpret_cast<int32_t*>(p + 3 * kMean + 3 * kKey + 2 * kCnt);
  }
  __device__ uint16_t* u16(int which) const {
    return reinterpret_cast<uint16_t*>(p + 3 * kMean + 3 * kKey + 2 * kCnt + (size_t)Mx * D * 4 +
                                       (size_t)which * Mx * 2);
  }
};
static_assert(tail32_bytes(kMaxD, kTailMax) <= (size_t)kFilterWords * 4,
              "the float32 tail's shared memory must fit in the filter's");

template <int D>
__device__ void run_tail32(const LoopArgs& A, int t, uint32_t m, uint32_t m_prev,
                           uint32_t base_prev, uint32_t base, unsigned long long cell_iters,
                           SegClock& clk, TailOut& out) {
  constexpr int Mx = TailMem32<D>::Mx;
  constexpr int GS = kTailLanes;
  constexpr int W = RowW<D>::value;
  extern __shared__ uint4 s_dyn[];
  const TailMem32<D> S(s_dyn);
  float* const contrib = S.contrib();
  uint64_t* const nk = S.nk();
  int32_t* const F = S.F();
  uint16_t* const lead = S.u16(0);
  uint16_t* const mcnt = S.u16(1);
  uint16_t* const nid = S.u16(2);
  uint16_t* const lidx = S.u16(3);
  __shared__ uint32_t s_nb, s_wc[kLoopBlock / 32];
  const uint32_t tid = threadIdx.x, nth = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int glane = lane & (GS - 1);
  const unsigned gmask = ((1u << GS) - 1u) << (lane & ~(GS - 1));
  const uint32_t group = threadIdx.x / GS, ngroups = blockDim.x / GS;
  const float h = g_plan.h32;

  // parent links of level t-1 and release of its table; level t into shared
  // memory and its table released
  {
    const LevelTable G = A.tab[t % 3];
    uint32_t* grow = reinterpret_cast<uint32_t*>(G.row);
    if (t > 0) {
      const LevelTable Lp = A.tab[(t + 2) % 3];
      uint32_t* prow = reinterpret_cast<uint32_t*>(Lp.row);
      const uint32_t* pp = A.pslot[(t - 1) & 1];
      for (uint32_t i = tid; i < m_prev; i += nth) {
        A.forest[base_prev + i] = base + G.id[pp[i]];
        row_release(prow + (size_t)Lp.list[i] * W);
      }
    }
    const Cells c = A.cells[t & 1];
    for (uint32_t i = tid; i < m; i += nth) {
      uint32_t* r = grow + (size_t)G.list[i] * W;
      S.key(0)[i] = c.key[i];
      S.cnt(0)[i] = c.cnt[i];
#pragma unroll
      for (int a = 0; a < D; ++a) S.mean(0)[(size_t)i * D + a] = __uint_as_float(r[3 + a]);
      row_release(r);
    }
  }
  __syncthreads();

  int cur = 0;
  bool converged = false;
  for (;;) {
    const uint64_t* key = S.key(cur);
    const uint32_t* cnt = S.cnt(cur);
    const float* mean = S.mean(cur);
    for (uint32_t i = tid; i < m; i += nth) {
      const uint64_t k = key[i];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int w = field_width(g_plan, a);
        const uint64_t f = k >> g_plan.off[a];
        F[a * Mx + i] = (int32_t)(w >= 64 ? f : (f & ((1ull << w) - 1ull)));
      }
    }
    if (tid == 0) s_nb = 0;
    __syncthreads();
    // ii-iii: GS lanes per cell compare it with a share of the level
    for (uint32_t j0 = 0; j0 < m; j0 += ngroups) {
      const uint32_t j = j0 + group;
      const bool live = j < m;
      const uint64_t kj = live ? key[j] : 0ull;
      const uint32_t cj = live ? cnt[j] : 0u;
      int32_t fj[D];
#pragma unroll
      for (int a = 0; a < D; ++a) fj[a] = live ? F[a * Mx + j] : 0;
      uint32_t Dc = 0;
      KS Nk[D];
      for (uint32_t i = glane; live && i < m; i += GS) {
        int32_t dv[D];
        bool adj = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          dv[a] = F[a * Mx + i] - fj[a];
          adj &= (uint32_t)(dv[a] + 1) <= 2u;
        }
        if (adj) {
          const uint32_t cn = cnt[i];
          const float fc = (float)cn;
          Dc += cn;
#pragma unroll
          for (int a = 0; a < D; ++a) Nk[a].add(fc * (mean[(size_t)i * D + a] + (float)dv[a] * h));
        }
      }
      FF N[D];
#pragma unroll
      for (int a = 0; a < D; ++a) N[a] = Nk[a].ff();
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1) {
        Dc += __shfl_xor_sync(gmask, Dc, o);
#pragma unroll
        for (int a = 0; a < D; ++a) N[a].add(shfl_xor_ff(gmask, N[a], o));
      }
#pragma unroll
      for (int a = 0; a < D; ++a) {
        N[a].hi = __shfl_sync(gmask, N[a].hi, 0, GS);
        N[a].lo = __shfl_sync(gmask, N[a].lo, 0, GS);
      }
      if (__any_sync(kFull, live && Dc > cj) && lane == 0) s_nb = 1u;
      if (!live) continue;  // the group's lanes take the same branch
      const float fD = (float)Dc;
      float rel[D];
      bool near = false;
      uint64_t field = kj;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        rel[a] = N[a].hi / fD + N[a].lo / fD;
        const int qa = rel[a] < 0.f ? -1 : (rel[a] >= h ? 1 : 0);
        near = near || fabsf(rel[a]) < kFaceBand * h || fabsf(rel[a] - h) < kFaceBand * h;
        field += (uint64_t)(int64_t)qa << g_plan.off[a];
      }
      if (near) {
        // float64 recheck (as phase_update32) over the same neighbours
        double N64[D], org[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          N64[a] = 0.0;
          org[a] = (double)(float)face_of(g_plan, A.thr, kj, a);
        }
        for (uint32_t i = glane; i < m; i += GS) {
          bool adj = true;
#pragma unroll
          for (int a = 0; a < D; ++a) adj &= (uint32_t)(F[a * Mx + i] - fj[a] + 1) <= 2u;
          if (!adj) continue;
          const double cn = (double)cnt[i];
#pragma unroll
          for (int a = 0; a < D; ++a) {
            const double of = (double)(float)face_of(g_plan, A.thr, key[i], a);
            N64[a] += cn * ((of - org[a]) + (double)mean[(size_t)i * D + a]);
          }
        }
#pragma unroll
        for (int o = GS / 2; o > 0; o >>= 1)
#pragma unroll
          for (int a = 0; a < D; ++a) N64[a] += __shfl_xor_sync(gmask, N64[a], o);
        field = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const double xa = org[a] + N64[a] / (double)Dc;
          const int64_t* thr = A.thr + g_plan.thr_off[a];
          int idx = key_index(thr, g_plan.span[a], g_plan.kmin[a], g_plan.inv_h,
                              (uint64_t)__double_as_longlong(xa));
          if (idx + 1 < g_plan.span[a]) {
            const int64_t o = __ldg(&thr[idx + 1]);
            const double fnext =
                __longlong_as_double((long long)(o ^ ((o >> 63) & 0x7FFFFFFFFFFFFFFFll)));
            if (fnext - xa < (double)kTieBand * (double)h) ++idx;
          }
          field |= (uint64_t)(idx + 1) << g_plan.off[a];
          rel[a] = (float)(xa - org[a]);
        }
        if (glane == 0) atomicAdd(&A.fl->rechecks, 1ull);
      }
      if (glane == 0) nk[j] = field;
      // this cell's count-weighted centroid about the new cell's lower face
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (a != glane) continue;
        const int w = field_width(g_plan, a);
        const uint64_t fm = w >= 64 ? ~0ull : (1ull << w) - 1ull;
        const int qa = (int)((field >> g_plan.off[a]) & fm) - (int)((kj >> g_plan.off[a]) & fm);
        contrib[(size_t)j * D + a] = (float)cj * (rel[a] - (float)qa * h);
      }
    }
    __syncthreads();
    clk.lap_step(kSegUpdateRest, t, A.res);
    if (!s_nb) {
      converged = true;
      break;
    }
    if (t == A.max_iter) break;
    // iv: merge (as run_tail): first member = lowest index with the new key
    for (uint32_t j0 = 0; j0 < m; j0 += ngroups) {
      const uint32_t i = j0 + group;
      const bool live = i < m;
      const uint64_t k = live ? nk[i] : 0ull;
      uint32_t l = kNone, c = 0;
      for (uint32_t q = glane; live && q < m; q += GS) {
        if (nk[q] == k) {
          l = min(l, q);
          ++c;
        }
      }
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1) {
        l = min(l, __shfl_xor_sync(kFull, l, o));
        c += __shfl_xor_sync(kFull, c, o);
      }
      if (live && glane == 0) {
        lead[i] = (uint16_t)l;
        mcnt[i] = (uint16_t)c;
      }
    }
    __syncthreads();
    uint32_t m1 = 0;
    {
      uint32_t base_w = 0;
      for (uint32_t i0 = 0; i0 < m; i0 += nth) {
        const uint32_t i = i0 + tid;
        const bool first = i < m && lead[i] == i;
        const unsigned bal = __ballot_sync(kFull, first);
        if (lane == 0) s_wc[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = base_w;
        for (int w = 0; w < warp; ++w) before += s_wc[w];
        if (first) {
          const uint32_t id = before + __popc(bal & ((1u << lane) - 1u));
          nid[i] = (uint16_t)id;
          lidx[id] = (uint16_t)i;
        }
        for (int w = 0; w < (int)(nth >> 5); ++w) base_w += s_wc[w];
        __syncthreads();
      }
      m1 = base_w;
    }
    const int nxtb = cur ^ 1;
    // one thread per (new cell, axis): members in index order
    for (uint32_t w = tid; w < m1 * D; w += nth) {
      const uint32_t id = w / D;
      const int ax = (int)(w - id * D);
      const uint32_t l = lidx[id];
      uint32_t c1 = 0;
      float sx = 0.f;
      if (mcnt[l] > 1) {
        for (uint32_t i = l; i < m; ++i) {
          if (lead[i] != l) continue;
          c1 += cnt[i];
          sx += contrib[(size_t)i * D + ax];
        }
      } else {
        c1 = cnt[l];
        sx = contrib[(size_t)l * D + ax];
      }
      S.mean(nxtb)[w] = sx / (float)c1;
      if (ax == 0) {
        S.key(nxtb)[id] = nk[l];
        S.cnt(nxtb)[id] = c1;
      }
    }
    for (uint32_t i = tid; i < m; i += nth) A.forest[base + i] = base + m + nid[lead[i]];
    __syncthreads();
    clk.lap_step(kSegCompact, t, A.res);
    cell_iters += m;
    base += m;
    m = m1;
    cur = nxtb;
    ++t;
  }

  // the final level back into its global table (float32 rows) and cell list
  {
    const LevelTable G = A.tab[t % 3];
    uint32_t* grow = reinterpret_cast<uint32_t*>(G.row);
    const Cells c = A.cells[t & 1];
    const uint32_t maskT = level_mask(m, A.capAB, A.tune.load_shift);
    for (uint32_t i = tid; i < m; i += nth) {
      bool won;
      const uint64_t k = S.key(cur)[i];
      const uint32_t s = row_insert<W>(grow, maskT, k, won, &A.fl->err);
      c.key[i] = k;
      c.cnt[i] = S.cnt(cur)[i];
      if (s == kNone) continue;
      uint32_t* r = grow + (size_t)s * W;
      r[2] = S.cnt(cur)[i];
#pragma unroll
      for (int a = 0; a < D; ++a) r[3 + a] = __float_as_uint(S.mean(cur)[(size_t)i * D + a]);
      G.id[s] = i;
      G.list[i] = s;
    }
    if (tid == 0) {
      A.st[t].m = m;
      A.st[t].mask = maskT;
      A.st[t].base = base;
    }
  }
  out.t = t;
  out.m = m;
  out.base = base;
  out.converged = converged ? 1 : 0;
  out.cell_iters = cell_iters;
}

// labels[i] = labslot[slot0[i]] for every point.  Where the labels are
// 16-byte aligned, a thread takes two words of four points at once, so eight
// independent gathers are in flight per thread (the loop is bound by the
// latency of those gathers, not by bandwidth).
__device__ __forceinline__ void write_labels(const LoopArgs& A, uint32_t tid, uint32_t nth) {
  int64_t done = 0;
  if (((uintptr_t)A.labels & 15u) == 0) {
    const int64_t n4 = A.n / 4;
    const uint4* __restrict__ s4 = reinterpret_cast<const uint4*>(A.slot0);
    int4* __restrict__ l4 = reinterpret_cast<int4*>(A.labels);
    const uint32_t* __restrict__ ls = A.labslot;
    for (int64_t q = tid; q < n4; q += 2 * (int64_t)nth) {
      const bool two = q + nth < n4;
      const uint4 a = s4[q];
      const uint4 b = two ? s4[q + nth] : make_uint4(0u, 0u, 0u, 0u);
      const int4 la = make_int4((int)ls[a.x], (int)ls[a.y], (int)ls[a.z], (int)ls[a.w]);
      int4 lb = make_int4(0, 0, 0, 0);
      if (two) lb = make_int4((int)ls[b.x], (int)ls[b.y], (int)ls[b.z], (int)ls[b.w]);
      l4[q] = la;
      if (two) l4[q + nth] = lb;
    }
    done = n4 * 4;
  }
  for (int64_t i = done + tid; i < A.n; i += nth) A.labels[i] = (int32_t)A.labslot[A.slot0[i]];
}

// ---------------------------------------------------------------------------
// Step i, second pass, and the final label writes, as ordinary launches
// before and after the loop kernel, for runs of at least Tuning::split_min
// points (smaller runs take them inside the loop kernel, where the launches'
// own latency would cost more than they gain).  They touch every point, and
// their gathers are bound by latency: outside the cooperative kernel (one
// block of 512 threads per SM) they run with as many warps per SM as their
// registers allow.  Each does nothing unless the plan is valid and binning
// fit its table (the same flags every block reads, so the decision is
// uniform).

constexpr int kPrepBlock = 256;
constexpr int kPrepCountGrid = 304;  // blocks of the count and offset launches

__device__ __forceinline__ bool prep_ok(const LoopArgs& A) {
  return A.n >= (int64_t)A.tune.split_min &&
         *(volatile uint32_t*)&A.fl->plan_status == kPlanOK &&
         (*(volatile uint32_t*)&A.fl->err & (kErrOverflow | kErrTableFull)) == 0u;
}

// Per-block totals of the cells' counts, then every cell's run offset
// (phase_count_totals, phase_offsets; both launches kPrepCountGrid blocks).
__global__ void __launch_bounds__(kLoopBlock) k_prep_counts(LoopArgs A) {
  if (!prep_ok(A)) return;
  phase_count_totals(A, *(volatile uint32_t*)&A.fl->m0);
}

__global__ void __launch_bounds__(kLoopBlock) k_prep_offsets(LoopArgs A) {
  if (!prep_ok(A)) return;
  phase_offsets(A, *(volatile uint32_t*)&A.fl->m0);
}

// The points sorted by cell (phase_scatter).
__global__ void __launch_bounds__(kPrepBlock) k_prep_scatter(LoopArgs A) {
  if (!prep_ok(A)) return;
  phase_scatter(A);
}

// The exact (FP64) or float32 cell sums (phase_cell_sums, phase_cell_sums32).
// Three blocks per SM where that costs no spills (the float32 sums, and the
// exact sums up to d = 3), else two (the exact sums' 128-bit partial sums
// need about 110 registers a thread at d = 5; d = 8 spills a little).
template <int D, bool F32>
__global__ void __launch_bounds__(kPrepBlock, (F32 || D <= 3) ? 3 : 2) k_prep_sums(LoopArgs A) {
  if (!prep_ok(A)) return;
  if (threadIdx.x == 0) g_plan = A.fl->plan;
  __syncthreads();
  unsigned inexact = 0, werr = 0;
  if (F32) {
    if (A.f32)
      phase_cell_sums32<D, float>(A);
    else
      phase_cell_sums32<D, double>(A);
  } else {
    if (A.f32)
      phase_cell_sums<D, float>(A, inexact, werr);
    else
      phase_cell_sums<D, double>(A, inexact, werr);
  }
  if (inexact) atomicAdd(&A.fl->inexact, 1ull);
  if (werr) atomicOr(&A.fl->err, kErrWindow);
}

// Every point's label, once the loop kernel has numbered the final cells
// (LoopResult::labels_ready; with too many clusters the radix-sort path
// writes them instead).
__global__ void __launch_bounds__(kPrepBlock) k_labels_out(LoopArgs A) {
  if (!*(volatile uint32_t*)&A.res->labels_ready) return;
  write_labels(A, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// The loop kernel.  SEQ: the sequential update of Eq. 5 (plain FP64 runs;
// A.srow holds the shifted rows), a separate instantiation so that the
// parallel kernels carry none of its code.
template <int D, bool BT, bool F32, bool SEQ = false>
__global__ void __launch_bounds__(kLoopBlock, 1) k_loop(LoopArgs A) {
  static_assert(!(SEQ && (BT || F32)), "the sequential update runs on plain FP64 runs only");
  unsigned inexact = 0, werr = 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nth = gridDim.x * blockDim.x;
  volatile IterState* vst = A.st;
  SegClock clk;
  clk.start();

  // no valid plan (the host reads the status), or binning overflowed its
  // table (the host regrows it and runs binning and this kernel again):
  // nothing to do
  if (*(volatile uint32_t*)&A.fl->plan_status != kPlanOK) return;
  if (threadIdx.x == 0) g_plan = A.fl->plan;
  __syncthreads();
  if (*(volatile uint32_t*)&A.fl->err & (kErrOverflow | kErrTableFull)) {
    if (tid == 0) A.res->bin_failed = 1;
    return;
  }

  // a value above the fixed-point window in the exact sums (k_prep_sums):
  // the host reports it
  if (*(volatile uint32_t*)&A.fl->err) return;

  // the sequential update's colour counts and cursors start at zero
  if constexpr (SEQ) {
    if (tid < 512) A.seq_aux[tid] = 0;
  }
  const uint32_t m0 = *(volatile uint32_t*)&A.fl->m0;
  // step i, second pass (the exact cell sums): in the k_prep_* launches
  // before this kernel when the run has split_min points or more, else here
  const bool split = A.n >= (int64_t)A.tune.split_min;
  if (!split) {
    phase_count_totals(A, m0);
    if (!grid_sync(A.bar, A.fl)) return;
    phase_offsets(A, m0);
    if (!grid_sync(A.bar, A.fl)) return;
    clk.lap(kSegOffsets);
    phase_scatter(A);
    if (!grid_sync(A.bar, A.fl)) return;
    clk.lap(kSegScatter);
    if (F32) {
      if (A.f32)
        phase_cell_sums32<D, float>(A);
      else
        phase_cell_sums32<D, double>(A);
    } else {
      if (A.f32)
        phase_cell_sums<D, float>(A, inexact, werr);
      else
        phase_cell_sums<D, double>(A, inexact, werr);
    }
    if (!grid_sync(A.bar, A.fl)) return;
    clk.lap(kSegSums);
  }

  // level 0
  const uint32_t maskA = level_mask(m0, A.capAB, A.tune.load_shift);
  if (tid == 0) {
    A.st[0].m = m0;
    A.st[0].mask = maskA;
    A.st[0].base = 0;
  }
  if (F32)
    phase_level0_32<D>(A, m0, maskA);
  else
    phase_level0<D>(A, m0, maskA, inexact, werr);
  if (BT) {
    // the same threads as phase_level0 (no barrier between): each reads the
    // keys it wrote
    for (uint32_t id = item_tid(m0); id < m0; id += nth)
      atomicAdd(&A.I.m0[(uint32_t)(A.cells[0].key[id] >> g_plan.inst_off)], 1u);
  }
  if (!grid_sync(A.bar, A.fl)) return;
  clk.lap(kSegLevel0);

  // the pencil form of step 0 (plain runs with enough cells): stage 1 along
  // axis 0 into tab[2]; from d = 6, where the second pencil table has room
  // for three times stage 1's positions at load 1/2, stage 2 along axis 1
  // (measured on GB300: at d = 5 building stage 2 costs more than the 27
  // probes per cell it saves; at d = 6 it saves 81 of 243)
  int pen = 0;
  uint32_t maskQ = 0, qn = 0, maskQ2 = 0, qn2 = 0;
  // the sequential update: colour passes of the generic update at every
  // level, no pencil form, no one-block tail
  constexpr bool seq = SEQ;
  if constexpr (!BT && D >= 3) {
    // Q holds at most 3 m0 keys: only where tab[2] keeps them at load <= 3/4
    if (!seq && m0 > A.tune.tail_enter && m0 >= A.tune.pencil_min && A.qlist != nullptr &&
        4ull * m0 <= (uint64_t)A.capAB) {
      pen = 1;
      maskQ = mask_for(3 * m0, A.capAB);
      if (F32)
        phase_pencil_keys32<D>(A, m0, maskQ);
      else
        phase_pencil_keys<D>(A, m0, maskQ);
      if (!grid_sync(A.bar, A.fl)) return;
      qn = vst[0].qn;
      if (D >= kPencil2MinD && A.ptab.cap != 0 && 6ull * qn <= (uint64_t)A.ptab.cap) {
        pen = 2;
        maskQ2 = mask_for(3 * qn, A.ptab.cap);
      }
      // stage 1's sums and stage 2's keys (which need only stage 1's keys)
      if (F32) {
        phase_pencil_sums32<D>(A, qn, maskA);
        if (pen == 2) phase_pencil_keys2_32<D>(A, qn, m0, maskQ2);
      } else {
        phase_pencil_sums<D>(A, qn, maskA);
        if (pen == 2) phase_pencil_keys2<D>(A, qn, m0, maskQ2);
      }
      if (!grid_sync(A.bar, A.fl)) return;
      if (pen == 2) {
        qn2 = vst[0].qn2;
        if (F32)
          phase_pencil_sums2_32<D>(A, qn2, maskQ);
        else
          phase_pencil_sums2<D>(A, qn2, maskQ);
        if (!grid_sync(A.bar, A.fl)) return;
      }
      clk.lap(kSegUpdateFirst);
    }
  }

  int t = 0;
  uint32_t m = m0, mask = maskA, base = 0, m_prev = 0, base_prev = 0;
  unsigned long long cell_iters = 0;
  bool converged = false;
  for (;;) {
    if constexpr (!BT) {
      // a small level: block 0 finishes the update steps in shared memory
      if (m <= A.tune.tail_enter && !seq) {
        if (blockIdx.x == 0) {
          TailOut to;
          if constexpr (F32)
            run_tail32<D>(A, t, m, m_prev, base_prev, base, cell_iters, clk, to);
          else
            run_tail<D>(A, t, m, m_prev, base_prev, base, cell_iters, clk, inexact, werr, to);
          if (threadIdx.x == 0) {
            A.res->tail_t = to.t;
            A.res->tail_m = to.m;
            A.res->tail_base = to.base;
            A.res->tail_conv = to.converged;
            A.res->tail_cells = to.cell_iters;
          }
        }
        if (!grid_sync(A.bar, A.fl)) return;
        volatile LoopResult* vr = A.res;
        t = vr->tail_t;
        m = vr->tail_m;
        base = vr->tail_base;
        converged = vr->tail_conv != 0;
        cell_iters = vr->tail_cells;
        break;
      }
    }
    bool any_nb = false;
    const uint32_t maskM = level_mask(m, A.capAB, A.tune.load_shift);
    // lanes per cell: the fewest (most cells in flight) while the level has
    // more cells than warps, else 32
    constexpr int GSmin = GatherLanes<D>::min;
    const bool few_lanes = 4ull * m > (uint64_t)A.tune.few_lanes_x4 * (nth >> 5);
    const int pt = t == 0 ? pen : 0;
    const uint32_t maskPt = pt == 2 ? maskQ2 : maskQ;
    if (F32) {
      if (GSmin < 32 && few_lanes)
        phase_update32<D, GSmin, BT>(A, t, m, mask, maskM, m_prev, base_prev, base, any_nb, pt,
                                     maskPt);
      else
        phase_update32<D, 32, BT>(A, t, m, mask, maskM, m_prev, base_prev, base, any_nb, pt,
                                  maskPt);
    } else if constexpr (SEQ) {
      // Eq. 5: the colours one after another, each reading the ones before.
      // The level's cells are first listed by colour (counts, offsets, then
      // a scatter into colour order), so a pass reads only its own cells and
      // an empty colour costs neither a pass nor a barrier.
      constexpr int NC = 1 << D;
      uint32_t* const chist = A.seq_aux;          // NC counts (zero here)
      uint32_t* const ccur = A.seq_aux + 256;     // NC cursors (zero here)
      uint32_t* const corder = A.seq_aux + 512;   // the cells in colour order
      __shared__ uint32_t s_coff[NC + 1];
      for (uint32_t j = tid; j < m; j += nth) atomicAdd(&chist[key_colour<D>(A.cells[t & 1].key[j])], 1u);
      if (!grid_sync(A.bar, A.fl)) return;
      if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int q = 0; q < NC; ++q) {
          s_coff[q] = run;
          run += __ldcg(&chist[q]);
        }
        s_coff[NC] = run;
      }
      __syncthreads();
      for (uint32_t j = tid; j < m; j += nth) {
        const uint32_t cl = key_colour<D>(A.cells[t & 1].key[j]);
        corder[s_coff[cl] + atomicAdd(&ccur[cl], 1u)] = j;
      }
      if (!grid_sync(A.bar, A.fl)) return;
      if (tid < (uint32_t)NC) {  // for the next step
        chist[tid] = 0;
        ccur[tid] = 0;
      }
      bool first = true;
      for (int col = 0; col < NC; ++col) {
        const uint32_t lo = s_coff[col], cnt = s_coff[col + 1] - lo;
        if (cnt == 0) continue;
        if (!first && !grid_sync(A.bar, A.fl)) return;
        phase_update<D, 32, false, true>(A, t, m, mask, maskM, m_prev, base_prev, base, any_nb,
                                         inexact, werr, 0, col, corder + lo, cnt, first);
        first = false;
      }
    } else {
      if (GSmin < 32 && few_lanes)
        phase_update<D, GSmin, BT>(A, t, m, pt ? maskPt : mask, maskM, m_prev, base_prev, base,
                                   any_nb, inexact, werr, pt);
      else
        phase_update<D, 32, BT>(A, t, m, pt ? maskPt : mask, maskM, m_prev, base_prev, base,
                                any_nb, inexact, werr, pt);
    }
    if (__any_sync(kFull, any_nb) && (threadIdx.x & 31) == 0) atomicOr(&A.st[t].has_nb, 1u);
    if (!grid_sync(A.bar, A.fl)) return;
    clk.lap_step(t == 0 ? kSegUpdateFirst : kSegUpdateRest, t, A.res);
    // the pencil table is read: back to clean (the next use of tab[2], as
    // step 1's merge table, is a grid barrier away)
    if (pen && t == 0) {
      if (F32) {
        pencil_release32<D>(A.tab[2], A.qlist, qn);
        if (pen == 2) pencil_release32<D>(A.ptab, A.ptab.list, qn2);
      } else {
        pencil_release<D>(A.tab[2], A.qlist, qn);
        if (pen == 2) pencil_release<D>(A.ptab, A.ptab.list, qn2);
      }
    }
    if (!vst[t].has_nb) {
      converged = true;
      break;
    }
    if (t == A.max_iter) break;
    const uint32_t m1 = vst[t + 1].m;
    if (F32)
      phase_compact32<D, BT>(A, t, m1);
    else
      phase_compact<D, BT>(A, t, m1, inexact, werr);
    if (tid == 0) {
      A.st[t + 1].mask = maskM;
      A.st[t + 1].base = base + m;
    }
    if (!grid_sync(A.bar, A.fl)) return;
    clk.lap_step(kSegCompact, t, A.res);
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
      if (F32) {
        row_release(reinterpret_cast<uint32_t*>(Ms.row) + (size_t)s * RowW<D>::value);
#pragma unroll
        for (int a = 0; a < D; ++a) reinterpret_cast<float*>(Ms.acc)[(size_t)s * D + a] = 0.f;
      } else {
        Ms.key[s] = kEmpty;
        Ms.row[(size_t)s * (D + 1)].x = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          uint64_t* acc = Ms.acc + ((size_t)s * D + a) * 4;
          acc[0] = acc[1] = acc[2] = acc[3] = 0;
        }
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
        atomicAdd(&A.I.k[(uint32_t)(c.key[j] >> g_plan.inst_off)], 1u);
    }
  }
  // numbering: label of a final cell = number of final keys below its key
  // (keys are unique), i.e. ascending lexicographic order of the integer keys
  const bool numbered = k <= A.rank_max;
  const Cells c = A.cells[T & 1];
  if (numbered) {
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
  }
  if (!grid_sync(A.bar, A.fl)) return;
  if (BT) {
    if (tid == 0) {
      // labels of instance b start at 0: subtract the final cells of earlier ones
      uint32_t run = 0;
      for (int b = 0; b < A.B; ++b) {
        A.I.koff[b] = run;
        run += A.I.k[b];
      }
    }
    if (!grid_sync(A.bar, A.fl)) return;
  }

  // the final cell of every initial cell: its chain of T merges walked
  // directly (T dependent loads, no barrier) for short runs, else pointer
  // jumping over the forest (after r rounds every node points 2^r levels up)
  const bool walk = T <= kWalkMax;
  if (!walk) {
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
  }
  for (uint32_t cc = tid; cc < m0; cc += nth) {
    uint32_t v = cc;
    if (walk) {
      for (int s = 0; s < T; ++s) v = A.forest[v];
      if (!numbered) A.forest[cc] = v;  // roots for the numbering after the kernel
    } else {
      v = A.forest[cc];
    }
    if (numbered) {
      const uint32_t r = v - base;
      uint32_t label = A.rank[r];
      if (BT) label -= A.I.koff[(uint32_t)(c.key[r] >> g_plan.inst_off)];
      A.labslot[A.T0.list[cc]] = label;
    }
  }
  if (!grid_sync(A.bar, A.fl)) return;
  if (numbered) {
    if (!split) write_labels(A, tid, nth);
    const LevelTable G = A.tab[T % 3];
    const bool write = (int64_t)k <= A.modes_cap;
    for (uint32_t r = tid; r < k; r += nth) {
      if (F32)
        mode_and_release32<D>(G, g_plan, A.thr, c.key, r, A.rank[r], A.modes, write);
      else
        mode_and_release<D>(G, g_plan, r, A.rank[r], A.modes, write, inexact);
    }
  }
  clk.lap(kSegLabels);
  if (tid == 0) {
    A.res->iterations = T;
    A.res->converged = converged ? 1 : 0;
    A.res->k = k;
    A.res->base = base;
    A.res->need_sort = numbered ? 0u : 1u;
    A.res->labels_ready = numbered && split ? 1u : 0u;  // k_labels_out writes the labels
    A.res->cell_iters = cell_iters;
#pragma unroll
    for (int i = 0; i < kLoopPhases; ++i) A.res->ns[i] = clk.ns[i];
  }
  if (inexact) atomicAdd(&A.fl->inexact, 1ull);
  if (werr) atomicOr(&A.fl->err, kErrWindow);
}

template <int D, bool F32>
__global__ void k_modes_tail(LevelTable G, Plan P, const int64_t* __restrict__ thr,
                             const uint64_t* __restrict__ keys, const uint32_t* __restrict__ rank,
                             double* __restrict__ modes, uint32_t k, bool write) {
  unsigned inexact = 0;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x) {
    if (F32)
      mode_and_release32<D>(G, P, thr, keys, r, rank[r], modes, write);
    else
      mode_and_release<D>(G, P, r, rank[r], modes, write, inexact);
  }
}


// Launch helpers, instantiated per precision in gs_loop64.cu / gs_loop32.cu.
template <int D, bool F32>
int loop_grid_d() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const int smem = (int)(kFilterWords * sizeof(uint32_t));
  if (cudaFuncSetAttribute(k_loop<D, false, F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_loop<D, true, F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem) != cudaSuccess)
    return -1;
  int per_sm_b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_loop<D, true, F32>, kLoopBlock,
                                                    smem) != cudaSuccess)
    return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_loop<D, false, F32>, kLoopBlock,
                                                    smem) != cudaSuccess)
    return -1;
  if (per_sm_b < per_sm) per_sm = per_sm_b;  // one grid size serves both variants
  if (per_sm < 1) return -1;
  if (per_sm > 2) per_sm = 2;  // fewer blocks make the grid barriers cheaper
  const int g = sms * per_sm;
  return g < kMaxLoopGrid ? g : kMaxLoopGrid;
}

template <bool F32>
int loop_grid_t(int d) {
  switch (d) {
    case 1: return loop_grid_d<1, F32>();
    case 2: return loop_grid_d<2, F32>();
    case 3: return loop_grid_d<3, F32>();
    case 4: return loop_grid_d<4, F32>();
    case 5: return loop_grid_d<5, F32>();
    case 6: return loop_grid_d<6, F32>();
    case 7: return loop_grid_d<7, F32>();
    case 8: return loop_grid_d<8, F32>();
  }
  return -1;
}

template <bool F32>
cudaError_t launch_loop_t(const LoopArgs& a, int grid, cudaStream_t s) {
  LoopArgs args = a;
  void* params[] = {&args};
  const size_t smem = kFilterWords * sizeof(uint32_t);
  if (a.B > 1) {
    GS_DISPATCH_D(a.P.d, return cudaLaunchCooperativeKernel((const void*)k_loop<D, true, F32>,
                                                            dim3(grid), dim3(kLoopBlock), params,
                                                            smem, s));
  }
  GS_DISPATCH_D(a.P.d, return cudaLaunchCooperativeKernel((const void*)k_loop<D, false, F32>,
                                                          dim3(grid), dim3(kLoopBlock), params,
                                                          smem, s));
  return cudaSuccess;
}

// Step i's second pass (counts and offsets; scatter; sums) and the label
// writes.  Templates only so that each translation unit that includes this
// file compiles what it uses.
template <bool F32>
cudaError_t launch_prep_offsets_t(const LoopArgs& a, cudaStream_t s) {
  k_prep_counts<<<kPrepCountGrid, kLoopBlock, 0, s>>>(a);
  k_prep_offsets<<<kPrepCountGrid, kLoopBlock, 0, s>>>(a);
  return cudaGetLastError();
}

// Grids of the per-point launches: about the blocks that are resident at once
// (152 SMs; by their registers 8 blocks of the scatter and label writes, 2 or
// 3 of the sums), so that every warp loops over several chunks instead of
// the SMs cycling through thousands of short blocks.
template <bool F32>
cudaError_t launch_prep_scatter_t(const LoopArgs& a, cudaStream_t s) {
  k_prep_scatter<<<grid_for(a.n, kPrepBlock * 4, 152u * 8u), kPrepBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <bool F32>
cudaError_t launch_prep_sums_t(const LoopArgs& a, cudaStream_t s) {
  const unsigned per_sm = (F32 || a.P.d <= 3) ? 3u : 2u;
  const unsigned g = grid_for(a.n, kPrepBlock * 4, 152u * per_sm);
  GS_DISPATCH_D(a.P.d, (k_prep_sums<D, F32><<<g, kPrepBlock, 0, s>>>(a)));
  return cudaGetLastError();
}

template <bool F32>
cudaError_t launch_labels_out_t(const LoopArgs& a, cudaStream_t s) {
  k_labels_out<<<grid_for(a.n / 8 + 1, kPrepBlock, 152u * 8u), kPrepBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <bool F32>
cudaError_t launch_modes_tail_t(const LoopArgs& a, uint32_t k, int T, cudaStream_t s) {
  const bool write = (int64_t)k <= a.modes_cap;
  GS_DISPATCH_D(a.P.d, k_modes_tail<D, F32><<<grid_for(k), kBlock, 0, s>>>(
                           a.tab[T % 3], a.P, a.thr, a.cells[T & 1].key, a.rank, a.modes, k,
                           write));
  return cudaGetLastError();
}

}  // namespace

}  // namespace gs
