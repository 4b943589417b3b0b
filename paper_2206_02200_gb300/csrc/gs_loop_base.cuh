// gs_loop_base.cuh -- the loop kernel's building blocks: the plan in shared
// memory, the software grid barrier, the device-clock split, grid-stride
// helpers, the occupancy filter, lanes per cell.  One part of the loop
// kernel of gs_loop.cuh, which includes the parts in order.
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

// The cell sums of all D axes as the float64 values of Sec. 2.1 (each exact
// sum in its four limb accumulators rounded once), held as the fixed-point
// integers they equal, into out[0 .. D-1]; clears the accumulators.  Every
// limb is loaded (from L2) before anything is stored: stores between the
// loads would make each axis wait for the one before.
template <int D>
__device__ __forceinline__ void settle_sums(uint64_t* acc, ulonglong2* out, const int* L,
                                            unsigned& werr) {
  ulonglong2 l[D][2];
  const ulonglong2* a2 = reinterpret_cast<const ulonglong2*>(acc);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    l[a][0] = __ldcg(a2 + 2 * a);
    l[a][1] = __ldcg(a2 + 2 * a + 1);
  }
  u128 v[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const uint64_t limbs[4] = {l[a][0].x, l[a][0].y, l[a][1].x, l[a][1].y};
    v[a] = round_to_double(limbs_value(limbs), L[a], werr);
  }
  ulonglong2* z = reinterpret_cast<ulonglong2*>(acc);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    out[a] = pack(v[a]);
    z[2 * a] = make_ulonglong2(0ull, 0ull);
    z[2 * a + 1] = make_ulonglong2(0ull, 0ull);
  }
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

}  // namespace

}  // namespace gs
