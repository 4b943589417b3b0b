// gs_loop_fp64.cuh -- the phases of the exact (GS_FP64) path: binning's
// second pass (counting sort, exact cell sums), level 0, the pencil form of
// the first update, parity colours, the update step (Eq. 1-4, parallel and
// sequential forms), compaction, modes.  One part of the loop kernel of
// gs_loop.cuh, which includes the parts in order.
#pragma once

#include "gs_loop_base.cuh"

namespace gs {

namespace {
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

// Adds V into the sum accumulators of the cell of id `id` (the counting
// sort's sums are indexed by the cell's id, its rank in the sorted order, so
// consecutive runs add to consecutive accumulators; sums formed in binning
// are indexed by the table slot).
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
      settle_sums<D>(T0.acc + (size_t)(A.tune.bin_sums ? s : id) * D * 4, r + 1, g_plan.L, werr);
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
    const uint32_t cnt = (uint32_t)__ldcg(&r[0].x);
    if (!restored) settle_sums<D>(M.acc + (size_t)s * D * 4, r + 1, g_plan.L, werr);
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

}  // namespace

}  // namespace gs
