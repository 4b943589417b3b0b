// gs_loop_tail.cuh -- the one-block tails that finish small levels in shared
// memory, in both precisions.  One part of the loop kernel of gs_loop.cuh,
// which includes the parts in order.
#pragma once

#include "gs_loop_fp32.cuh"

namespace gs {

namespace {
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

}  // namespace

}  // namespace gs
