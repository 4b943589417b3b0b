// gs_loop_fp32.cuh -- the phases of the float32 mixed-precision path
// (GS_FP32_MIXED).  One part of the loop kernel of gs_loop.cuh, which
// includes the parts in order.
#pragma once

#include "gs_loop_fp64.cuh"

namespace gs {

namespace {
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
    // the cells' ids (the sums are indexed by them, as in phase_cell_sums)
    // and keys, loaded while the coordinates are in flight
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

// Level 0 (float32): mean offsets of the initial cells from their lower faces;
// resets the binning table's slots.  The sums are the float sums of offsets
// of phase_cell_sums32, or, where binning formed them (Tuning::bin_sums), the
// exact coordinate sums, rounded once to float64 before the mean is taken.
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
      if (A.tune.bin_sums) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          uint64_t* acc = T0.acc + ((size_t)s * D + a) * 4;
          unsigned inx = 0;
          const double sum = round_fixed(limbs_value(acc), g_plan.L[a], inx);
          acc[0] = acc[1] = acc[2] = acc[3] = 0;
          const double org = (double)(float)face_of(g_plan, A.thr, key, a);
          r[3 + a] = __float_as_uint((float)(sum / (double)cnt - org));
        }
      } else {
        // all the sums are loaded before any store
        float sum[D];
#pragma unroll
        for (int a = 0; a < D; ++a) sum[a] = __ldcg(tacc + (size_t)id * D + a);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          r[3 + a] = __float_as_uint(sum[a] / (float)cnt);
          tacc[(size_t)id * D + a] = 0.f;
        }
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
        // the level's occupancy filter (a superset of its keys, also in the
        // pencil form of step 0) skips the absent neighbours on chip, as in
        // the main probe loop
        const uint32_t fb = filter_bit(qk, lg);
        if (A.tune.filter && !((s_filter[fb >> 5] >> (fb & 31)) & 1u)) continue;
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
      // all the sums are loaded before any store
      float sum[D];
#pragma unroll
      for (int a = 0; a < D; ++a) sum[a] = __ldcg(macc + (size_t)s * D + a);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        r[3 + a] = __float_as_uint(sum[a] / (float)cnt);
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

}  // namespace

}  // namespace gs
