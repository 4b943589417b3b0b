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

// The point array is read as one flat stream of n*D values: thread t reads the
// values t, t + S, t + 2S, ... with S a multiple of D, so every thread sees a
// single coordinate a = t mod D and consecutive threads read consecutive
// values (coalesced).  Per-coordinate extremes are reduced in shared memory
// and published with one global atomic per block and coordinate.
template <int D, typename T>
__global__ void __launch_bounds__(kBlock) k_range(const T* __restrict__ pts, int64_t n,
                                                  DevFlags* fl) {
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
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t S = nthreads - nthreads % D;  // stride, a multiple of D
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t mn = INT64_MAX, mx = INT64_MIN;
  uint64_t ma = 0;
  unsigned long long bad = 0;
  if (t < S) {
    for (int64_t e = t; e < total; e += S) {
      uint64_t b = load_bits<T>(pts + e);
      if (((b >> 52) & 0x7FF) == 0x7FF) {
        ++bad;
        continue;
      }
      int64_t o = ord_of_bits(b);
      mn = o < mn ? o : mn;
      mx = o > mx ? o : mx;
      uint64_t ab = b & 0x7FFFFFFFFFFFFFFFull;
      ma = ab > ma ? ab : ma;
    }
    const int a = (int)(t % D);
    if (mn != INT64_MAX) {
      atomicMin(&s_mn[a], (long long)mn);
      atomicMax(&s_mx[a], (long long)mx);
      atomicMax(&s_ma[a], (unsigned long long)ma);
    }
    if (bad) atomicAdd(&s_bad, bad);
  }
  __syncthreads();
  if (threadIdx.x < D && s_mn[threadIdx.x] != INT64_MAX) {
    atomicMin(&fl->min_ord[threadIdx.x], s_mn[threadIdx.x]);
    atomicMax(&fl->max_ord[threadIdx.x], s_mx[threadIdx.x]);
    atomicMax(&fl->maxabs[threadIdx.x], s_ma[threadIdx.x]);
  }
  if (threadIdx.x == 0 && s_bad) atomicAdd(&fl->bad, s_bad);
}

// ---------------------------------------------------------------------------
// Step i: binning
//
// A warp takes 32 consecutive points at a time.  It copies their d
// coordinates (one contiguous run of 32*d values) into shared memory with
// 16-byte loads, so the global reads are coalesced.  Lanes holding the same
// cell key (__match_any_sync) add their exact fixed-point values in shared
// memory, and only the lowest such lane touches the global table: one insert,
// one count add and one exact-sum add per distinct key per warp.

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

template <int D, typename T>
__global__ void __launch_bounds__(kBlock)
    k_bin(const T* __restrict__ pts, int64_t n, Plan P, const int64_t* __restrict__ thr,
          Table T0, uint32_t mask0, uint32_t maxcells, uint32_t* __restrict__ slot0,
          DevFlags* fl, bool vec_ok) {
  __shared__ __align__(16) T s_pts[kWarps][32 * D];
  __shared__ ulonglong2 s_val[kWarps][32 * D];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned inexact = 0, werr = 0;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = gwarp * 32; base < n; base += nwarps * 32) {
    const int cnt = n - base < 32 ? (int)(n - base) : 32;
    stage_points<T>(pts + base * D, cnt * D, s_pts[w], vec_ok, lane);
    __syncwarp();
    const bool valid = lane < cnt;
    uint64_t key = kEmpty;
    if (valid) {
      key = 0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        uint64_t b = bits_of(s_pts[w][lane * D + a]);
        int idx = key_index(thr + P.thr_off[a], P.span[a], P.kmin[a], P.inv_h, b);
        key |= (uint64_t)(idx + 1) << P.off[a];
        u128 V = to_fixed(b, P.L[a], inexact, werr);
        s_val[w][lane * D + a] = make_ulonglong2((uint64_t)V, (uint64_t)(V >> 64));
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
          uint32_t id = atomicAdd(&fl->m0, 1u);
          if (id < maxcells) T0.list[id] = s; else atomicOr(&fl->err, kErrOverflow);
        }
        atomicAdd(&T0.cnt[s], (uint32_t)__popc(peers));
#pragma unroll
        for (int a = 0; a < D; ++a) {
          u128 S = 0;
          for (unsigned pm = peers; pm; pm &= pm - 1) {
            const ulonglong2 v = s_val[w][(__ffs(pm) - 1) * D + a];
            S += (u128)v.x | ((u128)v.y << 64);
          }
          atomic_add_fixed(T0.acc + ((size_t)s * D + a) * 4, S);
        }
      }
    }
    s = __shfl_sync(kFull, s, leader);
    if (valid) slot0[base + lane] = s;
    __syncwarp();
  }
  if (inexact) atomicAdd(&fl->inexact, 1ull);
  if (werr) atomicOr(&fl->err, kErrWindow);
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

enum { kSegLevel0 = 0, kSegGather = 1, kSegMerge = 2, kSegCompact = 3, kSegLabels = 4 };

template <int D>
__device__ __forceinline__ u128 fix_at(const ulonglong2* __restrict__ fix, uint32_t i, int a) {
  const ulonglong2 v = fix[(size_t)i * D + a];
  return (u128)v.x | ((u128)v.y << 64);
}

__device__ __forceinline__ ulonglong2 pack(u128 v) {
  return make_ulonglong2((uint64_t)v, (uint64_t)(v >> 64));
}

// Lanes given to one cell in the gather: enough for the 3^d probes of small d.
template <int D>
struct GatherLanes {
  static constexpr int value = D == 1 ? 4 : (D == 2 ? 16 : 32);
};

// Level 0: the cells binning created (in arrival order), their sums rounded
// once, and their lookup table.  Resets the binning table's slots.
template <int D>
__device__ void phase_level0(const LoopArgs& A, uint32_t m0, uint32_t maskA, unsigned& inexact,
                             unsigned& werr) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nth = gridDim.x * blockDim.x;
  const Table T0 = A.T0;
  const Table G = A.tab[0];
  const Cells c = A.cells[0];
  for (uint32_t id = tid; id < m0; id += nth) {
    const uint32_t s = T0.list[id];
    const uint64_t key = T0.key[s];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      uint64_t* acc = T0.acc + ((size_t)s * D + a) * 4;
      const double v = round_fixed(limbs_value(acc), A.P.L[a], inexact);
      c.fix[(size_t)id * D + a] = pack(to_fixed(bits_of(v), A.P.L[a], inexact, werr));
      acc[0] = acc[1] = acc[2] = acc[3] = 0;
    }
    c.key[id] = key;
    c.cnt[id] = T0.cnt[s];
    T0.cnt[s] = 0;
    T0.key[s] = kEmpty;
    bool won;
    const uint32_t sa = table_insert(G.key, maskA, key, won, &A.fl->err);
    if (sa != kNone) {
      G.id[sa] = id;
      G.list[id] = sa;
    }
  }
}

// Steps ii-iii for every cell of level t, and the neighbour test of step v.
template <int D>
__device__ void phase_gather(const LoopArgs& A, int t, uint32_t m, uint32_t mask, bool& any_nb,
                             unsigned& inexact) {
  constexpr int GS = GatherLanes<D>::value;
  const int lane = threadIdx.x & 31;
  const int glane = lane & (GS - 1);
  const unsigned gmask = GS == 32 ? kFull : (((1u << GS) - 1u) << (lane & ~(GS - 1)));
  const uint32_t group = (blockIdx.x * blockDim.x + threadIdx.x) / GS;
  const uint32_t ngroups = (gridDim.x * blockDim.x) / GS;
  const Table G = (t & 1) ? A.tab[1] : A.tab[0];
  const Cells c = (t & 1) ? A.cells[1] : A.cells[0];
  const int nprobe = A.P.nprobe, center = A.P.center;
  for (uint32_t j = group; j < m; j += ngroups) {
    const uint64_t key = c.key[j];
    uint32_t Dc = 0;
    u128 N[D];
#pragma unroll
    for (int a = 0; a < D; ++a) N[a] = 0;
    for (int p = glane; p < nprobe; p += GS) {
      const uint32_t s = table_find(G.key, mask, key + __ldg(&A.dtab[p]));
      if (s == kNone) continue;
      const uint32_t id = G.id[s];
      Dc += c.cnt[id];
#pragma unroll
      for (int a = 0; a < D; ++a) N[a] += fix_at<D>(c.fix, id, a);
      if (p != center) any_nb = true;
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
    uint64_t field = 0;
    if (glane < D) {
      u128 Na = 0;
      int La = 0, off = 0, span = 1, toff = 0;
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
      A.sp[(size_t)j * D + glane] = sv;
      const int idx = key_index(A.thr + toff, span, kmin, A.P.inv_h, bits_of(sv));
      field = (uint64_t)(idx + 1) << off;
    }
#pragma unroll
    for (int o = GS / 2; o > 0; o >>= 1) field |= __shfl_xor_sync(gmask, field, o);
    if (glane == 0) A.nkey[j] = field;
  }
}

// Parent links of level t-1 (its merge slots now carry the ids of level t),
// and release of level t-1's lookup table, which the merge of step t reuses.
__device__ void phase_finish(const LoopArgs& A, int t, uint32_t m_prev, uint32_t base_prev,
                             uint32_t base) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nth = gridDim.x * blockDim.x;
  const Table cur = (t & 1) ? A.tab[1] : A.tab[0];
  const Table old = (t & 1) ? A.tab[0] : A.tab[1];
  for (uint32_t j = tid; j < m_prev; j += nth) {
    A.forest[base_prev + j] = base + cur.id[A.pslot[j]];
    old.key[old.list[j]] = kEmpty;
  }
}

// Step iv: every cell of level t adds its count and count-weighted centroid
// (Eq. 3-4) into the slot of its new key.
template <int D>
__device__ void phase_merge(const LoopArgs& A, int t, uint32_t m, uint32_t maskM,
                            unsigned& inexact, unsigned& werr) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nth = gridDim.x * blockDim.x;
  const Table M = (t & 1) ? A.tab[0] : A.tab[1];
  const Cells c = (t & 1) ? A.cells[1] : A.cells[0];
  for (uint32_t j = tid; j < m; j += nth) {
    bool won;
    const uint32_t s = table_insert(M.key, maskM, A.nkey[j], won, &A.fl->err);
    if (s == kNone) continue;
    if (won) {
      const uint32_t id = atomicAdd(&A.st[t + 1].m, 1u);
      M.list[id] = s;
    }
    const uint32_t cnt = c.cnt[j];
    atomicAdd(&M.cnt[s], cnt);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const u128 V = to_fixed(bits_of(A.sp[(size_t)j * D + a]), A.P.L[a], inexact, werr);
      atomic_add_fixed(M.acc + ((size_t)s * D + a) * 4, V * (u128)cnt);
    }
    A.pslot[j] = s;
  }
}

// The cells of level t+1 from the merge table: sums rounded once.
template <int D>
__device__ void phase_compact(const LoopArgs& A, int t, uint32_t m1, unsigned& inexact,
                              unsigned& werr) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nth = gridDim.x * blockDim.x;
  const Table M = (t & 1) ? A.tab[0] : A.tab[1];
  const Cells nx = (t & 1) ? A.cells[0] : A.cells[1];
  for (uint32_t id = tid; id < m1; id += nth) {
    const uint32_t s = M.list[id];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      uint64_t* acc = M.acc + ((size_t)s * D + a) * 4;
      const double v = round_fixed(limbs_value(acc), A.P.L[a], inexact);
      nx.fix[(size_t)id * D + a] = pack(to_fixed(bits_of(v), A.P.L[a], inexact, werr));
      acc[0] = acc[1] = acc[2] = acc[3] = 0;
    }
    nx.key[id] = M.key[s];
    nx.cnt[id] = M.cnt[s];
    M.cnt[s] = 0;
    M.id[s] = id;
  }
}

template <int D>
__global__ void __launch_bounds__(kBlock) k_loop(LoopArgs A) {
  unsigned inexact = 0, werr = 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nth = gridDim.x * blockDim.x;
  volatile IterState* vst = A.st;
  SegClock clk;
  clk.start();

  // level 0
  const uint32_t m0 = *(volatile uint32_t*)&A.fl->m0;
  const uint32_t maskA = mask_for(m0, A.capAB);
  if (tid == 0) {
    A.st[0].m = m0;
    A.st[0].mask = maskA;
    A.st[0].base = 0;
  }
  phase_level0<D>(A, m0, maskA, inexact, werr);
  if (!grid_sync(A.bar, A.fl)) return;
  clk.lap(kSegLevel0);

  int t = 0;
  uint32_t m = m0, mask = maskA, base = 0, m_prev = 0, base_prev = 0;
  unsigned long long cell_iters = 0;
  bool converged = false;
  for (;;) {
    bool any_nb = false;
    phase_gather<D>(A, t, m, mask, any_nb, inexact);
    if (t > 0) phase_finish(A, t, m_prev, base_prev, base);
    if (__any_sync(kFull, any_nb) && (threadIdx.x & 31) == 0) atomicOr(&A.st[t].has_nb, 1u);
    if (!grid_sync(A.bar, A.fl)) return;
    clk.lap(kSegGather);
    if (!vst[t].has_nb) {
      converged = true;
      break;
    }
    if (t == A.max_iter) break;
    const uint32_t maskM = mask_for(m, A.capAB);
    phase_merge<D>(A, t, m, maskM, inexact, werr);
    if (!grid_sync(A.bar, A.fl)) return;
    clk.lap(kSegMerge);
    const uint32_t m1 = vst[t + 1].m;
    phase_compact<D>(A, t, m1, inexact, werr);
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

  // the final level: every cell is its own root; release its lookup table
  {
    const Table G = (T & 1) ? A.tab[1] : A.tab[0];
    for (uint32_t j = tid; j < k; j += nth) {
      A.forest[base + j] = base + j;
      G.key[G.list[j]] = kEmpty;
    }
  }
  if (!grid_sync(A.bar, A.fl)) return;

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
    const Cells c = (T & 1) ? A.cells[1] : A.cells[0];
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
    for (uint32_t cc = tid; cc < m0; cc += nth)
      A.labslot[A.T0.list[cc]] = A.rank[A.forest[cc] - base];
    if (!grid_sync(A.bar, A.fl)) return;
    for (int64_t i = tid; i < A.n; i += nth) A.labels[i] = (int32_t)A.labslot[A.slot0[i]];
    if ((int64_t)k <= A.modes_cap) {
      for (uint32_t r = tid; r < k; r += nth) {
        const uint32_t rr = A.rank[r];
        const double cnt = (double)c.cnt[r];
#pragma unroll
        for (int a = 0; a < D; ++a)
          A.modes[(size_t)rr * D + a] =
              round_fixed(fix_at<D>(c.fix, r, a), A.P.L[a], inexact) / cnt;
      }
    }
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
__global__ void k_labslot_tail(const uint32_t* __restrict__ list0,
                               const uint32_t* __restrict__ root,
                               const uint32_t* __restrict__ rank, uint32_t baseT,
                               uint32_t* __restrict__ labslot, uint32_t m0) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m0; c += gridDim.x * blockDim.x)
    labslot[list0[c]] = rank[root[c] - baseT];
}

__global__ void k_labels_tail(const uint32_t* __restrict__ slot0,
                              const uint32_t* __restrict__ labslot, int32_t* __restrict__ labels,
                              int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    labels[i] = (int32_t)labslot[slot0[i]];
}

template <int D>
__global__ void k_modes_tail(Cells c, Plan P, const uint32_t* __restrict__ rank,
                             double* __restrict__ modes, uint32_t k) {
  unsigned inexact = 0;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x) {
    const uint32_t rr = rank[r];
    const double cnt = (double)c.cnt[r];
#pragma unroll
    for (int a = 0; a < D; ++a)
      modes[(size_t)rr * D + a] = round_fixed(fix_at<D>(c.fix, r, a), P.L[a], inexact) / cnt;
  }
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
  unsigned g = grid_for(n * d, kBlock * 8, 152u * 8u);
  if (f32) {
    GS_DISPATCH_D(d, k_range<D, float><<<g, kBlock, 0, s>>>((const float*)pts, n, fl));
  } else {
    GS_DISPATCH_D(d, k_range<D, double><<<g, kBlock, 0, s>>>((const double*)pts, n, fl));
  }
  return cudaGetLastError();
}

cudaError_t launch_bin(const void* pts, bool f32, int64_t n, const Plan& P, const int64_t* thr,
                       Table T0, uint32_t mask0, uint32_t maxcells, uint32_t* slot0,
                       DevFlags* fl, cudaStream_t s) {
  const unsigned g = grid_for((n + 31) / 32 * 32, kBlock, 152u * 6u);
  const bool vec_ok = ((uintptr_t)pts & 15u) == 0;
  if (f32) {
    GS_DISPATCH_D(P.d, k_bin<D, float><<<g, kBlock, 0, s>>>((const float*)pts, n, P, thr, T0,
                                                            mask0, maxcells, slot0, fl, vec_ok));
  } else {
    GS_DISPATCH_D(P.d, k_bin<D, double><<<g, kBlock, 0, s>>>((const double*)pts, n, P, thr, T0,
                                                             mask0, maxcells, slot0, fl, vec_ok));
  }
  return cudaGetLastError();
}

namespace {
template <int D>
int loop_grid_d() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_loop<D>, kBlock, 0) != cudaSuccess)
    return -1;
  if (per_sm < 1) return -1;
  if (per_sm > 2) per_sm = 2;  // fewer blocks make the grid barriers cheaper
  return sms * per_sm;
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
  GS_DISPATCH_D(a.P.d, return cudaLaunchCooperativeKernel((const void*)k_loop<D>, dim3(grid),
                                                          dim3(kBlock), params, 0, s));
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
  k_labslot_tail<<<grid_for(m0), kBlock, 0, s>>>(a.T0.list, a.forest, a.rank, baseT, a.labslot,
                                                 m0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_labels_tail<<<grid_for(a.n), kBlock, 0, s>>>(a.slot0, a.labslot, a.labels, a.n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((int64_t)k <= a.modes_cap) {
    const Cells c = (T & 1) ? a.cells[1] : a.cells[0];
    GS_DISPATCH_D(a.P.d, k_modes_tail<D><<<grid_for(k), kBlock, 0, s>>>(c, a.P, a.rank, a.modes,
                                                                         k));
  }
  return cudaGetLastError();
}

}  // namespace gs
