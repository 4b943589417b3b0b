// gs_kernels.cu -- the per-point kernels of the GridShift hot path on sm_103a
// (Kumar et al., arXiv 2206.02200, Sec. 2.1 and Algorithm 1):
//   k_range  key range, fixed-point window and finiteness of the input, then
//            (its last block) the plan of the call (key packing, face table,
//            offsets)
//   k_bin    step i, first pass: cell key and count of every point
// and the kernels that finish the labels when the final cells are numbered
// by a radix sort.  Everything between binning and the labels runs in the
// loop kernel (gs_loop.cuh).
#include <atomic>

#include "gs_common.cuh"
#include "gs_planner.cuh"

namespace gs {

namespace {

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

__device__ void plan_block(int d, int64_t n, const PlanJob& J, DevFlags* fl);

template <int D, typename T, int W>
__global__ void __launch_bounds__(kBlock) k_range(const T* __restrict__ pts, int64_t n,
                                                  DevFlags* fl, bool plan, PlanJob J) {
  constexpr int U = 4;  // words in flight per thread
  if (plan) {
    // the loop kernel's start state, cleared by the whole grid
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    for (uint32_t w = gt; w < J.filter_vec; w += gs) J.filters[w] = make_uint4(0, 0, 0, 0);
    for (uint32_t i = gt; i < J.n_st; i += gs) J.st[i] = IterState{};
    if (gt == 0) {
      *J.bar = GridBar{};
      *J.res = LoopResult{};
    }
  }
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
  if (!plan) return;
  // the last block to publish its extremes makes the plan
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&fl->range_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  plan_block(D, n, J, fl);
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

// The plan of a call (Sec. 2.1 i) from its key range, on the device, by one
// block (the last block of the key-range kernel, once every block has
// published its extremes): one thread per axis, then one thread for the key
// layout, into fl->plan; then the block fills the face table and the
// neighbour offsets.  A non-finite input, a key range the packing cannot
// hold, or a face table above thr_cap entries sets fl->plan_status instead
// (binning and the loop kernel then do nothing; the host reads the status).
__device__ void plan_block(int d, int64_t n, const PlanJob& J, DevFlags* fl) {
  __shared__ Plan s_plan;
  __shared__ PlanSizes s_z;
  __shared__ uint32_t s_st, s_ax[kMaxD];
  __shared__ DevFlags s_fl;  // the key range, read at L2 (other blocks wrote it)
  if (threadIdx.x == 0) {
    memset(&s_plan, 0, sizeof(s_plan));
    for (int a = 0; a < kMaxD; ++a) {
      s_fl.min_ord[a] = __ldcg(&fl->min_ord[a]);
      s_fl.max_ord[a] = __ldcg(&fl->max_ord[a]);
      s_fl.maxabs[a] = __ldcg(&fl->maxabs[a]);
    }
    s_fl.bad = __ldcg(&fl->bad);
  }
  __syncthreads();
  if ((int)threadIdx.x < d) s_ax[threadIdx.x] = plan_axis(threadIdx.x, J.h, n, s_fl, s_plan);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t status = s_fl.bad ? kPlanNonFinite : kPlanOK;
    for (int a = 0; a < d && status == kPlanOK; ++a) status = s_ax[a];
    if (status == kPlanOK) status = plan_finish(d, J.h, J.B, s_plan, s_z);
    if (status == kPlanOK && s_z.thr_words > J.thr_cap) status = kPlanTable;
    fl->plan = s_plan;
    fl->plan_sizes = s_z;
    fl->plan_status = status;
    s_st = status;
  }
  __syncthreads();
  if (s_st != kPlanOK) return;
  for (uint64_t j = threadIdx.x; j < s_z.thr_words; j += blockDim.x)
    J.thr[j] = plan_face_entry(s_plan, J.h, j);
  // dtab: nprobe packed-key offsets, then nprobe 32-bit offset vectors
  uint32_t* vpack = reinterpret_cast<uint32_t*>(J.dtab + s_plan.nprobe);
  for (int p = threadIdx.x; p < s_plan.nprobe; p += blockDim.x)
    plan_probe(s_plan, p, J.dtab + p, vpack + p);
}

// LISTED: new cells are listed per warp, 32 at a time (five blocks per SM:
// the warp's list costs registers); else each new cell takes one add on the
// cell count (six blocks per SM).  Tuning::bin_list chooses.
template <int D, typename T, bool LISTED>
__global__ void __launch_bounds__(kBlock, LISTED ? 5 : 6)
    k_bin(const T* __restrict__ pts, int64_t n, const int64_t* __restrict__ thr,
          BinTable T0, uint32_t mask0, uint32_t maxcells, uint32_t* __restrict__ slot0,
          DevFlags* fl, bool vec_ok, const int64_t* __restrict__ offsets, int B,
          const SweepPlan* __restrict__ sweep, uint32_t n0) {
  __shared__ __align__(16) T s_pts[kWarps][32 * D];
  __shared__ uint32_t s_new[kWarps][32];  // a warp's new cells not yet listed
  __shared__ Plan s_plan;
  __shared__ uint32_t s_ok;
  // the plan, into shared memory (nothing runs unless it is valid)
  if (threadIdx.x == 0) {
    s_ok = *(volatile uint32_t*)&fl->plan_status == kPlanOK;
    if (s_ok) s_plan = fl->plan;
  }
  __syncthreads();
  if (!s_ok) return;
  const Plan& P = s_plan;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // LISTED: new cells are listed per warp, 32 at a time.  The cell count is
  // one address for the whole grid, where atomics from different warps
  // serialise (about 0.7 ns each on GB300): one add per new cell costs 0.2 ms
  // on a 4K image's 268k cells.
  uint32_t pend = 0;  // entries of s_new[w] (warp-uniform)
  auto list_cells = [&](uint32_t& cnt) {
    __syncwarp();
    uint32_t b0 = 0;
    if (lane == 0) b0 = atomicAdd(&fl->m0, cnt);
    b0 = __shfl_sync(kFull, b0, 0);
    if ((uint32_t)lane < cnt) {
      const uint32_t id = b0 + lane;
      if (id < maxcells) T0.list[id] = s_new[w][lane]; else atomicOr(&fl->err, kErrOverflow);
    }
    __syncwarp();
    cnt = 0;
  };
  for (int64_t base = gwarp * 32; base < n; base += nwarps * 32) {
    const int cnt = n - base < 32 ? (int)(n - base) : 32;
    if (!sweep) stage_points<T>(pts + base * D, cnt * D, s_pts[w], vec_ok, lane);
    __syncwarp();
    const bool valid = lane < cnt;
    uint64_t key = kEmpty;
    if (valid && sweep) {
      // bandwidth sweep: point j of instance b is row j of pts, its cell
      // decided with b's bandwidth
      const int64_t i = base + lane;
      const uint32_t b = (uint32_t)(i / n0);
      const T* row = pts + (size_t)(i - (int64_t)b * n0) * D;
      const SweepPlan* S = sweep + b;
      key = (uint64_t)b << P.inst_off;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int idx = key_index(thr + __ldg(&S->thr_off[a]), __ldg(&S->span[a]),
                                  __ldg(&S->kmin[a]), __ldg(&S->inv_h), bits_of(__ldg(row + a)));
        key |= (uint64_t)(idx + 1) << P.off[a];
      }
    } else if (valid) {
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
    bool won = false;
    if (valid && lane == leader) {
      s = table_insert(T0.key, mask0, key, won, &fl->err);
      if (s != kNone) {
        if (!LISTED && won) {
          const uint32_t id = atomicAdd(&fl->m0, 1u);
          if (id < maxcells) T0.list[id] = s; else atomicOr(&fl->err, kErrOverflow);
        }
        atomicAdd(&T0.cnt[s], (uint32_t)__popc(peers));
      }
      won = won && s != kNone;
    }
    if constexpr (LISTED) {
      const unsigned wm = __ballot_sync(kFull, won);
      if (pend + __popc(wm) > 32) list_cells(pend);
      if (won) s_new[w][pend + __popc(wm & ((1u << lane) - 1u))] = s;
      pend += __popc(wm);
    }
    s = __shfl_sync(kFull, s, leader);
    if (valid) slot0[base + lane] = s;
    __syncwarp();
  }
  if (LISTED && pend) list_cells(pend);
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
                         const PlanJob* job, cudaStream_t s) {
  const bool vec = ((uintptr_t)pts & 15u) == 0;
  const int W = vec ? (f32 ? 4 : 2) : 1;
  const unsigned g = grid_for(n * d / W, kBlock * 4, 152u * 8u);
  const bool plan = job != nullptr;
  const PlanJob J = plan ? *job : PlanJob{};
  if (f32) {
    if (vec) {
      GS_DISPATCH_D(d, k_range<D, float, 4><<<g, kBlock, 0, s>>>((const float*)pts, n, fl, plan, J));
    } else {
      GS_DISPATCH_D(d, k_range<D, float, 1><<<g, kBlock, 0, s>>>((const float*)pts, n, fl, plan, J));
    }
  } else {
    if (vec) {
      GS_DISPATCH_D(d, k_range<D, double, 2><<<g, kBlock, 0, s>>>((const double*)pts, n, fl, plan, J));
    } else {
      GS_DISPATCH_D(d, k_range<D, double, 1><<<g, kBlock, 0, s>>>((const double*)pts, n, fl, plan, J));
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_bin(const void* pts, bool f32, int64_t n, int d, const int64_t* thr,
                       BinTable T0, uint32_t mask0, uint32_t maxcells, uint32_t* slot0,
                       DevFlags* fl, const int64_t* offsets, int B, const SweepPlan* sweep,
                       uint32_t n0, bool listed, cudaStream_t s) {
  const unsigned g = grid_for((n + 31) / 32 * 32, kBlock, 152u * (listed ? 5u : 6u));
  const bool vec_ok = ((uintptr_t)pts & 15u) == 0;
  if (sweep && n0 == 0) return cudaErrorInvalidValue;
#define GS_BIN(T, LST)                                                                         \
  GS_DISPATCH_D(d, (k_bin<D, T, LST><<<g, kBlock, 0, s>>>((const T*)pts, n, thr, T0, mask0,     \
                                                          maxcells, slot0, fl, vec_ok, offsets, \
                                                          B, sweep, n0)))
  if (f32) {
    if (listed) { GS_BIN(float, true); } else { GS_BIN(float, false); }
  } else {
    if (listed) { GS_BIN(double, true); } else { GS_BIN(double, false); }
  }
#undef GS_BIN
  return cudaGetLastError();
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
  return launch_modes_tail(a, k, T, s);
}

cudaError_t launch_modes_tail(const LoopArgs& a, uint32_t k, int T, cudaStream_t s) {
  return a.mixed ? launch_modes_tail_fp32(a, k, T, s) : launch_modes_tail_fp64(a, k, T, s);
}

// The loop kernel's co-resident grid for (device, d, precision), found once
// (function attributes and occupancy queries cost tens of microseconds).
int loop_grid(int d, bool mixed) {
  constexpr int kDevices = 64;
  static std::atomic<int> cache[kDevices][kMaxD + 1][2];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (dev < 0 || dev >= kDevices || d < 1 || d > kMaxD)
    return mixed ? loop_grid_fp32(d) : loop_grid_fp64(d);
  std::atomic<int>& c = cache[dev][d][mixed ? 1 : 0];
  int g = c.load(std::memory_order_acquire);
  if (g > 0) return g;
  g = mixed ? loop_grid_fp32(d) : loop_grid_fp64(d);
  if (g > 0) c.store(g, std::memory_order_release);
  return g;
}

cudaError_t launch_prep_sums(const LoopArgs& a, cudaStream_t s) {
  return a.mixed ? launch_prep_sums_fp32(a, s) : launch_prep_sums_fp64(a, s);
}

cudaError_t launch_loop(const LoopArgs& a, int grid, cudaStream_t s) {
  return a.mixed ? launch_loop_fp32(a, grid, s) : launch_loop_fp64(a, grid, s);
}

}  // namespace gs
