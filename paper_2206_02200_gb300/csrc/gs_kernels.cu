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
// (coalesced).  Four words per thread are in flight at once.  Extremes are
// kept in the input's own bit width (order codes of float32 values widen to
// those of float64 at the end: the widening is exact and keeps the order),
// combined per block without atomics and published with one global atomic
// per block and coordinate.
template <typename T>
struct Bits;  // the unsigned and signed integers of T's width
template <>
struct Bits<double> {
  using U = uint64_t;
  using S = int64_t;
  static constexpr int kExpShift = 52;
  static constexpr U kExpMask = 0x7FF;
  static __device__ __forceinline__ uint64_t widen(U b) { return b; }
};
template <>
struct Bits<float> {
  using U = uint32_t;
  using S = int32_t;
  static constexpr int kExpShift = 23;
  static constexpr U kExpMask = 0xFF;
  static __device__ __forceinline__ uint64_t widen(U b) { return f32_bits_to_f64_bits(b); }
};

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
  static __device__ __forceinline__ void load(const float* p, uint32_t (&b)[1]) {
    b[0] = __float_as_uint(__ldg(p));
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
  static __device__ __forceinline__ void load(const float* p, uint32_t (&b)[4]) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    b[0] = v.x;
    b[1] = v.y;
    b[2] = v.z;
    b[3] = v.w;
  }
};

// Extremes of one coordinate as order codes: signed integers whose order is
// the order of the values (code = bits with the magnitude bits flipped when
// the sign bit is set; -0 sits just below +0).  Per value only the code and
// one min/max pair: a non-finite value shows up as an extreme (+inf and
// positive NaNs above every finite code, -inf and negative NaNs below), and
// the largest magnitude is that of the least or the greatest value.
template <typename T>
struct RangeAcc {
  using U = typename Bits<T>::U;
  using S = typename Bits<T>::S;
  static constexpr int kBits = 8 * (int)sizeof(U);
  static constexpr U kSign = (U)1 << (kBits - 1);
  static constexpr U kInfBits = Bits<T>::kExpMask << Bits<T>::kExpShift;  // +inf
  S mn = (S)(kSign - 1), mx = (S)kSign;
  __device__ __forceinline__ void add(U b) {
    const S o = ord(b);
    mn = o < mn ? o : mn;
    mx = o > mx ? o : mx;
  }
  static __device__ __forceinline__ S ord(U b) {
    const S s = (S)b;
    return s ^ (S)((U)(s >> (kBits - 1)) >> 1);
  }
  static __device__ __forceinline__ U bits(S o) { return (U)(o ^ (S)((U)(o >> (kBits - 1)) >> 1)); }
  __device__ __forceinline__ bool empty() const { return mn > mx; }
  // some value was +-inf or NaN (non-empty accumulators)
  __device__ __forceinline__ bool nonfinite() const {
    return mx >= ord(kInfBits) || mn <= ord(kInfBits | kSign);
  }
  __device__ __forceinline__ void merge(const RangeAcc& r) {
    mn = r.mn < mn ? r.mn : mn;
    mx = r.mx > mx ? r.mx : mx;
  }
  __device__ __forceinline__ RangeAcc shfl_down(int o) const {
    RangeAcc r;
    r.mn = (S)__shfl_down_sync(kFull, (U)mn, o);
    r.mx = (S)__shfl_down_sync(kFull, (U)mx, o);
    return r;
  }
  // float64 order codes (-0 taken as +0) and the largest magnitude's bits
  // (finite, non-empty accumulators)
  __device__ __forceinline__ int64_t mn64() const { return ord_of_bits(Bits<T>::widen(bits(mn))); }
  __device__ __forceinline__ int64_t mx64() const { return ord_of_bits(Bits<T>::widen(bits(mx))); }
  __device__ __forceinline__ uint64_t ma64() const {
    const uint64_t a = Bits<T>::widen(bits(mn)) & 0x7FFFFFFFFFFFFFFFull;
    const uint64_t c = Bits<T>::widen(bits(mx)) & 0x7FFFFFFFFFFFFFFFull;
    return a > c ? a : c;
  }
};

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

// 16 bytes global -> shared without a register round trip (cp.async), one
// commit group per call site; wait_group<N>: at most N groups still in flight.
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The values of one 16-byte word.
template <typename T>
struct Unpack;
template <>
struct Unpack<double> {
  static __device__ __forceinline__ void get(const uint4 v, uint64_t (&b)[2]) {
    b[0] = (uint64_t)v.x | ((uint64_t)v.y << 32);
    b[1] = (uint64_t)v.z | ((uint64_t)v.w << 32);
  }
};
template <>
struct Unpack<float> {
  static __device__ __forceinline__ void get(const uint4 v, uint32_t (&b)[4]) {
    b[0] = v.x;
    b[1] = v.y;
    b[2] = v.z;
    b[3] = v.w;
  }
};

// Blocks of the key-range kernel per SM (its launch bound; the grid is at
// most this many per SM, one wave).
constexpr unsigned kRangeBlocksPerSM = 4;

__device__ void plan_block(int d, int64_t n, const PlanJob& J, DevFlags* fl);

template <int D, typename T, int W>
__global__ void __launch_bounds__(kBlock, kRangeBlocksPerSM)
    k_range(const T* __restrict__ pts, int64_t n, DevFlags* fl, bool plan, PlanJob J,
            bool read) {
  using Acc = RangeAcc<T>;
  using U = typename Bits<T>::U;
  constexpr int kInFlight = 4;  // words in flight per thread (unaligned arrays)
  // 16-byte words (an aligned array): each thread keeps kDepth words in
  // flight through its own column of a shared ring (cp.async), so the bytes
  // in flight cost no registers
  constexpr bool kStaged = W * sizeof(T) == 16;
  constexpr int kDepth = 8;
  __shared__ __align__(16) uint4 s_ring[kStaged ? kDepth : 1][kBlock];
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
  // Lane l's word slot j holds axis ((t0 + l) W + j) mod D: lanes P apart
  // (P = D / gcd(D, W)) hold the same axes, so a warp first combines its
  // lanes with shuffles P, 2P, 4P, ... apart, leaving P W = lcm(D, W) partial
  // extremes in its first P lanes; one thread per axis then combines the
  // warps' partials.  (Per-thread atomics on the D shared words serialise
  // every thread of the block on a few addresses.)
  constexpr int P = D / gcd_c(D, W);
  constexpr int PW = P * W;
  __shared__ Acc s_part[kWarps][PW];
  __shared__ long long s_mn[D], s_mx[D];
  __shared__ unsigned long long s_ma[D], s_bad;
  if (threadIdx.x < D) {
    s_mn[threadIdx.x] = INT64_MAX;
    s_mx[threadIdx.x] = INT64_MIN;
    s_ma[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  // read == false: the extremes are in fl already (published by the kernel
  // that wrote the points); only the start state and the plan remain
  const int64_t total = read ? n * D : 0;
  const int64_t words = total / W;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t S = nthreads - nthreads % D;  // stride in words, a multiple of D
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Acc acc[W];
  if constexpr (kStaged) {
    if (t < S) {
      const unsigned ring = (unsigned)__cvta_generic_to_shared(&s_ring[0][threadIdx.x]);
      constexpr unsigned kSlot = 16u * kBlock;  // bytes between a thread's slots
#pragma unroll
      for (int p = 0; p < kDepth; ++p) {
        const int64_t qp = t + p * S;
        if (qp < words) cp_async16(ring + p * kSlot, pts + qp * W);
        cp_async_commit();
      }
      int slot = 0;
      for (int64_t q = t; q < words; q += S) {
        cp_async_wait<kDepth - 1>();  // word q has landed in its slot
        U b[W];
        Unpack<T>::get(s_ring[slot][threadIdx.x], b);
#pragma unroll
        for (int j = 0; j < W; ++j) acc[j].add(b[j]);
        // the slot is read (into registers): its next word
        const int64_t qn = q + kDepth * S;
        if (qn < words) cp_async16(ring + slot * kSlot, pts + qn * W);
        cp_async_commit();
        slot = slot + 1 == kDepth ? 0 : slot + 1;
      }
      cp_async_wait<0>();
    }
  } else if (t < S) {
    int64_t q = t;
    for (; q + (kInFlight - 1) * S < words; q += kInFlight * S) {
      U b[kInFlight][W];
#pragma unroll
      for (int u = 0; u < kInFlight; ++u) Word<W, T>::load(pts + (q + u * S) * W, b[u]);
#pragma unroll
      for (int u = 0; u < kInFlight; ++u)
#pragma unroll
        for (int j = 0; j < W; ++j) acc[j].add(b[u][j]);
    }
    for (; q < words; q += S) {
      U b[W];
      Word<W, T>::load(pts + q * W, b);
#pragma unroll
      for (int j = 0; j < W; ++j) acc[j].add(b[j]);
    }
  }
  // threads at or past S hold empty accumulators, which combine as no-ops
  {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = P; o < 32; o <<= 1)
#pragma unroll
      for (int j = 0; j < W; ++j) acc[j].merge(acc[j].shfl_down(o));
    if (lane < P) {
#pragma unroll
      for (int j = 0; j < W; ++j) s_part[w][lane * W + j] = acc[j];
    }
  }
  __syncthreads();
  if (threadIdx.x < D) {
    // warp w's partial e = l W + j belongs to thread t0 + 32 w + l, slot j:
    // axis (base_w + e) mod D with base_w = (t0 + 32 w) W mod D, so axis a
    // has the partials e = (a - base_w) mod D, then every D-th
    const int a = threadIdx.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x;
    Acc r;
    for (int w = 0; w < kWarps; ++w) {
      const int base_w = (int)(((t0 + 32 * w) * W) % D);
      for (int e = (a - base_w + D) % D; e < PW; e += D) r.merge(s_part[w][e]);
    }
    if (!r.empty()) {
      if (r.nonfinite()) {
        atomicAdd(&s_bad, 1ull);
      } else {
        s_mn[a] = r.mn64();
        s_mx[a] = r.mx64();
        s_ma[a] = r.ma64();
      }
    }
  }
  __syncthreads();
  if (t == 0) {
    // values after the last whole word
    for (int64_t e = words * W; e < total; ++e) {
      U b[1];
      Word<1, T>::load(pts + e, b);
      Acc r;
      r.add(b[0]);
      const int a = (int)(e % D);
      if (r.nonfinite()) {
        atomicAdd(&s_bad, 1ull);
      } else {
        atomicMin(&s_mn[a], (long long)r.mn64());
        atomicMax(&s_mx[a], (long long)r.mx64());
        atomicMax(&s_ma[a], (unsigned long long)r.ma64());
      }
    }
  }
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

// The same copy as cp.async 16-byte pieces (global -> shared without a
// register round trip), for the next chunk while the warp works on this one:
// the whole 16-byte pieces of the run, in the calling lane's share.  The rest
// of a run whose size is not a multiple of 16 bytes is copied by
// stage_points_rest once the pieces are waited for.
template <typename T>
__device__ __forceinline__ void stage_points_async(const T* __restrict__ src, int count,
                                                   T* __restrict__ dst, int lane) {
  const int nvec = (int)((size_t)count * sizeof(T) / 16);
  const char* s = reinterpret_cast<const char*>(src);
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  for (int v = lane; v < nvec; v += 32) cp_async16(d + 16u * v, s + 16 * (size_t)v);
}
template <typename T>
__device__ __forceinline__ void stage_points_rest(const T* __restrict__ src, int count,
                                                  T* __restrict__ dst, int lane) {
  const int done = (int)((size_t)count * sizeof(T) / 16 * 16 / sizeof(T));
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

// LISTED: new cells are listed per warp, 32 at a time (the warp's list costs
// registers); else each new cell takes one add on the cell count.
// Tuning::bin_list chooses.
//
// SUMS: binning also forms the exact cell sums of Sec. 2.1 i (else a counting
// sort does, after it).  A coordinate's fixed-point value (units of 2^L_a,
// 128-bit two's complement) is cut into six 24-bit pieces; the lanes that
// share a cell add each piece with one warp reduction over their match mask
// (32 pieces of 24 bits fit 29 bits), and the group's first lane adds the
// reassembled sum (mod 2^128) into the cell's limb accumulators, which are
// indexed by the cell's table slot.  Exact integer sums make the grouping and
// the order of the adds irrelevant.  Tuning::bin_sums chooses.
constexpr unsigned bin_blocks_per_sm(bool listed, bool sums) {
  return sums ? 4u : (listed ? 5u : 6u);
}

template <int D, typename T, bool LISTED, bool SUMS>
__global__ void __launch_bounds__(kBlock, bin_blocks_per_sm(LISTED, SUMS))
    k_bin(const T* __restrict__ pts, int64_t n, const int64_t* __restrict__ thr,
          BinTable T0, uint32_t mask0, uint32_t maxcells, uint32_t* __restrict__ slot0,
          DevFlags* fl, bool vec_ok, const int64_t* __restrict__ offsets, int B,
          const SweepPlan* __restrict__ sweep, uint32_t n0) {
  // a warp's chunk of 32 points, double-buffered: with a 16-byte aligned
  // array the next chunk is copied (cp.async) while this one is worked on
  __shared__ __align__(16) T s_pts[kWarps][2][32 * D];
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
  unsigned inexact = 0, werr = 0;  // SUMS: values outside the fixed-point window
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
  const bool pipe = !sweep && vec_ok;
  const int64_t step = nwarps * 32;
  if (pipe && gwarp * 32 < n) {
    const int64_t b0 = gwarp * 32;
    stage_points_async<T>(pts + b0 * D, (n - b0 < 32 ? (int)(n - b0) : 32) * D, s_pts[w][0], lane);
    cp_async_commit();
  }
  int par = 0;
  for (int64_t base = gwarp * 32; base < n; base += step, par ^= 1) {
    const int cnt = n - base < 32 ? (int)(n - base) : 32;
    T* const cur = s_pts[w][par];
    if (pipe) {
      const int64_t nb = base + step;
      if (nb < n)
        stage_points_async<T>(pts + nb * D, (n - nb < 32 ? (int)(n - nb) : 32) * D,
                              s_pts[w][par ^ 1], lane);
      cp_async_commit();
      cp_async_wait<1>();  // this chunk's pieces have landed
      stage_points_rest<T>(pts + base * D, cnt * D, cur, lane);
    } else if (!sweep) {
      stage_points<T>(pts + base * D, cnt * D, cur, vec_ok, lane);
    }
    __syncwarp();
    const bool valid = lane < cnt;
    uint64_t key = kEmpty;
    const T* row = nullptr;  // a sweep's point row
    if (valid && sweep) {
      // bandwidth sweep: point j of instance b is row j of pts, its cell
      // decided with b's bandwidth
      const int64_t i = base + lane;
      const uint32_t b = (uint32_t)(i / n0);
      row = pts + (size_t)(i - (int64_t)b * n0) * D;
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
        const uint64_t b = bits_of(cur[lane * D + a]);
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
    if constexpr (SUMS) {
#pragma unroll 1
      for (int a = 0; a < D; ++a) {
        uint64_t bits = 0;
        if (valid) bits = sweep ? bits_of(__ldg(row + a)) : bits_of(cur[lane * D + a]);
        const u128 V = valid ? to_fixed(bits, P.L[a], inexact, werr) : (u128)0;
        u128 G = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const uint32_t piece = (uint32_t)(V >> (24 * j)) & 0xFFFFFFu;
          if (__any_sync(kFull, piece != 0u)) G += (u128)__reduce_add_sync(peers, piece) << (24 * j);
        }
        if (lane == leader && s != kNone) atomic_add_fixed(T0.acc + ((size_t)s * D + a) * 4, G);
      }
    }
    __syncwarp();
  }
  if (LISTED && pend) list_cells(pend);
  if constexpr (SUMS) {
    if (inexact) atomicAdd(&fl->inexact, 1ull);
    if (werr) atomicOr(&fl->err, kErrWindow);
  }
}

// Pixel features of an image (the (r, g, b) or (r, g, b, x, y) inputs of the
// segmentation experiment, Sec. 4.2): pixel p of a row-major image of width
// w is the point (c_0 .. c_{C-1}[, x s, y s]), x = p mod w, y = p div w.  A
// warp takes 32 consecutive pixels at a time: each lane builds its pixel's
// row in the warp's slice of shared memory, and the warp writes the 32 rows
// out as one contiguous run (consecutive lanes write consecutive values,
// whole 128-byte lines).  Warps synchronise only with themselves.
//
// The channel count and the position flag are template parameters: a
// runtime loop over up to eight channels issued every channel's
// instructions, predicated off or not.
//
// No float64 instruction runs per pixel (GB300's float64 pipe issues about
// one lane-operation per clock per SM, which bounded a per-pixel
// conversion-and-multiply version at 7 clocks a pixel): a channel byte
// becomes a double through its bit pattern (u32_to_f64_bits), and the
// positions' products x s and y s come from a table of the W + H products
// that k_axis_products computes once per image.
//
// With fl, the kernel also publishes the key range of the features it writes
// (what k_range would find reading them back): each thread keeps the least
// and greatest channel byte (packed four to a word, compared byte by byte)
// and column and row index it has seen, as integers; a channel's extremes as
// float64 are those bytes, and a position's are the table's products of the
// extreme indices, since x -> x s rounded is monotone for s > 0.  Warps combine with shuffles, blocks in shared memory, and
// a block publishes an extreme only where it improves on the one already
// published (most blocks publish nothing once the image's extremes are in).
constexpr int kImgMaxC = 8;
constexpr int kImgMaxD = kImgMaxC + 2;

// Per-byte extremes of four channel bytes in a word.
__device__ __forceinline__ unsigned min_bytes(unsigned a, unsigned b) { return __vminu4(a, b); }
__device__ __forceinline__ unsigned max_bytes(unsigned a, unsigned b) { return __vmaxu4(a, b); }

// tab[x] = x s for the W columns, then tab[W + y] = y s for the H rows: the
// rounded products the features hold.
__global__ void __launch_bounds__(kBlock) k_axis_products(int64_t W, int64_t H, double s,
                                                           double* __restrict__ tab) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < W + H;
       i += (int64_t)gridDim.x * blockDim.x)
    tab[i] = (double)(i < W ? i : i - W) * s;
}

__device__ __forceinline__ double exact_double(uint32_t v) {
  return __longlong_as_double((long long)u32_to_f64_bits(v));
}

template <int C, bool XY>
__global__ void __launch_bounds__(kBlock) k_image_features(const uint8_t* __restrict__ px,
                                                            int64_t n, int64_t width,
                                                            const double* __restrict__ tab,
                                                            double* __restrict__ out,
                                                            DevFlags* fl) {
  constexpr int d = C + (XY ? 2 : 0);
  __shared__ double s_rows[kWarps][32 * d];
  // per warp: channel-byte minima (two words), maxima (two), then the least
  // and greatest column and row index
  __shared__ unsigned s_ext[kWarps][8];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double* rows = s_rows[wp];
  // (bytes of absent channels are kept too, and never read)
  unsigned lo0 = 0xFFFFFFFFu, lo1 = 0xFFFFFFFFu, hi0 = 0, hi1 = 0;
  unsigned xlo = 0xFFFFFFFFu, xhi = 0, ylo = 0xFFFFFFFFu, yhi = 0;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p0 = gwarp * 32; p0 < n; p0 += nwarps * 32) {
    const int cnt = n - p0 < 32 ? (int)(n - p0) : 32;
    if (lane < cnt) {
      const int64_t p = p0 + lane;
      double* r = rows + lane * d;
      unsigned w0 = 0, w1 = 0;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const unsigned v = __ldg(px + p * C + c);
        r[c] = exact_double(v);
        if (c < 4)
          w0 |= v << (8 * c);
        else
          w1 |= v << (8 * (c - 4));
      }
      lo0 = min_bytes(lo0, w0);
      hi0 = max_bytes(hi0, w0);
      if (C > 4) {
        lo1 = min_bytes(lo1, w1);
        hi1 = max_bytes(hi1, w1);
      }
      if (XY) {  // p and width are below 2^31
        const uint32_t y = (uint32_t)p / (uint32_t)width;
        const uint32_t x = (uint32_t)p - y * (uint32_t)width;
        r[C] = __ldg(tab + x);
        r[C + 1] = __ldg(tab + width + y);
        xlo = x < xlo ? x : xlo;
        xhi = x > xhi ? x : xhi;
        ylo = y < ylo ? y : ylo;
        yhi = y > yhi ? y : yhi;
      }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < d; ++k) {
      const int e = lane + 32 * k;
      if (e < cnt * d) out[p0 * d + e] = rows[e];
    }
    __syncwarp();
  }
  if (!fl) return;
  // every lane of every warp reaches this point (the loop is warp-uniform)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo0 = min_bytes(lo0, __shfl_xor_sync(kFull, lo0, o));
    lo1 = min_bytes(lo1, __shfl_xor_sync(kFull, lo1, o));
    hi0 = max_bytes(hi0, __shfl_xor_sync(kFull, hi0, o));
    hi1 = max_bytes(hi1, __shfl_xor_sync(kFull, hi1, o));
  }
  xlo = __reduce_min_sync(kFull, xlo);
  xhi = __reduce_max_sync(kFull, xhi);
  ylo = __reduce_min_sync(kFull, ylo);
  yhi = __reduce_max_sync(kFull, yhi);
  if (lane == 0) {
    s_ext[wp][0] = lo0;
    s_ext[wp][1] = lo1;
    s_ext[wp][2] = hi0;
    s_ext[wp][3] = hi1;
    s_ext[wp][4] = xlo;
    s_ext[wp][5] = xhi;
    s_ext[wp][6] = ylo;
    s_ext[wp][7] = yhi;
  }
  __syncthreads();
  if (threadIdx.x < d) {
    const int a = threadIdx.x;
    unsigned vlo = 0xFFFFFFFFu, vhi = 0;
    bool seen = false;  // a warp of the block wrote a pixel
    for (int q = 0; q < kWarps; ++q) {
      unsigned l, h;
      if (a < C) {
        const int sh = 8 * (a & 3);
        l = (s_ext[q][a >> 2] >> sh) & 0xFFu;
        h = (s_ext[q][2 + (a >> 2)] >> sh) & 0xFFu;
      } else {
        l = s_ext[q][a == C ? 4 : 6];
        h = s_ext[q][a == C ? 5 : 7];
      }
      // a warp that wrote no pixel still holds minima 0xFF and maxima 0
      if (l > h) continue;
      seen = true;
      vlo = l < vlo ? l : vlo;
      vhi = h > vhi ? h : vhi;
    }
    if (seen) {
      const int64_t t0 = a == C ? 0 : width;  // the products of columns, then of rows
      const double vmin = a < C ? exact_double(vlo) : __ldg(tab + t0 + vlo);
      const double vmax = a < C ? exact_double(vhi) : __ldg(tab + t0 + vhi);
      RangeAcc<double> r;
      r.add((uint64_t)__double_as_longlong(vmin));
      r.add((uint64_t)__double_as_longlong(vmax));
      if (r.nonfinite()) {
        atomicAdd(&fl->bad, 1ull);
      } else {
        const long long mn = r.mn64(), mx = r.mx64();
        const unsigned long long ma = r.ma64();
        if (mn < *(volatile long long*)&fl->min_ord[a]) atomicMin(&fl->min_ord[a], mn);
        if (mx > *(volatile long long*)&fl->max_ord[a]) atomicMax(&fl->max_ord[a], mx);
        if (ma > *(volatile unsigned long long*)&fl->maxabs[a]) atomicMax(&fl->maxabs[a], ma);
      }
    }
  }
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
                         const PlanJob* job, cudaStream_t s, bool read) {
  const bool vec = ((uintptr_t)pts & 15u) == 0;
  const int W = vec ? (f32 ? 4 : 2) : 1;
  // without the read, one block per SM clears the start state
  const unsigned g = read ? grid_for(n * d / W, kBlock * 4, 152u * kRangeBlocksPerSM) : 152u;
  const bool plan = job != nullptr;
  if (!read && !plan) return cudaErrorInvalidValue;
  const PlanJob J = plan ? *job : PlanJob{};
  if (f32) {
    if (vec) {
      GS_DISPATCH_D(d, k_range<D, float, 4><<<g, kBlock, 0, s>>>((const float*)pts, n, fl, plan, J, read));
    } else {
      GS_DISPATCH_D(d, k_range<D, float, 1><<<g, kBlock, 0, s>>>((const float*)pts, n, fl, plan, J, read));
    }
  } else {
    if (vec) {
      GS_DISPATCH_D(d, k_range<D, double, 2><<<g, kBlock, 0, s>>>((const double*)pts, n, fl, plan, J, read));
    } else {
      GS_DISPATCH_D(d, k_range<D, double, 1><<<g, kBlock, 0, s>>>((const double*)pts, n, fl, plan, J, read));
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_bin(const void* pts, bool f32, int64_t n, int d, const int64_t* thr,
                       BinTable T0, uint32_t mask0, uint32_t maxcells, uint32_t* slot0,
                       DevFlags* fl, const int64_t* offsets, int B, const SweepPlan* sweep,
                       uint32_t n0, bool listed, bool sums, cudaStream_t s) {
  const unsigned g = grid_for((n + 31) / 32 * 32, kBlock, 152u * bin_blocks_per_sm(listed, sums));
  const bool vec_ok = ((uintptr_t)pts & 15u) == 0;
  if (sweep && n0 == 0) return cudaErrorInvalidValue;
#define GS_BIN(T, LST, SUM)                                                                    \
  GS_DISPATCH_D(d, (k_bin<D, T, LST, SUM><<<g, kBlock, 0, s>>>((const T*)pts, n, thr, T0, mask0, \
                                                               maxcells, slot0, fl, vec_ok,      \
                                                               offsets, B, sweep, n0)))
#define GS_BIN_T(T)                                              \
  if (sums) {                                                    \
    if (listed) { GS_BIN(T, true, true); } else { GS_BIN(T, false, true); }   \
  } else {                                                       \
    if (listed) { GS_BIN(T, true, false); } else { GS_BIN(T, false, false); } \
  }
  if (f32) {
    GS_BIN_T(float)
  } else {
    GS_BIN_T(double)
  }
#undef GS_BIN_T
#undef GS_BIN
  return cudaGetLastError();
}

cudaError_t launch_axis_products(int64_t W, int64_t H, double s, double* tab, cudaStream_t st) {
  if (W < 1 || H < 0) return cudaErrorInvalidValue;
  k_axis_products<<<grid_for(W + H, kBlock, 152u), kBlock, 0, st>>>(W, H, s, tab);
  return cudaGetLastError();
}

template <int C, bool XY>
static cudaError_t launch_image_features_c(const uint8_t* px, int64_t n, int64_t width,
                                           const double* tab, double* out, DevFlags* fl,
                                           cudaStream_t st) {
  // one wave: as many blocks as are resident at once (queried once)
  static std::atomic<int> s_per_sm{0};
  int per_sm = s_per_sm.load(std::memory_order_relaxed);
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_image_features<C, XY>, kBlock, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    s_per_sm.store(per_sm, std::memory_order_relaxed);
  }
  const unsigned g = grid_for(n, kBlock, 152u * (unsigned)per_sm);
  k_image_features<C, XY><<<g, kBlock, 0, st>>>(px, n, width, tab, out, fl);
  return cudaGetLastError();
}

template <int C>
static cudaError_t launch_image_features_xy(const uint8_t* px, int64_t n, int64_t width, bool xy,
                                            const double* tab, double* out, DevFlags* fl,
                                            cudaStream_t st) {
  return xy ? launch_image_features_c<C, true>(px, n, width, tab, out, fl, st)
            : launch_image_features_c<C, false>(px, n, width, tab, out, fl, st);
}

cudaError_t launch_image_features(const uint8_t* px, int64_t n, int64_t width, int C, bool xy,
                                  const double* tab, double* out, DevFlags* fl, cudaStream_t st) {
  if (C < 1 || C > kImgMaxC || (xy && (width < 1 || !tab))) return cudaErrorInvalidValue;
  if (fl && C + (xy ? 2 : 0) > kMaxD) return cudaErrorInvalidValue;
  if (n == 0) return cudaSuccess;
  switch (C) {
    case 1: return launch_image_features_xy<1>(px, n, width, xy, tab, out, fl, st);
    case 2: return launch_image_features_xy<2>(px, n, width, xy, tab, out, fl, st);
    case 3: return launch_image_features_xy<3>(px, n, width, xy, tab, out, fl, st);
    case 4: return launch_image_features_xy<4>(px, n, width, xy, tab, out, fl, st);
    case 5: return launch_image_features_xy<5>(px, n, width, xy, tab, out, fl, st);
    case 6: return launch_image_features_xy<6>(px, n, width, xy, tab, out, fl, st);
    case 7: return launch_image_features_xy<7>(px, n, width, xy, tab, out, fl, st);
    default: return launch_image_features_xy<8>(px, n, width, xy, tab, out, fl, st);
  }
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
