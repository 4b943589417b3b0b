// gs_kernels.cu -- the GridShift hot path on sm_103a.
//
// Steps (Kumar et al., arXiv 2206.02200, Sec. 2.1 and Algorithm 1):
//   k_range     key range, fixed-point window and finiteness of the input
//   k_bin       step i: cell key of every point, per-cell count and exact sum
//   k_compact0  active-cell list of level 0 and its lookup table
//   k_gather    steps ii-iii: Eq. 1-2 over the 3^d neighbours (parallel form,
//               Eq. 6), rounded centroid, new key, neighbour flag (step v)
//   k_merge     step iv: cells sharing a new key add counts and count-weighted
//               centroids (Eq. 3-4) exactly, in a fresh table
//   k_compact   active-cell list of the next level
//   k_finish    parent of every cell in the forest of merges (the union of
//               resident sets of Eq. 4), and reset of the used table
//   k_jump      pointer jumping over that forest: the final cell of every
//               initial cell
//   k_labels    the label of every point
#include <cstdio>

#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {

constexpr int kBlock = 256;

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

template <int D, typename T>
__global__ void __launch_bounds__(kBlock)
    k_bin(const T* __restrict__ pts, int64_t n, Plan P, const int64_t* __restrict__ thr,
          Table T0, uint32_t mask0, uint32_t maxcells, uint32_t* __restrict__ slot0,
          DevFlags* fl) {
  unsigned inexact = 0, werr = 0;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint64_t b[D];
    uint64_t key = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      b[a] = load_bits<T>(pts + i * D + a);
      int idx = key_index(thr + P.thr_off[a], P.span[a], ord_of_bits(b[a]));
      key |= (uint64_t)(idx + 1) << P.off[a];
    }
    bool won;
    uint32_t s = table_insert(T0.key, mask0, key, won, &fl->err);
    if (s == kNone) continue;
    if (won) {
      uint32_t id = atomicAdd(&fl->m0, 1u);
      if (id < maxcells) T0.list[id] = s; else atomicOr(&fl->err, kErrOverflow);
    }
    atomicAdd(&T0.cnt[s], 1u);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      u128 V = to_fixed(b[a], P.L[a], inexact, werr);
      atomic_add_fixed(T0.acc + ((size_t)s * D + a) * 4, V);
    }
    slot0[i] = s;
  }
  if (inexact) atomicAdd(&fl->inexact, 1ull);
  if (werr) atomicOr(&fl->err, kErrWindow);
}

// ---------------------------------------------------------------------------
// Level 0: cell list and lookup table

template <int D>
__global__ void __launch_bounds__(kBlock)
    k_compact0(Plan P, Table T0, Cells c0, Table A, uint32_t capA, IterState* st,
               DevFlags* fl) {
  uint32_t m0 = fl->m0;
  uint32_t maskA = mask_for(m0, capA);
  uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0) {
    st[0].m = m0;
    st[0].mask = maskA;
    st[0].base = 0;
  }
  unsigned inexact = 0;
  for (uint32_t id = tid; id < m0; id += gridDim.x * blockDim.x) {
    uint32_t s = T0.list[id];
    uint64_t key = T0.key[s];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      uint64_t* acc = T0.acc + ((size_t)s * D + a) * 4;
      c0.cs[(size_t)id * D + a] = round_fixed(limbs_value(acc), P.L[a], inexact);
      acc[0] = acc[1] = acc[2] = acc[3] = 0;
    }
    c0.key[id] = key;
    c0.cnt[id] = T0.cnt[s];
    T0.cnt[s] = 0;
    T0.key[s] = kEmpty;
    T0.id[s] = id;
    bool won;
    uint32_t sa = table_insert(A.key, maskA, key, won, &fl->err);
    if (sa != kNone) {
      A.id[sa] = id;
      A.list[id] = sa;
    }
  }
  if (inexact) atomicAdd(&fl->inexact, 1ull);
}

// ---------------------------------------------------------------------------
// Steps ii-iii (and the test of step v): one warp per cell

template <int D>
__global__ void __launch_bounds__(kBlock)
    k_gather(Plan P, const int64_t* __restrict__ thr, const uint64_t* __restrict__ dtab,
             Table G, Cells c, double* __restrict__ sp, uint64_t* __restrict__ nkey,
             IterState* st, int t, DevFlags* fl) {
  const uint32_t m = st[t].m;
  const uint32_t mask = st[t].mask;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned inexact = 0, werr = 0;
  bool any_nb = false;
  for (uint32_t j = warp; j < m; j += nwarps) {
    const uint64_t key = c.key[j];
    uint32_t Dc = 0;
    u128 N[D];
#pragma unroll
    for (int a = 0; a < D; ++a) N[a] = 0;
    for (int p = lane; p < P.nprobe; p += 32) {
      uint64_t q = key + __ldg(&dtab[p]);
      uint32_t s = table_find(G.key, mask, q);
      if (s == kNone) continue;
      uint32_t id = G.id[s];
      Dc += c.cnt[id];
#pragma unroll
      for (int a = 0; a < D; ++a)
        N[a] += to_fixed((uint64_t)__double_as_longlong(c.cs[(size_t)id * D + a]), P.L[a],
                         inexact, werr);
      if (p != P.center) any_nb = true;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Dc += __shfl_xor_sync(kFull, Dc, o);
#pragma unroll
      for (int a = 0; a < D; ++a) N[a] += shfl_xor_u128(N[a], o);
    }
    uint64_t field = 0;
    if (lane < D) {
      u128 Na = 0;
      int La = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a == lane) {
          Na = N[a];
          La = P.L[a];
        }
      double s = div_round(Na, Dc, La, inexact);
      sp[(size_t)j * D + lane] = s;
      int idx = key_index(thr + P.thr_off[lane], P.span[lane],
                          ord_of_bits((uint64_t)__double_as_longlong(s)));
      field = (uint64_t)(idx + 1) << P.off[lane];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) field |= __shfl_xor_sync(kFull, field, o);
    if (lane == 0) nkey[j] = field;
  }
  if (__any_sync(kFull, any_nb) && lane == 0) st[t].has_nb = 1u;
  if (inexact) atomicAdd(&fl->inexact, 1ull);
  if (werr) atomicOr(&fl->err, kErrWindow);
}

// ---------------------------------------------------------------------------
// Step iv: merge cells that share a key (Eq. 3-4)

template <int D>
__global__ void __launch_bounds__(kBlock)
    k_merge(Plan P, Cells c, const double* __restrict__ sp, const uint64_t* __restrict__ nkey,
            Table M, uint32_t* __restrict__ pslot, IterState* st, int t, DevFlags* fl) {
  const uint32_t m = st[t].m;
  const uint32_t maskM = mask_for(m, M.cap);
  uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0) {
    st[t + 1].mask = maskM;
    st[t + 1].base = st[t].base + m;
  }
  unsigned inexact = 0, werr = 0;
  for (uint32_t j = tid; j < m; j += gridDim.x * blockDim.x) {
    bool won;
    uint32_t s = table_insert(M.key, maskM, nkey[j], won, &fl->err);
    if (s == kNone) continue;
    if (won) {
      uint32_t id = atomicAdd(&st[t + 1].m, 1u);
      M.list[id] = s;
    }
    uint32_t cnt = c.cnt[j];
    atomicAdd(&M.cnt[s], cnt);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      u128 V = to_fixed((uint64_t)__double_as_longlong(sp[(size_t)j * D + a]), P.L[a], inexact,
                        werr);
      atomic_add_fixed(M.acc + ((size_t)s * D + a) * 4, V * (u128)cnt);
    }
    pslot[j] = s;
  }
  if (inexact) atomicAdd(&fl->inexact, 1ull);
  if (werr) atomicOr(&fl->err, kErrWindow);
}

template <int D>
__global__ void __launch_bounds__(kBlock)
    k_compact(Plan P, Table M, Cells next, IterState* st, int t, DevFlags* fl) {
  const uint32_t m1 = st[t + 1].m;
  unsigned inexact = 0;
  for (uint32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < m1;
       id += gridDim.x * blockDim.x) {
    uint32_t s = M.list[id];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      uint64_t* acc = M.acc + ((size_t)s * D + a) * 4;
      next.cs[(size_t)id * D + a] = round_fixed(limbs_value(acc), P.L[a], inexact);
      acc[0] = acc[1] = acc[2] = acc[3] = 0;
    }
    next.key[id] = M.key[s];
    next.cnt[id] = M.cnt[s];
    M.cnt[s] = 0;
    M.id[s] = id;
  }
  if (inexact) atomicAdd(&fl->inexact, 1ull);
}

__global__ void k_finish(Table G, Table M, const uint32_t* __restrict__ pslot,
                         uint32_t* __restrict__ forest, IterState* st, int t) {
  const uint32_t m = st[t].m;
  const uint32_t base = st[t].base, base1 = st[t + 1].base;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    forest[base + j] = base1 + M.id[pslot[j]];
    G.key[G.list[j]] = kEmpty;
  }
}

__global__ void k_final_level(Table G, uint32_t* __restrict__ forest, IterState* st, int T) {
  const uint32_t m = st[T].m;
  const uint32_t base = st[T].base;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    forest[base + j] = base + j;
    G.key[G.list[j]] = kEmpty;
  }
}

__global__ void k_jump(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                       uint32_t nodes) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nodes; v += gridDim.x * blockDim.x)
    out[v] = in[in[v]];
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

__global__ void k_label_slots(const uint32_t* __restrict__ list0, const uint32_t* __restrict__ root,
                              const uint32_t* __restrict__ rank, uint32_t baseT,
                              uint32_t* __restrict__ labslot, uint32_t m0) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m0; c += gridDim.x * blockDim.x)
    labslot[list0[c]] = rank[root[c] - baseT];
}

__global__ void k_labels(const uint32_t* __restrict__ slot0, const uint32_t* __restrict__ labslot,
                         int32_t* __restrict__ labels, int64_t n) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    labels[i] = (int32_t)labslot[slot0[i]];
}

__global__ void k_modes(Cells c, const uint32_t* __restrict__ rank, double* __restrict__ modes,
                        uint32_t k, int d) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < k; r += gridDim.x * blockDim.x) {
    uint32_t rr = rank[r];
    double cnt = (double)c.cnt[r];
    for (int a = 0; a < d; ++a) modes[(size_t)rr * d + a] = c.cs[(size_t)r * d + a] / cnt;
  }
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
  unsigned g = grid_for(n);
  if (f32) {
    GS_DISPATCH_D(P.d, k_bin<D, float><<<g, kBlock, 0, s>>>((const float*)pts, n, P, thr, T0,
                                                            mask0, maxcells, slot0, fl));
  } else {
    GS_DISPATCH_D(P.d, k_bin<D, double><<<g, kBlock, 0, s>>>((const double*)pts, n, P, thr, T0,
                                                             mask0, maxcells, slot0, fl));
  }
  return cudaGetLastError();
}

cudaError_t launch_compact0(const Plan& P, Table T0, Cells c0, Table A, uint32_t capA,
                            uint32_t m0_bound, IterState* st, DevFlags* fl, cudaStream_t s) {
  unsigned g = grid_for(m0_bound);
  GS_DISPATCH_D(P.d, k_compact0<D><<<g, kBlock, 0, s>>>(P, T0, c0, A, capA, st, fl));
  return cudaGetLastError();
}

cudaError_t launch_gather(const Plan& P, const int64_t* thr, const uint64_t* dtab, Table G,
                          Cells c, double* sp, uint64_t* nkey, IterState* st, int t,
                          uint32_t m_bound, DevFlags* fl, cudaStream_t s) {
  unsigned g = grid_for((int64_t)m_bound * 32);
  GS_DISPATCH_D(P.d, k_gather<D><<<g, kBlock, 0, s>>>(P, thr, dtab, G, c, sp, nkey, st, t, fl));
  return cudaGetLastError();
}

cudaError_t launch_merge(const Plan& P, Cells c, const double* sp, const uint64_t* nkey,
                         Table M, uint32_t* pslot, IterState* st, int t, uint32_t m_bound,
                         DevFlags* fl, cudaStream_t s) {
  unsigned g = grid_for(m_bound);
  GS_DISPATCH_D(P.d, k_merge<D><<<g, kBlock, 0, s>>>(P, c, sp, nkey, M, pslot, st, t, fl));
  return cudaGetLastError();
}

cudaError_t launch_compact(const Plan& P, Table M, Cells next, IterState* st, int t,
                           uint32_t m_bound, DevFlags* fl, cudaStream_t s) {
  unsigned g = grid_for(m_bound);
  GS_DISPATCH_D(P.d, k_compact<D><<<g, kBlock, 0, s>>>(P, M, next, st, t, fl));
  return cudaGetLastError();
}

cudaError_t launch_finish(Table G, Table M, const uint32_t* pslot, uint32_t* forest,
                          IterState* st, int t, uint32_t m_bound, cudaStream_t s) {
  k_finish<<<grid_for(m_bound), kBlock, 0, s>>>(G, M, pslot, forest, st, t);
  return cudaGetLastError();
}

cudaError_t launch_final_level(Table G, uint32_t* forest, IterState* st, int T,
                               uint32_t m_bound, cudaStream_t s) {
  k_final_level<<<grid_for(m_bound), kBlock, 0, s>>>(G, forest, st, T);
  return cudaGetLastError();
}

cudaError_t launch_jump(const uint32_t* in, uint32_t* out, uint32_t nodes, cudaStream_t s) {
  k_jump<<<grid_for(nodes), kBlock, 0, s>>>(in, out, nodes);
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

cudaError_t launch_label_slots(const uint32_t* list0, const uint32_t* root, const uint32_t* rank,
                               uint32_t baseT, uint32_t* labslot, uint32_t m0, cudaStream_t s) {
  k_label_slots<<<grid_for(m0), kBlock, 0, s>>>(list0, root, rank, baseT, labslot, m0);
  return cudaGetLastError();
}

cudaError_t launch_labels(const uint32_t* slot0, const uint32_t* labslot, int32_t* labels,
                          int64_t n, cudaStream_t s) {
  k_labels<<<grid_for(n), kBlock, 0, s>>>(slot0, labslot, labels, n);
  return cudaGetLastError();
}

cudaError_t launch_modes(Cells c, const uint32_t* rank, double* modes, uint32_t k, int d,
                         cudaStream_t s) {
  k_modes<<<grid_for(k), kBlock, 0, s>>>(c, rank, modes, k, d);
  return cudaGetLastError();
}

}  // namespace gs
