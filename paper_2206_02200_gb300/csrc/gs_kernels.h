// gs_kernels.h -- host-callable launchers of the GridShift kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gs_plan.h"

namespace gs {

// A hash table of packed cell keys with per-slot payload.  key[] is kEmpty
// where free; cnt[] and acc[] (d x 4 limb accumulators per slot) are zero
// where free.  list[i] is the slot of the i-th key inserted (in arrival order).
struct Table {
  uint64_t* key;
  uint32_t* id;
  uint32_t* cnt;
  uint64_t* acc;
  uint32_t* list;
  uint32_t cap;  // power of two
};

// The active cells of one level: packed key, resident count and coordinate
// sum (row-major m x d, float64).
struct Cells {
  uint64_t* key;
  uint32_t* cnt;
  double* cs;
};

cudaError_t launch_range(const void* pts, bool f32, int64_t n, int d, DevFlags* fl,
                         cudaStream_t s);
cudaError_t launch_bin(const void* pts, bool f32, int64_t n, const Plan& P, const int64_t* thr,
                       Table T0, uint32_t mask0, uint32_t maxcells, uint32_t* slot0,
                       DevFlags* fl, cudaStream_t s);
cudaError_t launch_compact0(const Plan& P, Table T0, Cells c0, Table A, uint32_t capA,
                            uint32_t m0_bound, IterState* st, DevFlags* fl, cudaStream_t s);
cudaError_t launch_gather(const Plan& P, const int64_t* thr, const uint64_t* dtab, Table G,
                          Cells c, double* sp, uint64_t* nkey, IterState* st, int t,
                          uint32_t m_bound, DevFlags* fl, cudaStream_t s);
cudaError_t launch_merge(const Plan& P, Cells c, const double* sp, const uint64_t* nkey,
                         Table M, uint32_t* pslot, IterState* st, int t, uint32_t m_bound,
                         DevFlags* fl, cudaStream_t s);
cudaError_t launch_compact(const Plan& P, Table M, Cells next, IterState* st, int t,
                           uint32_t m_bound, DevFlags* fl, cudaStream_t s);
cudaError_t launch_finish(Table G, Table M, const uint32_t* pslot, uint32_t* forest,
                          IterState* st, int t, uint32_t m_bound, cudaStream_t s);
cudaError_t launch_final_level(Table G, uint32_t* forest, IterState* st, int T,
                               uint32_t m_bound, cudaStream_t s);
cudaError_t launch_jump(const uint32_t* in, uint32_t* out, uint32_t nodes, cudaStream_t s);
cudaError_t launch_iota_keys(Cells c, uint64_t* keys, uint32_t* vals, uint32_t k,
                             cudaStream_t s);
cudaError_t launch_rank(const uint32_t* sorted_vals, uint32_t* rank, uint32_t k, cudaStream_t s);
cudaError_t launch_label_slots(const uint32_t* list0, const uint32_t* root, const uint32_t* rank,
                               uint32_t baseT, uint32_t* labslot, uint32_t m0, cudaStream_t s);
cudaError_t launch_labels(const uint32_t* slot0, const uint32_t* labslot, int32_t* labels,
                          int64_t n, cudaStream_t s);
cudaError_t launch_modes(Cells c, const uint32_t* rank, double* modes, uint32_t k, int d,
                         cudaStream_t s);

// Stable LSD radix sort of (key, val) pairs by key bits [0, nbits).  keys/vals
// hold the input and receive the output; tkeys/tvals are scratch of the same
// size; hist needs radix_hist_words(n) words.
size_t radix_hist_words(uint32_t n);
int radix_sort_launches(uint32_t n, int nbits);  // kernels one radix_sort call launches
cudaError_t radix_sort(uint64_t* keys, uint32_t* vals, uint64_t* tkeys, uint32_t* tvals,
                       uint32_t* hist, uint32_t n, int nbits, cudaStream_t s);

}  // namespace gs
