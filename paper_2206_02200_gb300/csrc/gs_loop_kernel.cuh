// gs_loop_kernel.cuh -- the label writes, the launches of binning's second
// pass, the cooperative loop kernel and the launch helpers.  One part of the
// loop kernel of gs_loop.cuh, which includes the parts in order.
#pragma once

#include "gs_loop_tail.cuh"

namespace gs {

namespace {
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
  return A.n >= (int64_t)A.tune.split_min && A.tune.bin_sums == 0u &&
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
  // step i, second pass (the exact cell sums), unless binning formed them: in
  // the k_prep_* launches before this kernel when the run has split_min
  // points or more, else here
  const bool split = A.n >= (int64_t)A.tune.split_min;
  if (!split && !A.tune.bin_sums) {
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
    // one flag add per block (atomics on one address from different warps
    // serialise; 152 instead of up to 2432 per step)
    if (__syncthreads_or(any_nb ? 1 : 0) && threadIdx.x == 0) atomicOr(&A.st[t].has_nb, 1u);
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
