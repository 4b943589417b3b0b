// gs_kernels.h -- host-callable launchers of the GridShift kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gs_plan.h"

namespace gs {

// The binning table of step i: packed cell keys with, per slot, the resident
// count, the offset of the cell's run in the counting sort of the points and
// the cell's id (its arrival order).  list[i] is the slot of the cell with
// id i.  acc holds, per cell id, the exact coordinate sums (d x 4 limb
// accumulators; float sums in the float32 variant).  key[] is kEmpty where
// free; cnt[] and acc[] are zero where unused (off[] and id[] need no
// clearing).
struct BinTable {
  uint64_t* key;
  uint32_t* cnt;
  uint32_t* off;
  uint32_t* id;
  uint64_t* acc;   // cap x d x 4: the exact sums' limb accumulators, by cell id (the
                   // counting sort) or by slot (sums formed in binning); float32
                   // variant with a counting sort: d float sums of offsets per id
  uint32_t* list;  // maxcells
  uint32_t cap;    // power of two
};

// A table of the cells of one level, also the merge target of the update
// that creates the next level.  Per slot:
//   key  packed cell key (kEmpty where free)
//   id   the cell's index in the level's cell list
//   row  d + 1 pairs of 64-bit words: row[0].x = resident count, row[1 + a] =
//        the cell's coordinate sum of axis a (the float64 value of Sec. 2.1,
//        an exact sum rounded once) as the two's-complement 128-bit integer it
//        equals in units of 2^L_a, {low word, high word}
//   acc  d x 4 limb accumulators of exact sums while the table is a merge
//        target (zero otherwise)
// A clean table has every key empty, every row[0] and every acc zero.
// list[i] is the slot of the level's i-th cell.
struct LevelTable {
  uint64_t* key;
  uint32_t* id;
  ulonglong2* row;
  uint64_t* acc;
  uint32_t* list;
  uint32_t cap;  // power of two
};

// Least d for the second stage of the pencil form of step 0 (the loop
// kernel), which needs the second pencil table (LoopArgs::ptab).
constexpr int kPencil2MinD = 6;

// Occupancy filter of a level (see the loop kernel): at most 2^20 bits.
constexpr int kFilterLog2Max = 20;
constexpr uint32_t kFilterWords = (1u << kFilterLog2Max) / 32;

// The active cells of one level, in list order: packed key and resident count.
struct Cells {
  uint64_t* key;
  uint32_t* cnt;
};

// Everything the persistent update loop reads and writes.
struct LoopArgs {
  Plan P;
  const void* pts;       // the points (n x d, float64 or float32)
  bool f32;              // points are float32
  uint32_t* perm;        // n: the points sorted by cell (counting sort)
  uint32_t* blocksum;    // one word per block of the loop kernel
  const int64_t* thr;    // cell-face table (order codes)
  const uint64_t* dtab;  // packed-key offsets of the 3^d neighbours
  const uint32_t* vpack; // the same offsets v as 2 bits per axis (v_a + 1 at bit 2a)
  BinTable T0;           // binning table (its slots are the points' cell slots)
  LevelTable tab[3];     // level t uses tab[t % 3]; its update merges into tab[(t + 1) % 3]
  uint32_t capAB;        // capacity of each of tab[0..2]
  Cells cells[2];        // cells of alternate levels
  uint32_t* pslot[2];    // merge slot of every cell of alternate levels
  uint32_t* filter[2];   // occupancy filters of alternate levels, kFilterWords each,
                         // zeroed before the launch
  uint32_t* qlist;       // 3 x (level-0 cell bound): slots of the pencil set of step 0
  LevelTable ptab;       // second pencil table of step 0 (key, row, list of 9 x the
                         // level-0 cell bound; cap 0: none)
  uint32_t* forest;      // parent of every cell of every level, then its final cell
  uint32_t* forest2;     // pointer-jumping buffer
  uint32_t* labslot;     // label of every binning slot
  uint32_t* rank;        // label of every final cell
  const uint32_t* slot0;  // binning slot of every point
  int32_t* labels;        // output: label of every point
  int64_t n;
  double* modes;          // output: k x d modes (written if k <= modes_cap)
  int64_t modes_cap;
  IterState* st;          // max_iter + 2 levels, zeroed before the launch
  DevFlags* fl;
  GridBar* bar;           // zeroed before the launch
  LoopResult* res;
  int max_iter;
  uint32_t rank_max;      // largest k numbered inside the loop kernel
  int B;                  // instances (1: a plain run)
  InstState I;            // per-instance state when B > 1
  bool mixed;             // the float32 mixed-precision variant (GS_FP32_MIXED)
  ulonglong2* srow;       // sequential update (plain FP64 runs): count x new centroid of
                          // every slot of the level tables (capAB x d); null: parallel update
  const SweepPlan* sweep; // bandwidth sweep (batched FP64 runs): per-instance cell decisions
                          // (B entries); null otherwise
  uint32_t n0;            // bandwidth sweep: points per instance (instance b's point j is
                          // row j of pts); 0 otherwise
  Tuning tune;            // launch choices (lanes per cell, table load, filter, tail, pencil)
  uint32_t* seq_aux;      // sequential update: 256 colour counts, 256 cursors, then the
                          // level's cells in colour order (capAB words)
};

// Accumulators of one tracking window step (gs_track_window).
struct TrackAcc {
  unsigned long long count;
  unsigned long long bad;  // colours without an exact cell (non-finite, |c / h| >= 2^52)
  long long sum_x, sum_y;
  long long min_x, max_x, min_y, max_y;
};

// Cell decisions of the tracking window step: per channel a, B's keys span
// lo[a] .. lo[a] + span[a] - 1, and the face table at thr + toff[a] holds the
// order codes of the span[a] + 1 faces (least double >= q h) of
// q = lo[a] .. lo[a] + span[a]; lim_bits = the bits of 4e15 h (|c| at or
// above it: no exact cell).
struct TrackPlan {
  int64_t lo[kMaxD];
  int span[kMaxD];
  int toff[kMaxD];
  uint64_t lim_bits;
  float inv_h;
};

// The window step of Algorithm 2 over the pixels x0 <= x < x0 + ww,
// y0 <= y < y0 + wh of a width-wide frame of d channels: R = the pixels whose
// colour cell lies in bins (k >= 1 keys of d channels, sorted
// lexicographically, unique); count, sums and extent of R's positions into
// acc (initialised by the caller), present[j] = 1 for each bin j that R's
// pixels occupy.
cudaError_t launch_track(const void* frame, bool f32, int d, int64_t width, int64_t x0,
                         int64_t y0, int64_t ww, int64_t wh, const TrackPlan& tp,
                         const int64_t* thr, const int64_t* bins, int64_t k, TrackAcc* acc,
                         uint8_t* present, cudaStream_t s);

// The plan a key-range launch makes once the range is known (Sec. 2.1 i:
// key packing, face table, neighbour offsets into fl->plan, fl->plan_status,
// thr and dtab; the face table gets at most thr_cap entries), and the loop
// kernel's start state it clears meanwhile: both occupancy filters
// (filter_vec 16-byte words), n_st level states, the grid barrier, the result.
struct PlanJob {
  double h;
  int B;
  int64_t* thr;
  uint64_t thr_cap;
  uint64_t* dtab;
  uint4* filters;
  uint32_t filter_vec;
  IterState* st;
  uint32_t n_st;
  GridBar* bar;
  LoopResult* res;
};

// Key range, fixed-point window and finiteness of n points of dimension d
// into fl; with job != null, the last block to finish also makes the plan.
// read == false (job required): the points are not read, their extremes
// being in fl already (launch_image_features with fl); the kernel clears
// the loop kernel's start state and makes the plan.
cudaError_t launch_range(const void* pts, bool f32, int64_t n, int d, DevFlags* fl,
                         const PlanJob* job, cudaStream_t s, bool read = true);
// Binning, first pass.  offsets (device, B + 1 entries) give the points of
// each instance of a batched run (B > 1); ignored when B == 1.
// Binning with the plan in fl->plan (nothing runs unless fl->plan_status is 0).
// A bandwidth sweep (sweep != null) bins B x n0 points: instance b's point j
// is row j of pts, decided with sweep[b] (n = B x n0).  listed: new cells
// are listed per warp, 32 at a time (Tuning::bin_list).  sums: the exact cell
// sums are added into T0.acc as well (Tuning::bin_sums; a value outside the
// fixed-point window sets kErrWindow).
cudaError_t launch_bin(const void* pts, bool f32, int64_t n, int d, const int64_t* thr,
                       BinTable T0, uint32_t mask0, uint32_t maxcells, uint32_t* slot0,
                       DevFlags* fl, const int64_t* offsets, int B, const SweepPlan* sweep,
                       uint32_t n0, bool listed, bool sums, cudaStream_t s);

// Blocks of the cooperative loop kernel for dimension d on the current device
// (all co-resident, at most kMaxLoopGrid), or a negative value on error;
// mixed selects the float32 variant.
constexpr int kMaxLoopGrid = 4096;
int loop_grid(int d, bool mixed);
// The rest of step i, steps ii-v for every level, then labels and modes
// (Sec. 2.1, Algorithm 1), in one cooperative launch of `grid` blocks
// (a.mixed selects the float32 variant).
cudaError_t launch_loop(const LoopArgs& a, int grid, cudaStream_t s);
// Step i, second pass, before the loop kernel: per-block count totals and
// the cells' run offsets in a counting sort of the points by cell (two
// launches); the points sorted by cell; the exact cell sums (a.mixed: the
// float32 sums).  After the loop kernel: every point's label, when the loop
// kernel numbered the final cells.  Each does nothing unless the plan is
// valid and binning fit its table.
cudaError_t launch_prep_offsets(const LoopArgs& a, cudaStream_t s);
cudaError_t launch_prep_scatter(const LoopArgs& a, cudaStream_t s);
cudaError_t launch_prep_sums(const LoopArgs& a, cudaStream_t s);
cudaError_t launch_prep_sums_fp64(const LoopArgs& a, cudaStream_t s);
cudaError_t launch_prep_sums_fp32(const LoopArgs& a, cudaStream_t s);
cudaError_t launch_labels_out(const LoopArgs& a, cudaStream_t s);
// Kernels launch_prep_offsets makes.
constexpr int kPrepOffsetsLaunches = 2;

// Modes of the final cells and release of their table, after numbering by
// a radix sort (a.mixed selects the float32 variant).
cudaError_t launch_modes_tail(const LoopArgs& a, uint32_t k, int T, cudaStream_t s);

// Per-precision implementations (gs_loop64.cu, gs_loop32.cu).
int loop_grid_fp64(int d);
int loop_grid_fp32(int d);
cudaError_t launch_loop_fp64(const LoopArgs& a, int grid, cudaStream_t s);
cudaError_t launch_loop_fp32(const LoopArgs& a, int grid, cudaStream_t s);
cudaError_t launch_modes_tail_fp64(const LoopArgs& a, uint32_t k, int T, cudaStream_t s);
cudaError_t launch_modes_tail_fp32(const LoopArgs& a, uint32_t k, int T, cudaStream_t s);

// The sequential update's loop kernel (gs_loop64s.cu; GS_FP64 plain runs with
// a.srow set): its co-resident grid, and its launch.
int loop_grid_seq(int d);
cudaError_t launch_loop_seq(const LoopArgs& a, int grid, cudaStream_t s);

// Numbering of the final cells when k > rank_max: labels of the final cells
// from the sorted order (sorted_vals[p] = cell of rank p), then labels and
// modes.  forest holds the final cell of every initial cell.
// The position products of an image of W columns and H rows: tab[x] = x s
// (x < W), then tab[W + y] = y s (y < H); W + H doubles.
cudaError_t launch_axis_products(int64_t W, int64_t H, double s, double* tab, cudaStream_t st);
// Pixel features of a row-major image (n pixels, width columns, C uint8
// channels) into out (n x (C + 2 xy) float64): the channel values, then, if
// xy, the column and row products from tab (launch_axis_products, earlier on
// the stream).  C <= 8.  With fl (C + 2 xy <= kMaxD), the features' key
// range is published into fl as launch_range would (fl's extremes start
// empty): launch_range then need not read the features.
cudaError_t launch_image_features(const uint8_t* px, int64_t n, int64_t width, int C, bool xy,
                                  const double* tab, double* out, DevFlags* fl, cudaStream_t st);
cudaError_t launch_iota_keys(Cells c, uint64_t* keys, uint32_t* vals, uint32_t k,
                             cudaStream_t s);
cudaError_t launch_rank(const uint32_t* sorted_vals, uint32_t* rank, uint32_t k, cudaStream_t s);
cudaError_t launch_label_tail(const LoopArgs& a, uint32_t m0, uint32_t k, uint32_t baseT, int T,
                              cudaStream_t s);
// Launches launch_label_tail makes.
constexpr int kLabelTailLaunches = 3;

// Stable LSD radix sort of (key, val) pairs by key bits [0, nbits).  keys/vals
// hold the input and receive the output; tkeys/tvals are scratch of the same
// size; hist needs radix_hist_words(n) words.
size_t radix_hist_words(uint32_t n);
int radix_sort_launches(uint32_t n, int nbits);  // kernels one radix_sort call launches
cudaError_t radix_sort(uint64_t* keys, uint32_t* vals, uint64_t* tkeys, uint32_t* tvals,
                       uint32_t* hist, uint32_t n, int nbits, cudaStream_t s);

}  // namespace gs
