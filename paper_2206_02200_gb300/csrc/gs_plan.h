// gs_plan.h -- per-call parameters and device-resident state shared by the host
// driver and the kernels (plain structs, passed to kernels by value).
#pragma once

#include <cstdint>

namespace gs {

constexpr int kMaxD = 8;

// Error bits written to DevFlags::err.
constexpr uint32_t kErrTableFull = 1u;  // a hash table ran out of free slots
constexpr uint32_t kErrOverflow = 2u;   // more cells than the cell arrays hold
constexpr uint32_t kErrWindow = 4u;     // a value above the fixed-point window
constexpr uint32_t kErrBarrier = 8u;    // a grid barrier wait gave up (time limit)

// How integer cell keys (Sec. 2.1 i: floor(x / h) per coordinate) are packed
// into one 64-bit word, and how sums are held in fixed point.
struct Plan {
  int d;
  int nprobe;               // 3^d neighbour offsets v in {-1,0,1}^d (Eq. 1)
  int center;               // index of v = 0 among them
  int off[kMaxD];           // bit offset of the field of axis a (axis 0 most significant)
  int span[kMaxD];          // kmax_a - kmin_a + 1 cells along axis a
  int thr_off[kMaxD];       // start of axis a's face table in the threshold array
  int L[kMaxD];             // fixed-point unit 2^L of axis a
  int64_t kmin[kMaxD];      // smallest key of axis a
  float inv_h;              // 1/h rounded to float: first guess of a cell index only
  int inst_off;             // batched runs: bit offset of the instance field (above all axes)
  float h32;                // h rounded to float (the float32 variant)
};

// The cell decisions of one bandwidth of a bandwidth sweep (gs_fit_sweep):
// B instances share the points and the packed-key layout (each axis field as
// wide as the largest span over the bandwidths), and differ in h.  Instance b
// decides floor(x / h_b) along axis a against its own faces, the span[a] + 1
// entries at thr_off[a] of the call's face table, for the cell indices
// kmin[a] .. kmin[a] + span[a] (Sec. 2.1 i with its own h).
struct SweepPlan {
  int64_t kmin[kMaxD];
  int span[kMaxD];
  int thr_off[kMaxD];
  float inv_h;  // 1/h_b rounded to float: first guess of a cell index only
  int pad;
};

// Launch choices of the loop kernel that do not change its results (only
// which lanes, tables and phases compute them); chosen per workload by the
// autotuner (gs_set_tuning), else the defaults below.
struct Tuning {
  uint32_t few_lanes_x4;  // a level is updated with GatherLanes<D>::min lanes per cell when
                          // 4 x its cells exceed few_lanes_x4 x the grid's warps, else 32
  uint32_t load_shift;    // level tables sized for load <= 2^-load_shift (1 or 2)
  uint32_t filter;        // 1: neighbour probes pass the level's occupancy filter first
  uint32_t tail_enter;    // levels of at most this many cells finish in one block (<= 256)
  uint32_t pencil_min;    // least initial cells for the pencil form of the first update
  uint32_t split_min;     // least points for step i's second pass and the label writes as
                          // launches of their own (fewer: inside the loop kernel)
  uint32_t bin_list;      // 1: binning lists new cells per warp, 32 at a time (one add on
                          // the cell count for each 32); 0: one add per new cell
  uint32_t bin_sums;      // 1: binning forms the exact cell sums as it reads the points (one
                          // set of limb adds per distinct cell of a warp); 0: a counting
                          // sort of the points by cell, then sums over the sorted runs
};

constexpr Tuning kDefaultTuning = {4u, 2u, 1u, 128u, 4096u, 1u << 22, 1u, 0u};
constexpr uint32_t kTailMaxCells = 256;  // the one-block tail's shared memory holds this many

// Device-resident state of one level t (the cells before update step t).
struct IterState {
  uint32_t m;       // active cells at level t
  uint32_t mask;    // capacity mask of the lookup table of level t
  uint32_t has_nb;  // 1 if some cell of level t has an active neighbour (v != 0)
  uint32_t base;    // first node of level t in the forest of merges
  uint32_t qn;      // level 0 only: positions of the pencil set of step 0
  uint32_t qn2;     // level 0 only: positions of the second pencil set
};

// Plan status (DevFlags::plan_status).
constexpr uint32_t kPlanOK = 0;
constexpr uint32_t kPlanNonFinite = 1;  // a coordinate is NaN or infinite
constexpr uint32_t kPlanRangeH = 2;     // a coordinate divided by h exceeds 2^52
constexpr uint32_t kPlanSpan = 3;       // more than 2^22 cells along one axis
constexpr uint32_t kPlanBits = 4;       // the packed key needs more than 63 bits
constexpr uint32_t kPlanTable = 5;      // face table above the device-side capacity

// Sizes that follow from a plan.
struct PlanSizes {
  uint64_t thr_words;  // face-table entries (sum over axes of span + 1)
  uint64_t span_prod;  // product of the spans (saturating above 2^40)
  int32_t total_bits;  // width of the packed key
  int32_t pad;
};

// Global device flags and counters of a call.
struct DevFlags {
  uint32_t err;                 // kErr* bits
  uint32_t m0;                  // cells created by binning
  unsigned long long inexact;   // values truncated by the fixed-point window
  unsigned long long bad;       // non-finite input coordinates
  unsigned long long rechecks;  // float32 variant: key decisions redone in float64
  long long min_ord[kMaxD];     // order code of min_i x_ia
  long long max_ord[kMaxD];     // order code of max_i x_ia
  unsigned long long maxabs[kMaxD];  // bits of max_i |x_ia|
  // the plan of the call (written by the key-range kernel or the host), read by
  // binning and the loop kernel; nothing after the key range runs unless
  // plan_status is 0
  Plan plan;
  PlanSizes plan_sizes;
  uint32_t plan_status;
  uint32_t range_done;  // blocks of the key-range kernel that have published their extremes
};

// Segments of the loop kernel timed on the device clock by block 0 (between
// grid barriers): counting-sort offsets, scatter, exact cell sums (the second
// pass of binning), level 0, the first update step, the later update steps,
// compaction, labels.
constexpr int kLoopPhases = 8;

// What the update loop reports back (written by one thread at its end).
struct LoopResult {
  int32_t iterations;   // update steps applied
  int32_t converged;    // 1: stopped by the criterion of Sec. 2.1 v
  uint32_t k;           // final cells
  uint32_t base;        // first forest node of the final level
  uint32_t need_sort;   // 1: k too large for the in-loop numbering; labels not written
  uint32_t bin_failed;  // 1: binning overflowed its table; nothing after it ran
  uint32_t labels_ready;  // 1: the final cells are numbered; the labels are to be written
  unsigned long long cell_iters;  // sum of m_t over applied updates
  unsigned long long ns[kLoopPhases];  // nanoseconds spent in each segment
  unsigned long long step_ns[16][2];   // first 16 update steps: update phase, compaction
  // the state block 0 leaves after finishing the update steps alone
  int32_t tail_t;
  uint32_t tail_m, tail_base;
  int32_t tail_conv;
  unsigned long long tail_cells;
};

constexpr int kClockSteps = 16;

// Per-instance state of a batched run (B point sets in one run, each cell
// key carrying its instance in the field above the axes).  Arrays of B
// entries; [2] arrays alternate between update steps.
struct InstState {
  uint32_t* done[2];       // 1 once the instance has stopped updating (step t uses done[t & 1])
  uint32_t* nbf[2];        // 1 if a cell of the instance had a neighbour at step t
  uint32_t* mt[2];         // cells of the instance at level t
  int32_t* iters;          // update steps applied to the instance
  int32_t* conv;           // 1 if the instance stopped by the criterion of Sec. 2.1 v
  uint32_t* m0;            // initial cells of the instance
  uint32_t* k;             // final cells of the instance
  uint32_t* koff;          // final cells of all earlier instances
  unsigned long long* cell_iters;  // sum over its applied steps of the instance's cells
};

// Arrival counter and generation of a software grid barrier, and the stop
// decision its last arrival takes for every block (any error bit set).
// count and gen sit on separate 128-byte lines, so the polling of gen does
// not contend with the arrivals.
struct GridBar {
  alignas(128) unsigned int count;
  alignas(128) unsigned int gen;
  unsigned int stop;
};

}  // namespace gs
