// gs_driver.h -- the host-side order of one GridShift run, shared by gs_fit
// (growable workspace owned by a context) and gs_fit_noalloc (workspace carved
// from a static device array).  Where the device buffers come from is the only
// difference between the two, so it sits behind the Workspace interface.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/gridshift.h"
#include "gs_kernels.h"

namespace gs {

// Device views of every buffer one run uses.
struct Bufs {
  DevFlags* flags = nullptr;
  IterState* st = nullptr;     // max_iter + 2 entries
  LoopResult* res = nullptr;
  GridBar* bar = nullptr;
  int64_t* thr = nullptr;      // cell-face table
  uint64_t* dtab = nullptr;    // neighbour offsets (nprobe words), then nprobe packed offset vectors
  uint32_t* slot0 = nullptr;   // n
  uint32_t* perm = nullptr;    // n
  uint32_t* blocksum = nullptr;  // kMaxLoopGrid
  BinTable t0{};               // binning table
  uint32_t t0_maxcells = 0;    // length of t0.list
  LevelTable tab[3]{};         // level tables, capacity capAB each, lists of m0
  uint32_t capAB = 0;
  Cells cells[2]{};            // m0 cells each
  uint32_t* pslot[2] = {nullptr, nullptr};  // m0 each
  uint32_t* filter = nullptr;  // 2 * kFilterWords
  int64_t* offsets = nullptr;  // batched runs: B + 1 point offsets
  uint32_t* inst = nullptr;    // batched runs: per-instance state (inst_words(B) words)
  uint32_t* qlist = nullptr;   // 3 * m0 (pencil set of step 0)
  LevelTable ptab{};           // second pencil table (optional; cap 0: none)
  uint32_t* forest = nullptr;  // m0 * (max_iter + 1)
  uint32_t* forest2 = nullptr; // m0 * (max_iter + 1)
  uint32_t* labslot = nullptr; // t0.cap
  uint32_t* rank = nullptr;    // m0
  uint64_t* skey = nullptr;    // sort of k final keys (only when k > rank_max)
  uint64_t* skey2 = nullptr;
  uint32_t* sval = nullptr;
  uint32_t* sval2 = nullptr;
  uint32_t* shist = nullptr;   // radix_hist_words(k)
  ulonglong2* srow = nullptr;  // sequential update: capAB * d
  uint32_t* seq_aux = nullptr; // sequential update: 512 + capAB words
  SweepPlan* sweep = nullptr;  // bandwidth sweep: B per-instance cell decisions
};

// Source of the device buffers and host staging of one run.  Each method
// returns GS_OK or an error status (setting *err where it has text).
class Workspace {
 public:
  virtual ~Workspace() = default;
  // Host mirrors of DevFlags and LoopResult (pinned where the workspace can).
  virtual DevFlags* host_flags() = 0;
  virtual LoopResult* host_result() = 0;
  // Host staging of `words` 64-bit words for the face and offset tables.
  virtual gs_status host_words(size_t words, int64_t** out, std::string* err) = 0;
  // b.flags (needed before the plan).
  virtual gs_status begin(Bufs& b, std::string* err) = 0;
  // Face-table entries the device-side plan may use (prepare is first called
  // with this many; a plan that needs more is made on the host).
  virtual size_t plan_thr_cap() const = 0;
  // Everything up to and including binning, for n points, a face table of
  // thr_words entries, 3^d offsets, and a binning table for at most m_bound
  // cells (load factor <= 1/2).  Tables handed out are clean (keys empty,
  // counts and sums zero).
  virtual gs_status prepare(int64_t n, int d, int max_iter, size_t thr_words, int nprobe,
                            uint64_t m_bound, cudaStream_t s, Bufs& b, std::string* err) = 0;
  // Binning found more cells than b.t0 holds: a larger clean table in b.t0
  // (and b.t0_maxcells), or an error.
  virtual gs_status regrow_bin(int d, cudaStream_t s, Bufs& b, std::string* err) = 0;
  // Workspace of the cell levels for at most m0 initial cells.
  virtual gs_status levels(uint32_t m0, int d, int max_iter, cudaStream_t s, Bufs& b,
                           std::string* err) = 0;
  // Sort buffers for k final cells.
  virtual gs_status sort_space(uint32_t k, Bufs& b, std::string* err) = 0;
  // Batched runs: b.offsets (B + 1) and b.inst (inst_words(B)), and host
  // staging of per-instance results (inst_words(B) words).
  virtual gs_status batch_space(int B, Bufs& b, uint32_t** host, std::string* err) = 0;
  // The run stopped before the kernels returned every table to clean.
  virtual void mark_dirty(bool dirty) = 0;
  // The number of initial cells binning found (sizes later binning tables).
  virtual void note_cells(uint32_t m0) = 0;
  // The sequential update's shifted rows for level tables of `cap` slots
  // (b.srow, cap * d entries) and its colour lists (b.seq_aux, 512 + cap
  // words), or an error.
  virtual gs_status shift_rows(uint32_t cap, int d, Bufs& b, std::string* err) = 0;
  // A bandwidth sweep's per-instance cell decisions (b.sweep, B entries), or
  // an error.
  virtual gs_status sweep_space(int B, Bufs& b, std::string* err) = 0;
};

// Optional per-phase CUDA-event timing of a run.
class EventTimer {
 public:
  virtual ~EventTimer() = default;
  virtual cudaError_t begin(int phase, cudaStream_t s) = 0;
  virtual cudaError_t end(cudaStream_t s) = 0;
};

struct FitArgs {
  int d;
  double h;
  int max_iter;
  cudaStream_t stream;
  const void* points;
  bool f32;
  int64_t n;  // >= 1
  int32_t* labels;
  double* modes;
  int64_t modes_cap;
  bool mixed = false;  // the float32 mixed-precision variant (GS_FP32_MIXED)
  bool sequential = false;  // the sequential update (Eq. 5; plain FP64 runs only)
  // batched runs (B > 1): host offsets (B + 1), per-instance results (host)
  int B = 1;
  const int64_t* offsets = nullptr;
  gs_fit_info* infos = nullptr;
  int64_t* mode_offsets = nullptr;
  // bandwidth sweep (B > 1): the B values of h (host), one instance per h over
  // the same n0 points (n = B * n0, offsets[b] = b * n0); GS_FP64, parallel
  // update
  const double* sweep_h = nullptr;
  uint32_t n0 = 0;
  // where a plan was refused, its status (kPlan*), for callers that have
  // another way to run (the wide-key pipeline); may be null
  uint32_t* plan_status_out = nullptr;
  // launch choices of the loop kernel (results do not depend on them)
  Tuning tune = kDefaultTuning;
  // image calls: the run first builds the float64 features of these uint8
  // pixels (img_C channels, img_width columns, positions times img_s if
  // img_xy, their products tabulated in img_tab: img_width + n / img_width
  // doubles) into img_feat, which `points` names, and takes their key range
  // from the pixels as it does, so the key-range kernel reads no points
  const uint8_t* img = nullptr;
  double* img_feat = nullptr;
  double* img_tab = nullptr;
  int64_t img_width = 1;
  int img_C = 0;
  bool img_xy = false;
  double img_s = 0.0;
};

// 32-bit words of per-instance state of a batched run of B instances: one
// array of B 64-bit counters and eleven of B 32-bit words (see InstState).
inline size_t inst_words(int B) { return (size_t)B * 13; }

// Device views of the per-instance state laid out in `base` (inst_words(B)
// 32-bit words, 8-byte aligned).
InstState inst_views(uint32_t* base, int B);

// Runs GridShift end to end on the workspace.  Fills *k_out and *info
// (statistics and in-kernel phase times) and returns a status; err receives a
// description of any error (may be null).
// inkernel_ms (optional): kLoopPhases device-clock phase times, then
// 2 * kClockSteps per-step times (update, compaction).
gs_status fit_pipeline(const FitArgs& a, Workspace& ws, EventTimer* timer, int64_t* k_out,
                       gs_fit_info* info, double* inkernel_ms, std::string* err);

// Largest number of final cells numbered inside the loop kernel; more are
// numbered by a radix sort of their keys.
constexpr uint32_t kRankMax = 16384;

// Largest number of instances of one batched call.
constexpr int kMaxBatch = 1 << 20;

// Host helpers shared by the entry points.
uint32_t pow2_at_least(uint64_t v, uint32_t lo);

}  // namespace gs
