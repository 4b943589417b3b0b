// gs_api.cu -- host side of the C ABI declared in include/gridshift.h: argument
// checks, the context and its growable device workspace.  The order of the
// steps of one run is in gs_driver.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gridshift.h"
#include "gs_driver.h"
#include "gs_planner.cuh"
#include "gs_wide.h"

using namespace gs;

namespace {

// A growable device allocation.
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t cap = 0;  // elements
  cudaError_t ensure(size_t n, bool* grew = nullptr) {
    if (grew) *grew = false;
    if (n <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = n + n / 4 + 64;
    cudaError_t e = cudaMalloc((void**)&p, want * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    cap = want;
    if (grew) *grew = true;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

// Device storage of the binning table (see gs::BinTable).
struct BinTableBuf {
  DBuf<uint64_t> key;
  DBuf<uint32_t> cnt, off, id, list;
  DBuf<uint64_t> acc;
  uint32_t cap = 0;
  int d = 0;
  // Allocates capacity c (power of two) for d-dimensional sums of up to c / 2
  // cells; a new or regrown table is cleared.
  cudaError_t ensure(uint32_t c, int dd, cudaStream_t s) {
    cudaError_t e;
    if (c > cap || dd != d) {
      key.release(); cnt.release(); off.release(); id.release(); acc.release(); list.release();
      cap = 0;
      if ((e = key.ensure(c)) != cudaSuccess) return e;
      if ((e = cnt.ensure(c)) != cudaSuccess) return e;
      if ((e = off.ensure(c)) != cudaSuccess) return e;
      if ((e = id.ensure(c)) != cudaSuccess) return e;
      if ((e = acc.ensure((size_t)c * dd * 4)) != cudaSuccess) return e;
      if ((e = list.ensure(c / 2)) != cudaSuccess) return e;
      cap = c;
      d = dd;
      if ((e = clear(s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t clear(cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(key.p, 0xFF, sizeof(uint64_t) * key.cap, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cnt.p, 0, sizeof(uint32_t) * cnt.cap, s)) != cudaSuccess) return e;
    return cudaMemsetAsync(acc.p, 0, sizeof(uint64_t) * acc.cap, s);
  }
  BinTable view() const { return BinTable{key.p, cnt.p, off.p, id.p, acc.p, list.p, cap}; }
  void release() {
    key.release(); cnt.release(); off.release(); id.release(); acc.release(); list.release();
    cap = 0;
  }
};

// Device storage of a level table (see gs::LevelTable).
struct LevelTableBuf {
  DBuf<uint64_t> key;
  DBuf<uint32_t> id, list;
  DBuf<ulonglong2> row;
  DBuf<uint64_t> acc;
  uint32_t cap = 0;
  int d = 0;
  cudaError_t ensure(uint32_t c, int dd, uint32_t lmax, cudaStream_t s) {
    cudaError_t e;
    if (c > cap || dd != d) {
      key.release(); id.release(); row.release(); acc.release();
      cap = 0;
      if ((e = key.ensure(c)) != cudaSuccess) return e;
      if ((e = id.ensure(c)) != cudaSuccess) return e;
      if ((e = row.ensure((size_t)c * (dd + 1))) != cudaSuccess) return e;
      if ((e = acc.ensure((size_t)c * dd * 4)) != cudaSuccess) return e;
      cap = c;
      d = dd;
      if ((e = clear(s)) != cudaSuccess) return e;
    }
    return list.ensure(lmax);
  }
  cudaError_t clear(cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(key.p, 0xFF, sizeof(uint64_t) * key.cap, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(row.p, 0, sizeof(ulonglong2) * row.cap, s)) != cudaSuccess) return e;
    return cudaMemsetAsync(acc.p, 0, sizeof(uint64_t) * acc.cap, s);
  }
  LevelTable view() const { return LevelTable{key.p, id.p, row.p, acc.p, list.p, cap}; }
  void release() {
    key.release(); id.release(); row.release(); acc.release(); list.release();
    cap = 0;
  }
};

// A table of keys and rows without merge accumulators (the second pencil
// table of step 0).
struct PencilTableBuf {
  DBuf<uint64_t> key;
  DBuf<uint32_t> list;
  DBuf<ulonglong2> row;
  uint32_t cap = 0;
  int d = 0;
  cudaError_t ensure(uint32_t c, int dd, size_t lmax, cudaStream_t s) {
    cudaError_t e;
    if (c > cap || dd != d) {
      key.release(); row.release();
      cap = 0;
      if ((e = key.ensure(c)) != cudaSuccess) return e;
      if ((e = row.ensure((size_t)c * (dd + 1))) != cudaSuccess) return e;
      cap = c;
      d = dd;
      if ((e = clear(s)) != cudaSuccess) return e;
    }
    return list.ensure(lmax);
  }
  cudaError_t clear(cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(key.p, 0xFF, sizeof(uint64_t) * key.cap, s)) != cudaSuccess) return e;
    return cudaMemsetAsync(row.p, 0, sizeof(ulonglong2) * row.cap, s);
  }
  LevelTable view() const { return LevelTable{key.p, nullptr, row.p, nullptr, list.p, cap}; }
  void release() {
    key.release(); row.release(); list.release();
    cap = 0;
  }
};

struct CellBuf {
  DBuf<uint64_t> key;
  DBuf<uint32_t> cnt;
  cudaError_t ensure(uint32_t m) {
    cudaError_t e;
    if ((e = key.ensure(m)) != cudaSuccess) return e;
    return cnt.ensure(m);
  }
  Cells view() const { return Cells{key.p, cnt.p}; }
  void release() { key.release(); cnt.release(); }
};

// CUDA events around the launch groups of one call (opt-in, gs_set_timing).
struct PhaseTimer : public EventTimer {
  std::vector<cudaEvent_t> pool;
  std::vector<int> phase;  // phase of the event pair (2i, 2i+1)
  size_t used = 0;
  cudaError_t record(cudaStream_t s) {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      pool.push_back(e);
    }
    return cudaEventRecord(pool[used++], s);
  }
  cudaError_t begin(int ph, cudaStream_t s) override {
    phase.push_back(ph);
    return record(s);
  }
  cudaError_t end(cudaStream_t s) override { return record(s); }
  void reset() {
    used = 0;
    phase.clear();
  }
  void release() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    phase.clear();
    used = 0;
  }
};

// The growable workspace of a context: buffers are allocated on first need,
// grown when a call needs more, and kept for later calls.
struct CtxWorkspace : public Workspace {
  DBuf<DevFlags> flags;
  DBuf<IterState> st;
  DBuf<LoopResult> res;
  DBuf<GridBar> bar;
  DBuf<int64_t> thr;
  DBuf<uint64_t> dtab;
  DBuf<uint32_t> slot0, perm, blocksum;
  BinTableBuf t0;
  LevelTableBuf tab[3];
  PencilTableBuf ptab;
  CellBuf cells[2];
  DBuf<uint32_t> pslot[2], qlist, forest, forest2, labslot, rank, filter;
  DBuf<uint64_t> skey, skey2;
  DBuf<uint32_t> sval, sval2, shist;
  DBuf<int64_t> offsets;
  DBuf<uint32_t> inst;
  DBuf<ulonglong2> srow;          // the sequential update's shifted rows
  DBuf<uint32_t> seq_aux;         // the sequential update's colour lists
  DBuf<SweepPlan> sweep;          // a bandwidth sweep's per-instance cell decisions
  std::vector<uint64_t> h_inst;   // host copy of the per-instance state (8-byte aligned)

  DevFlags* h_flags = nullptr;    // pinned
  LoopResult* h_res = nullptr;    // pinned
  int64_t* h_words = nullptr;     // pinned staging of the face and offset tables
  size_t h_words_cap = 0;
  bool dirty = false;             // a call stopped with tables not returned to clean
  uint64_t last_m0 = 0;           // initial cells of the last call (sizes the binning table)

  std::string alloc_err(cudaError_t e, const char* what) {
    return std::string(what) + ": " + cudaGetErrorName(e);
  }

  DevFlags* host_flags() override { return h_flags; }
  LoopResult* host_result() override { return h_res; }

  gs_status host_words(size_t words, int64_t** out, std::string* err) override {
    if (words > h_words_cap) {
      if (h_words) cudaFreeHost(h_words);
      h_words = nullptr;
      h_words_cap = 0;
      cudaError_t e = cudaMallocHost((void**)&h_words, sizeof(int64_t) * words);
      if (e != cudaSuccess) {
        h_words = nullptr;
        *err = alloc_err(e, "cudaMallocHost");
        return GS_E_NOMEM;
      }
      h_words_cap = words;
    }
    *out = h_words;
    return GS_OK;
  }

  gs_status begin(Bufs& b, std::string* err) override {
    cudaError_t e = cudaSuccess;
    if (!h_flags) e = cudaMallocHost((void**)&h_flags, sizeof(DevFlags));
    if (e == cudaSuccess && !h_res) e = cudaMallocHost((void**)&h_res, sizeof(LoopResult));
    if (e == cudaSuccess) e = flags.ensure(1);
    if (e != cudaSuccess) {
      *err = alloc_err(e, "workspace");
      return e == cudaErrorMemoryAllocation ? GS_E_NOMEM : GS_E_CUDA;
    }
    b.flags = flags.p;
    return GS_OK;
  }

  size_t plan_thr_cap() const override { return size_t(1) << 16; }

  gs_status prepare(int64_t n, int d, int max_iter, size_t thr_words, int nprobe,
                    uint64_t m_bound, cudaStream_t s, Bufs& b, std::string* err) override {
    cudaError_t e;
#define WS_CU(call, what)                                              \
  do {                                                                 \
    e = (call);                                                        \
    if (e != cudaSuccess) {                                            \
      *err = alloc_err(e, what);                                       \
      return e == cudaErrorMemoryAllocation ? GS_E_NOMEM : GS_E_CUDA;  \
    }                                                                  \
  } while (0)
    WS_CU(st.ensure(max_iter + 2), "alloc state");
    WS_CU(res.ensure(1), "alloc result");
    WS_CU(bar.ensure(1), "alloc barrier");
    WS_CU(thr.ensure(thr_words), "alloc face table");
    WS_CU(dtab.ensure(2 * (size_t)nprobe), "alloc offsets");
    WS_CU(slot0.ensure(n), "alloc slot0");
    WS_CU(perm.ensure(n), "alloc perm");
    WS_CU(blocksum.ensure(kMaxLoopGrid), "alloc block sums");
    // binning table for the cells expected: as many as the last call found
    // (plus a quarter), else n / 32; an overflow regrows it (regrow_bin)
    uint64_t est = last_m0 ? last_m0 + last_m0 / 4 + 1024 : (uint64_t)n / 32 + 65536;
    if (est > m_bound) est = m_bound;
    uint32_t cap0 = pow2_at_least(2 * est, 1024);
    if (t0.cap > cap0 && t0.d == d) cap0 = t0.cap;
    if (dirty) {
      if (t0.cap) WS_CU(t0.clear(s), "clear T0");
      for (int i = 0; i < 3; ++i)
        if (tab[i].cap) WS_CU(tab[i].clear(s), "clear level table");
      if (ptab.cap) WS_CU(ptab.clear(s), "clear pencil table");
    }
    WS_CU(t0.ensure(cap0, d, s), "alloc T0");
    b.st = st.p;
    b.res = res.p;
    b.bar = bar.p;
    b.thr = thr.p;
    b.dtab = dtab.p;
    b.slot0 = slot0.p;
    b.perm = perm.p;
    b.blocksum = blocksum.p;
    b.t0 = t0.view();
    b.t0_maxcells = t0.cap / 2;
    return GS_OK;
  }

  gs_status regrow_bin(int d, cudaStream_t s, Bufs& b, std::string* err) override {
    if (t0.cap >= (1u << 29)) {
      *err = "binning table overflow";
      return GS_E_INTERNAL;
    }
    cudaError_t e;
    WS_CU(t0.clear(s), "clear T0");
    WS_CU(t0.ensure(t0.cap << 2, d, s), "alloc T0");
    b.t0 = t0.view();
    b.t0_maxcells = t0.cap / 2;
    return GS_OK;
  }

  gs_status levels(uint32_t m0, int d, int max_iter, cudaStream_t s, Bufs& b,
                   std::string* err) override {
    cudaError_t e;
    const uint32_t capAB = pow2_at_least(4ull * m0, 64);
    const uint32_t m = m0 > 0 ? m0 : 1;
    for (int i = 0; i < 3; ++i) WS_CU(tab[i].ensure(capAB, d, m, s), "alloc level table");
    for (int i = 0; i < 2; ++i) {
      WS_CU(cells[i].ensure(m), "alloc cells");
      WS_CU(pslot[i].ensure(m), "alloc pslot");
    }
    WS_CU(qlist.ensure((size_t)m * 3), "alloc pencil list");
    // the second pencil table: 12 slots per cell bound, at most 2^24 slots
    // (2 GB at d = 6); where it is short, step 0 uses one pencil stage
    if (d >= kPencil2MinD) {
      uint32_t cp = pow2_at_least(12ull * m, 64);
      if (cp > (1u << 24)) cp = 1u << 24;
      WS_CU(ptab.ensure(cp, d, (size_t)m * 9, s), "alloc pencil table");
    }
    b.ptab = ptab.view();
    WS_CU(forest.ensure((size_t)m * (max_iter + 1)), "alloc forest");
    WS_CU(forest2.ensure((size_t)m * (max_iter + 1)), "alloc forest");
    WS_CU(labslot.ensure(t0.cap), "alloc labslot");
    WS_CU(rank.ensure(m), "alloc rank");
    WS_CU(filter.ensure(2 * kFilterWords), "alloc filters");
    b.filter = filter.p;
    b.capAB = tab[0].cap;
    for (int i = 0; i < 3; ++i) {
      b.tab[i] = tab[i].view();
      if (tab[i].cap < b.capAB) b.capAB = tab[i].cap;
    }
    for (int i = 0; i < 2; ++i) {
      b.cells[i] = cells[i].view();
      b.pslot[i] = pslot[i].p;
    }
    b.qlist = qlist.p;
    b.forest = forest.p;
    b.forest2 = forest2.p;
    b.labslot = labslot.p;
    b.rank = rank.p;
    return GS_OK;
  }

  gs_status sort_space(uint32_t k, Bufs& b, std::string* err) override {
    cudaError_t e;
    WS_CU(skey.ensure(k), "alloc sort");
    WS_CU(skey2.ensure(k), "alloc sort");
    WS_CU(sval.ensure(k), "alloc sort");
    WS_CU(sval2.ensure(k), "alloc sort");
    WS_CU(shist.ensure(radix_hist_words(k)), "alloc sort");
    b.skey = skey.p;
    b.skey2 = skey2.p;
    b.sval = sval.p;
    b.sval2 = sval2.p;
    b.shist = shist.p;
    return GS_OK;
  }

  gs_status batch_space(int B, Bufs& b, uint32_t** host, std::string* err) override {
    cudaError_t e;
    WS_CU(offsets.ensure((size_t)B + 1), "alloc offsets");
    WS_CU(inst.ensure(inst_words(B) + 2), "alloc instance state");
    h_inst.resize(inst_words(B) / 2 + 2);
    b.offsets = offsets.p;
    b.inst = inst.p;
    *host = reinterpret_cast<uint32_t*>(h_inst.data());
    return GS_OK;
  }
  gs_status shift_rows(uint32_t cap, int d, Bufs& b, std::string* err) override {
    cudaError_t e;
    WS_CU(srow.ensure((size_t)cap * d), "alloc shifted rows");
    WS_CU(seq_aux.ensure((size_t)cap + 512), "alloc colour lists");
    b.srow = srow.p;
    b.seq_aux = seq_aux.p;
    return GS_OK;
  }
  gs_status sweep_space(int B, Bufs& b, std::string* err) override {
    cudaError_t e;
    WS_CU(sweep.ensure((size_t)B), "alloc sweep plans");
    b.sweep = sweep.p;
    return GS_OK;
  }
#undef WS_CU

  void mark_dirty(bool d) override { dirty = d; }
  void note_cells(uint32_t m0) override { last_m0 = m0; }

  void release() {
    flags.release(); st.release(); res.release(); bar.release(); thr.release(); dtab.release();
    slot0.release(); perm.release(); blocksum.release(); t0.release();
    for (int i = 0; i < 3; ++i) tab[i].release();
    for (int i = 0; i < 2; ++i) {
      cells[i].release();
      pslot[i].release();
    }
    qlist.release(); ptab.release(); forest.release(); forest2.release(); labslot.release(); rank.release(); filter.release();
    skey.release(); skey2.release(); sval.release(); sval2.release(); shist.release();
    offsets.release(); inst.release(); srow.release(); sweep.release(); seq_aux.release();
    if (h_flags) cudaFreeHost(h_flags);
    if (h_res) cudaFreeHost(h_res);
    if (h_words) cudaFreeHost(h_words);
    h_flags = nullptr;
    h_res = nullptr;
    h_words = nullptr;
    h_words_cap = 0;
    dirty = false;
  }
};

}  // namespace

struct gs_ctx {
  int d = 0;
  double h = 0;
  int max_iter = 0;
  gs_precision prec = GS_FP64;
  gs_update update = GS_UPDATE_PARALLEL;
  Tuning tune = kDefaultTuning;
  cudaStream_t stream = nullptr;
  int device = -1;
  std::string err;
  bool timing = false;
  PhaseTimer tm;
  gs_phase_times last_times{};
  CtxWorkspace ws;
  WideWorkspace* wide = nullptr;  // the wide-key pipeline's buffers (made on first use)
  // the tracking window step: one device block [accumulators | reference
  // cells | cell flags] and its pinned host staging
  DBuf<uint4> tbuf;
  unsigned char* h_track = nullptr;
  size_t h_track_cap = 0;
  DBuf<double> feat;  // gs_fit_image: the pixels' float64 features
  // gs_fit_images_host: double-buffered device copies of an image, its
  // labels and modes, the copy stream and its events
  DBuf<uint8_t> himg[2];
  DBuf<int32_t> hlab[2];
  DBuf<double> hmodes[2];
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t up_ev[2] = {nullptr, nullptr}, done_ev[2] = {nullptr, nullptr},
              down_ev[2] = {nullptr, nullptr};

  void release_stream() {
    for (int i = 0; i < 2; ++i) {
      for (cudaEvent_t* e : {&up_ev[i], &done_ev[i], &down_ev[i]}) {
        if (*e) cudaEventDestroy(*e);
        *e = nullptr;
      }
      himg[i].release();
      hlab[i].release();
      hmodes[i].release();
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
    copy_stream = nullptr;
  }

  void release_device() {
    release_stream();
    feat.release();
    ws.release();
    wide_workspace_free(wide);
    wide = nullptr;
    tm.release();
    tbuf.release();
    if (h_track) cudaFreeHost(h_track);
    h_track = nullptr;
    h_track_cap = 0;
  }
};

namespace {

gs_status fail(gs_ctx* c, gs_status s, const std::string& msg) {
  c->err = msg;
  return s;
}

}  // namespace

extern "C" {

const char* gs_status_string(gs_status s) {
  switch (s) {
    case GS_OK: return "GS_OK";
    case GS_E_INVALID: return "GS_E_INVALID";
    case GS_E_NOMEM: return "GS_E_NOMEM";
    case GS_E_KEYRANGE: return "GS_E_KEYRANGE";
    case GS_E_CAPACITY: return "GS_E_CAPACITY";
    case GS_E_CUDA: return "GS_E_CUDA";
    case GS_E_INTERNAL: return "GS_E_INTERNAL";
    case GS_E_SCRATCH: return "GS_E_SCRATCH";
  }
  return "GS_E_UNKNOWN";
}

gs_status gs_create(int d, double h, int max_iter, gs_ctx** out) {
  if (!out) return GS_E_INVALID;
  *out = nullptr;
  if (d < 1 || d > kMaxWideD || !(h > 0) || !std::isfinite(h) || max_iter < 0 ||
      max_iter > 100000)
    return GS_E_INVALID;
  gs_ctx* c = new (std::nothrow) gs_ctx();
  if (!c) return GS_E_NOMEM;
  c->d = d;
  c->h = h;
  c->max_iter = max_iter;
  *out = c;
  return GS_OK;
}

gs_status gs_set_precision(gs_ctx* ctx, gs_precision p) {
  if (!ctx) return GS_E_INVALID;
  if (p != GS_FP64 && p != GS_FP32_MIXED) return fail(ctx, GS_E_INVALID, "unknown precision");
  // the two precisions keep different state in the same tables: clear them
  if (p != ctx->prec) ctx->ws.mark_dirty(true);
  ctx->prec = p;
  return GS_OK;
}

gs_status gs_set_update(gs_ctx* ctx, gs_update u) {
  if (!ctx) return GS_E_INVALID;
  if (u != GS_UPDATE_PARALLEL && u != GS_UPDATE_SEQUENTIAL)
    return fail(ctx, GS_E_INVALID, "unknown update form");
  ctx->update = u;
  return GS_OK;
}

gs_status gs_set_stream(gs_ctx* ctx, void* cuda_stream) {
  if (!ctx) return GS_E_INVALID;
  ctx->stream = (cudaStream_t)cuda_stream;
  return GS_OK;
}

gs_status gs_set_tuning(gs_ctx* ctx, const gs_tuning* t) {
  if (!ctx) return GS_E_INVALID;
  if (!t) {
    ctx->tune = kDefaultTuning;
    return GS_OK;
  }
  if (t->few_lanes_x4 < 0 || t->few_lanes_x4 > (1 << 20) || (t->load_shift != 1 && t->load_shift != 2) ||
      (t->filter != 0 && t->filter != 1) || t->tail_enter < 0 ||
      t->tail_enter > (int32_t)kTailMaxCells || t->pencil_min < 0 || t->split_min < 0 ||
      (t->bin_list != 0 && t->bin_list != 1) || (t->bin_sums != 0 && t->bin_sums != 1))
    return fail(ctx, GS_E_INVALID, "tuning value out of range");
  ctx->tune.few_lanes_x4 = (uint32_t)t->few_lanes_x4;
  ctx->tune.load_shift = (uint32_t)t->load_shift;
  ctx->tune.filter = (uint32_t)t->filter;
  ctx->tune.tail_enter = (uint32_t)t->tail_enter;
  ctx->tune.pencil_min = (uint32_t)t->pencil_min;
  ctx->tune.split_min = (uint32_t)t->split_min;
  ctx->tune.bin_list = (uint32_t)t->bin_list;
  ctx->tune.bin_sums = (uint32_t)t->bin_sums;
  return GS_OK;
}

gs_status gs_get_tuning(gs_ctx* ctx, gs_tuning* out) {
  if (!ctx || !out) return GS_E_INVALID;
  out->few_lanes_x4 = (int32_t)ctx->tune.few_lanes_x4;
  out->load_shift = (int32_t)ctx->tune.load_shift;
  out->filter = (int32_t)ctx->tune.filter;
  out->tail_enter = (int32_t)ctx->tune.tail_enter;
  out->pencil_min = (int32_t)ctx->tune.pencil_min;
  out->split_min = (int32_t)ctx->tune.split_min;
  out->bin_list = (int32_t)ctx->tune.bin_list;
  out->bin_sums = (int32_t)ctx->tune.bin_sums;
  return GS_OK;
}

gs_status gs_set_timing(gs_ctx* ctx, int enable) {
  if (!ctx) return GS_E_INVALID;
  ctx->timing = enable != 0;
  return GS_OK;
}

gs_status gs_get_phase_times(gs_ctx* ctx, gs_phase_times* out) {
  if (!ctx || !out) return GS_E_INVALID;
  *out = ctx->last_times;
  return GS_OK;
}

gs_status gs_get_last_error(gs_ctx* ctx, char* buf, size_t len) {
  if (!ctx || !buf || len == 0) return GS_E_INVALID;
  std::snprintf(buf, len, "%s", ctx->err.c_str());
  return GS_OK;
}

void gs_destroy(gs_ctx* ctx) {
  if (!ctx) return;
  ctx->release_device();
  delete ctx;
}

// The pixels of an image call (see FitArgs::img): the run builds their
// features into the context's feature buffer.
struct ImgSrc {
  const uint8_t* px;
  int64_t width;
  int C;
  bool xy;
  double s;
  double* tab;  // xy: width + n / width doubles of the buffer (position products)
};

static gs_status batched_entry(gs_ctx* ctx, const void* points, gs_dtype dtype,
                               const int64_t* offsets, int B, int32_t* labels, double* modes,
                               int64_t modes_cap, int64_t* mode_offsets, gs_fit_info* infos,
                               const ImgSrc* img);

static void set_image(FitArgs& a, const ImgSrc* img) {
  if (!img) return;
  a.img = img->px;
  a.img_feat = const_cast<double*>(static_cast<const double*>(a.points));
  a.img_width = img->width;
  a.img_C = img->C;
  a.img_xy = img->xy;
  a.img_s = img->s;
  a.img_tab = img->tab;
}

// gs_fit, and the image calls (img: `points` is the context's feature
// buffer, which the run fills).
static gs_status fit_entry(gs_ctx* ctx, const void* points, gs_dtype dtype, int64_t n,
                           int32_t* labels, double* modes, int64_t modes_cap, int64_t* k_out,
                           gs_fit_info* info, const ImgSrc* img) {
  if (!ctx) return GS_E_INVALID;
  ctx->err.clear();
  if (!k_out) return fail(ctx, GS_E_INVALID, "k_out is NULL");
  if (n < 0 || n >= (1ll << 31)) return fail(ctx, GS_E_INVALID, "n out of range");
  if (dtype != GS_IN_F64 && dtype != GS_IN_F32) return fail(ctx, GS_E_INVALID, "bad dtype");
  if (modes_cap < 0 || (modes_cap > 0 && !modes))
    return fail(ctx, GS_E_INVALID, "modes is NULL with modes_cap > 0");
  if (n > 0 && (!points || !labels)) return fail(ctx, GS_E_INVALID, "NULL points or labels");
  if (ctx->update == GS_UPDATE_SEQUENTIAL && ctx->prec != GS_FP64)
    return fail(ctx, GS_E_INVALID, "the sequential update runs in GS_FP64 only");
  gs_fit_info inf;
  std::memset(&inf, 0, sizeof(inf));
  *k_out = 0;
  ctx->tm.reset();
  std::memset(&ctx->last_times, 0, sizeof(ctx->last_times));
  if (n == 0) {
    inf.converged = 1;
    if (info) *info = inf;
    return GS_OK;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(ctx, GS_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorName(ce));
  if (ctx->device != dev) {
    ctx->release_device();
    ctx->device = dev;
  }
  FitArgs a;
  a.d = ctx->d;
  a.h = ctx->h;
  a.max_iter = ctx->max_iter;
  a.stream = ctx->stream;
  a.points = points;
  a.f32 = dtype == GS_IN_F32;
  a.n = n;
  a.labels = labels;
  a.modes = modes;
  a.modes_cap = modes_cap;
  a.tune = ctx->tune;
  a.mixed = ctx->prec == GS_FP32_MIXED;
  a.sequential = ctx->update == GS_UPDATE_SEQUENTIAL;
  set_image(a, img);
  double kms[kLoopPhases + 2 * kClockSteps] = {};
  gs_status st;
  const bool wide_ok = !a.mixed && !a.sequential;
  if (ctx->d > kMaxD) {
    // more axes than the packed key holds: the wide-key pipeline
    if (!wide_ok)
      return fail(ctx, GS_E_INVALID, "d > 8 runs in GS_FP64 with the parallel update only");
    if (!ctx->wide && !(ctx->wide = wide_workspace_new())) return fail(ctx, GS_E_NOMEM, "wide workspace");
    if (img) {
      // the features first (the wide pipeline takes its own key range)
      if (img->xy) {
        ce = launch_axis_products(img->width, n / img->width, img->s, img->tab, ctx->stream);
        if (ce != cudaSuccess)
          return fail(ctx, GS_E_CUDA, std::string("k_axis_products: ") + cudaGetErrorName(ce));
        inf.launches += 1;
      }
      ce = launch_image_features(img->px, n, img->width, img->C, img->xy, img->tab, a.img_feat,
                                 nullptr, ctx->stream);
      if (ce != cudaSuccess)
        return fail(ctx, GS_E_CUDA, std::string("k_image_features: ") + cudaGetErrorName(ce));
      inf.launches += 1;
    }
    st = wide_fit(ctx->wide, a, k_out, &inf, &ctx->err);
  } else {
    uint32_t plan_st = kPlanOK;
    a.plan_status_out = &plan_st;
    st = fit_pipeline(a, ctx->ws, ctx->timing ? &ctx->tm : nullptr, k_out, &inf, kms, &ctx->err);
    if (st == GS_E_KEYRANGE && wide_ok && (plan_st == kPlanBits || plan_st == kPlanSpan)) {
      // the keys do not fit the 63-bit packed key: the wide-key pipeline
      // (its kernels count on top of the refused attempt's)
      if (!ctx->wide && !(ctx->wide = wide_workspace_new()))
        return fail(ctx, GS_E_NOMEM, "wide workspace");
      ctx->err.clear();
      st = wide_fit(ctx->wide, a, k_out, &inf, &ctx->err);
    }
  }
  if (info) *info = inf;
  if (st != GS_OK && st != GS_E_CAPACITY) return st;
  if (ctx->timing) {
    for (size_t i = 0; i < ctx->tm.phase.size(); ++i) {
      float ms = 0.f;
      ce = cudaEventElapsedTime(&ms, ctx->tm.pool[2 * i], ctx->tm.pool[2 * i + 1]);
      if (ce != cudaSuccess)
        return fail(ctx, GS_E_CUDA, std::string("cudaEventElapsedTime: ") + cudaGetErrorName(ce));
      ctx->last_times.ms[ctx->tm.phase[i]] += ms;
      ctx->last_times.count[ctx->tm.phase[i]] += 1;
    }
    // in-kernel device-clock phases, added to the event-timed launches of
    // the same phase (the second pass of step i and the label writes)
    for (int i = 0; i < kLoopPhases; ++i) {
      ctx->last_times.ms[GS_PHASE_K_OFFSETS + i] += kms[i];
      ctx->last_times.count[GS_PHASE_K_OFFSETS + i] = 1;
    }
    for (int i = 0; i < kClockSteps; ++i)
      for (int c = 0; c < 2; ++c) ctx->last_times.step_ms[i][c] = kms[kLoopPhases + 2 * i + c];
  }
  return st;
}

gs_status gs_fit(gs_ctx* ctx, const void* points, gs_dtype dtype, int64_t n, int32_t* labels,
                 double* modes, int64_t modes_cap, int64_t* k_out, gs_fit_info* info) {
  return fit_entry(ctx, points, dtype, n, labels, modes, modes_cap, k_out, info, nullptr);
}

// The device the context last ran on: a change releases its buffers.
static gs_status bind_device(gs_ctx* ctx) {
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(ctx, GS_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorName(ce));
  if (ctx->device != dev) {
    ctx->release_device();
    ctx->device = dev;
  }
  return GS_OK;
}

// The context's feature buffer of `words` doubles (the run of an image call
// fills it: the features, then any position products).
static gs_status feature_space(gs_ctx* ctx, int64_t words) {
  gs_status st = bind_device(ctx);
  if (st != GS_OK) return st;
  cudaError_t ce = ctx->feat.ensure((size_t)words);
  if (ce != cudaSuccess)
    return fail(ctx, ce == cudaErrorMemoryAllocation ? GS_E_NOMEM : GS_E_CUDA,
                std::string("image features: ") + cudaGetErrorName(ce));
  return GS_OK;
}

gs_status gs_fit_image(gs_ctx* ctx, const uint8_t* pixels, int64_t height, int64_t width,
                       int channels, double xy_scale, int32_t* labels, double* modes,
                       int64_t modes_cap, int64_t* k_out, gs_fit_info* info) {
  if (!ctx) return GS_E_INVALID;
  ctx->err.clear();
  if (!k_out) return fail(ctx, GS_E_INVALID, "k_out is NULL");
  *k_out = 0;
  if (height < 0 || width < 0 || height >= (1ll << 31) || width >= (1ll << 31) ||
      height * width >= (1ll << 31))
    return fail(ctx, GS_E_INVALID, "image size out of range");
  if (channels < 1 || channels > 8) return fail(ctx, GS_E_INVALID, "channels out of range");
  if (!(xy_scale >= 0) || !std::isfinite(xy_scale))
    return fail(ctx, GS_E_INVALID, "xy_scale must be 0 or finite and > 0");
  const bool xy = xy_scale > 0;
  if (channels + (xy ? 2 : 0) != ctx->d)
    return fail(ctx, GS_E_INVALID, "the context's d is not channels (+ 2 with positions)");
  const int64_t n = height * width;
  if (n > 0 && (!pixels || !labels)) return fail(ctx, GS_E_INVALID, "NULL pixels or labels");
  if (modes_cap < 0 || (modes_cap > 0 && !modes))
    return fail(ctx, GS_E_INVALID, "modes is NULL with modes_cap > 0");
  if (n == 0) return gs_fit(ctx, nullptr, GS_IN_F64, 0, labels, modes, modes_cap, k_out, info);
  gs_status st = feature_space(ctx, n * ctx->d + (xy ? width + height : 0));
  if (st != GS_OK) return st;
  const ImgSrc img{pixels, width, channels, xy, xy_scale, xy ? ctx->feat.p + n * ctx->d : nullptr};
  return fit_entry(ctx, ctx->feat.p, GS_IN_F64, n, labels, modes, modes_cap, k_out, info, &img);
}

gs_status gs_fit_images_host(gs_ctx* ctx, int count, const uint8_t* const* images, int64_t height,
                             int64_t width, int channels, double xy_scale, int32_t* const* labels,
                             double* const* modes, int64_t modes_cap, int64_t* k_out,
                             gs_fit_info* infos) {
  if (!ctx) return GS_E_INVALID;
  ctx->err.clear();
  if (count < 0) return fail(ctx, GS_E_INVALID, "count < 0");
  if (count == 0) return GS_OK;
  if (!k_out || !images || !labels) return fail(ctx, GS_E_INVALID, "NULL images, labels or k_out");
  if (height < 0 || width < 0 || height >= (1ll << 31) || width >= (1ll << 31) ||
      height * width >= (1ll << 31))
    return fail(ctx, GS_E_INVALID, "image size out of range");
  if (channels < 1 || channels > 8) return fail(ctx, GS_E_INVALID, "channels out of range");
  if (!(xy_scale >= 0) || !std::isfinite(xy_scale))
    return fail(ctx, GS_E_INVALID, "xy_scale must be 0 or finite and > 0");
  const int d = channels + (xy_scale > 0 ? 2 : 0);
  if (d != ctx->d)
    return fail(ctx, GS_E_INVALID, "the context's d is not channels (+ 2 with positions)");
  if (modes_cap < 0 || (modes_cap > 0 && !modes))
    return fail(ctx, GS_E_INVALID, "modes is NULL with modes_cap > 0");
  const int64_t n = height * width;
  for (int i = 0; i < count; ++i) {
    k_out[i] = 0;
    if (n > 0 && (!images[i] || !labels[i])) return fail(ctx, GS_E_INVALID, "NULL image or labels");
    if (modes_cap > 0 && !modes[i]) return fail(ctx, GS_E_INVALID, "NULL modes with modes_cap > 0");
  }
  if (infos) std::memset(infos, 0, sizeof(gs_fit_info) * (size_t)count);
  if (n == 0) {
    for (int i = 0; i < count; ++i)
      if (infos) infos[i].converged = 1;
    return GS_OK;
  }
  gs_status st = bind_device(ctx);
  if (st != GS_OK) return st;
  const size_t img_bytes = (size_t)n * channels;
  cudaError_t ce = cudaSuccess;
  if (!ctx->copy_stream) ce = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
  for (int b = 0; b < 2 && ce == cudaSuccess; ++b) {
    for (cudaEvent_t* e : {&ctx->up_ev[b], &ctx->done_ev[b], &ctx->down_ev[b]})
      if (ce == cudaSuccess && !*e) ce = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = ctx->himg[b].ensure(img_bytes);
    if (ce == cudaSuccess) ce = ctx->hlab[b].ensure((size_t)n);
    if (ce == cudaSuccess && modes_cap > 0) ce = ctx->hmodes[b].ensure((size_t)modes_cap * d);
  }
  if (ce != cudaSuccess)
    return fail(ctx, ce == cudaErrorMemoryAllocation ? GS_E_NOMEM : GS_E_CUDA,
                std::string("image stream buffers: ") + cudaGetErrorName(ce));
  const cudaStream_t cs = ctx->copy_stream, fs = ctx->stream;
#define GS_IMG_CU(call, what)                                                              \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      cudaStreamSynchronize(cs);                                                           \
      return fail(ctx, GS_E_CUDA, std::string(what) + ": " + cudaGetErrorName(e_));        \
    }                                                                                      \
  } while (0)
  GS_IMG_CU(cudaMemcpyAsync(ctx->himg[0].p, images[0], img_bytes, cudaMemcpyHostToDevice, cs),
            "H2D image");
  GS_IMG_CU(cudaEventRecord(ctx->up_ev[0], cs), "cudaEventRecord");
  gs_status result = GS_OK;
  for (int i = 0; i < count; ++i) {
    const int b = i & 1;
    // the next image's upload (the fit that last read that buffer is done:
    // every fit returns after its stream has finished)
    if (i + 1 < count) {
      GS_IMG_CU(cudaMemcpyAsync(ctx->himg[b ^ 1].p, images[i + 1], img_bytes,
                                cudaMemcpyHostToDevice, cs), "H2D image");
      GS_IMG_CU(cudaEventRecord(ctx->up_ev[b ^ 1], cs), "cudaEventRecord");
    }
    GS_IMG_CU(cudaStreamWaitEvent(fs, ctx->up_ev[b], 0), "cudaStreamWaitEvent");
    // this buffer's labels and modes have been read back (image i - 2)
    if (i >= 2) GS_IMG_CU(cudaStreamWaitEvent(fs, ctx->down_ev[b], 0), "cudaStreamWaitEvent");
    gs_fit_info inf;
    st = gs_fit_image(ctx, ctx->himg[b].p, height, width, channels, xy_scale, ctx->hlab[b].p,
                      modes_cap > 0 ? ctx->hmodes[b].p : nullptr, modes_cap, &k_out[i], &inf);
    if (infos) infos[i] = inf;
    if (st != GS_OK && st != GS_E_CAPACITY) {
      cudaStreamSynchronize(cs);
      return st;
    }
    if (st == GS_E_CAPACITY) result = st;
    // the read-back of image i, on the copy stream after its fit
    GS_IMG_CU(cudaEventRecord(ctx->done_ev[b], fs), "cudaEventRecord");
    GS_IMG_CU(cudaStreamWaitEvent(cs, ctx->done_ev[b], 0), "cudaStreamWaitEvent");
    GS_IMG_CU(cudaMemcpyAsync(labels[i], ctx->hlab[b].p, sizeof(int32_t) * (size_t)n,
                              cudaMemcpyDeviceToHost, cs), "D2H labels");
    const int64_t rows = k_out[i] < modes_cap ? k_out[i] : modes_cap;
    if (st == GS_OK && rows > 0)
      GS_IMG_CU(cudaMemcpyAsync(modes[i], ctx->hmodes[b].p, sizeof(double) * (size_t)(rows * d),
                                cudaMemcpyDeviceToHost, cs), "D2H modes");
    GS_IMG_CU(cudaEventRecord(ctx->down_ev[b], cs), "cudaEventRecord");
  }
#undef GS_IMG_CU
  ce = cudaStreamSynchronize(cs);
  if (ce != cudaSuccess) return fail(ctx, GS_E_CUDA, std::string("copy stream: ") + cudaGetErrorName(ce));
  return result;
}

gs_status gs_fit_image_batched(gs_ctx* ctx, const uint8_t* pixels, int channels,
                               const int64_t* offsets, int B, int32_t* labels, double* modes,
                               int64_t modes_cap, int64_t* mode_offsets, gs_fit_info* infos) {
  if (!ctx) return GS_E_INVALID;
  ctx->err.clear();
  if (channels < 1 || channels > 8) return fail(ctx, GS_E_INVALID, "channels out of range");
  if (channels != ctx->d) return fail(ctx, GS_E_INVALID, "the context's d is not channels");
  if (!offsets || !mode_offsets || !infos) return fail(ctx, GS_E_INVALID, "NULL offsets, mode_offsets or infos");
  if (B < 1 || B > kMaxBatch) return fail(ctx, GS_E_INVALID, "B out of range");
  if (offsets[0] != 0) return fail(ctx, GS_E_INVALID, "offsets[0] must be 0");
  for (int i = 0; i < B; ++i)
    if (offsets[i + 1] < offsets[i]) return fail(ctx, GS_E_INVALID, "offsets must not decrease");
  const int64_t n = offsets[B];
  if (n >= (1ll << 31)) return fail(ctx, GS_E_INVALID, "n out of range");
  if (n > 0 && (!pixels || !labels)) return fail(ctx, GS_E_INVALID, "NULL pixels or labels");
  if (n == 0)
    return gs_fit_batched(ctx, nullptr, GS_IN_F64, offsets, B, labels, modes, modes_cap,
                          mode_offsets, infos);
  gs_status st = feature_space(ctx, n * ctx->d);
  if (st != GS_OK) return st;
  const ImgSrc img{pixels, 1, channels, false, 0.0, nullptr};
  return batched_entry(ctx, ctx->feat.p, GS_IN_F64, offsets, B, labels, modes, modes_cap,
                       mode_offsets, infos, &img);
}

gs_status gs_track_window(gs_ctx* ctx, const void* frame, gs_dtype dtype, int64_t width,
                          int64_t height, const int64_t* bins, int64_t k, int64_t x0,
                          int64_t y0, int64_t x1, int64_t y1, gs_track_result* out,
                          uint8_t* present) {
  if (!ctx) return GS_E_INVALID;
  ctx->err.clear();
  if (!out) return fail(ctx, GS_E_INVALID, "out is NULL");
  out->count = 0;
  out->sum_x = out->sum_y = 0;
  out->mean_x = out->mean_y = std::nan("");
  out->min_x = out->min_y = INT64_MAX;
  out->max_x = out->max_y = INT64_MIN;
  if (width < 0 || height < 0 || k < 0 || width > (1ll << 31) || height > (1ll << 31))
    return fail(ctx, GS_E_INVALID, "negative size or count");
  if (k > 0 && !bins) return fail(ctx, GS_E_INVALID, "bins is NULL with k > 0");
  if (ctx->d > kMaxD) return fail(ctx, GS_E_INVALID, "the tracking window step needs d <= 8");
  if (dtype != GS_IN_F64 && dtype != GS_IN_F32) return fail(ctx, GS_E_INVALID, "bad dtype");
  if (present)
    for (int64_t j = 0; j < k; ++j) present[j] = 0;
  // the window, clipped to the frame
  x0 = x0 < 0 ? 0 : x0;
  y0 = y0 < 0 ? 0 : y0;
  x1 = x1 > width ? width : x1;
  y1 = y1 > height ? height : y1;
  const int64_t ww = x1 > x0 ? x1 - x0 : 0, wh = y1 > y0 ? y1 - y0 : 0;
  if (ww == 0 || wh == 0) return GS_OK;
  if (!frame) return fail(ctx, GS_E_INVALID, "frame is NULL");
  const int d = ctx->d;
  // B sorted lexicographically without duplicates; uidx maps bins[j] to it
  std::vector<int64_t> order((size_t)k);
  for (int64_t j = 0; j < k; ++j) order[(size_t)j] = j;
  auto less = [&](int64_t p, int64_t q) {
    for (int a = 0; a < d; ++a) {
      const int64_t u = bins[p * d + a], v = bins[q * d + a];
      if (u != v) return u < v;
    }
    return false;
  };
  std::sort(order.begin(), order.end(), less);
  std::vector<int64_t> ukeys;
  std::vector<int64_t> uidx((size_t)k);
  ukeys.reserve((size_t)k * d);
  int64_t nu = 0;
  for (int64_t r = 0; r < k; ++r) {
    const int64_t j = order[(size_t)r];
    if (r == 0 || less(order[(size_t)r - 1], j)) {
      for (int a = 0; a < d; ++a) ukeys.push_back(bins[j * d + a]);
      ++nu;
    }
    uidx[(size_t)j] = nu - 1;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(ctx, GS_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorName(ce));
  if (ctx->device != dev) {
    ctx->release_device();
    ctx->device = dev;
  }
  const cudaStream_t s = ctx->stream;
#define TR_CU(call, what)                                                                   \
  do {                                                                                      \
    ce = (call);                                                                            \
    if (ce != cudaSuccess)                                                                  \
      return fail(ctx, ce == cudaErrorMemoryAllocation ? GS_E_NOMEM : GS_E_CUDA,            \
                  std::string(what) + ": " + cudaGetErrorName(ce));                         \
  } while (0)
  // cell decisions: per channel, the exact faces spanning B's keys
  TrackPlan tp;
  std::memset(&tp, 0, sizeof(tp));
  size_t nthr = 0;
  for (int a = 0; a < d; ++a) {
    int64_t lo = 0, hi = -1;  // no keys: an empty span (one face)
    for (int64_t u = 0; u < nu; ++u) {
      const int64_t v = ukeys[(size_t)u * d + a];
      if (u == 0 || v < lo) lo = v;
      if (u == 0 || v > hi) hi = v;
    }
    if (hi - lo >= (1ll << 22))
      return fail(ctx, GS_E_KEYRANGE, "bins span more than 2^22 cells on one channel");
    tp.lo[a] = lo;
    tp.span[a] = (int)(hi - lo + 1);
    tp.toff[a] = (int)nthr;
    nthr += (size_t)tp.span[a] + 1;
  }
  const double lim = 4.0e15 * ctx->h;
  std::memcpy(&tp.lim_bits, &lim, 8);
  tp.inv_h = (float)(1.0 / ctx->h);
  // [TrackAcc | nu * d keys | faces | nu flags], 16-byte aligned pieces
  const size_t off_bins = (sizeof(TrackAcc) + 15) & ~size_t(15);
  const size_t off_thr = off_bins + sizeof(int64_t) * (size_t)nu * d;
  const size_t off_flags = off_thr + sizeof(int64_t) * nthr;
  const size_t bytes = off_flags + (size_t)(nu > 0 ? nu : 1);
  TR_CU(ctx->tbuf.ensure((bytes + 15) / 16), "alloc track buffers");
  if (ctx->h_track_cap < bytes) {
    if (ctx->h_track) cudaFreeHost(ctx->h_track);
    ctx->h_track = nullptr;
    ctx->h_track_cap = 0;
    TR_CU(cudaHostAlloc((void**)&ctx->h_track, bytes, cudaHostAllocDefault), "alloc track staging");
    ctx->h_track_cap = bytes;
  }
  unsigned char* hb = ctx->h_track;
  unsigned char* db = reinterpret_cast<unsigned char*>(ctx->tbuf.p);
  TrackAcc* h_acc = reinterpret_cast<TrackAcc*>(hb);
  h_acc->count = 0;
  h_acc->bad = 0;
  h_acc->sum_x = h_acc->sum_y = 0;
  h_acc->min_x = h_acc->min_y = INT64_MAX;
  h_acc->max_x = h_acc->max_y = INT64_MIN;
  if (nu > 0) std::memcpy(hb + off_bins, ukeys.data(), sizeof(int64_t) * (size_t)nu * d);
  int64_t* hthr = reinterpret_cast<int64_t*>(hb + off_thr);
  for (int a = 0; a < d; ++a)
    for (int j = 0; j <= tp.span[a]; ++j)
      hthr[tp.toff[a] + j] = plan_ord_of(plan_face(tp.lo[a] + j, ctx->h));
  std::memset(hb + off_flags, 0, (size_t)(nu > 0 ? nu : 1));
  TR_CU(cudaMemcpyAsync(db, hb, bytes, cudaMemcpyHostToDevice, s), "H2D track inputs");
  TR_CU(launch_track(frame, dtype == GS_IN_F32, d, width, x0, y0, ww, wh, tp,
                     reinterpret_cast<const int64_t*>(db + off_thr),
                     reinterpret_cast<const int64_t*>(db + off_bins), nu,
                     reinterpret_cast<TrackAcc*>(db), db + off_flags, s), "k_track");
  // the accumulators and the flags back (the keys between them come along)
  TR_CU(cudaMemcpyAsync(hb, db, bytes, cudaMemcpyDeviceToHost, s), "D2H track results");
  TR_CU(cudaStreamSynchronize(s), "sync track");
  const uint8_t* upresent = hb + off_flags;
#undef TR_CU
  if (h_acc->bad) {
    out->count = -1;
    return fail(ctx, GS_E_INVALID, "a colour in the window is not finite or has |c| >= 4e15 h");
  }
  out->count = (int64_t)h_acc->count;
  out->sum_x = h_acc->sum_x;
  out->sum_y = h_acc->sum_y;
  if (out->count > 0) {
    out->mean_x = (double)out->sum_x / (double)out->count;
    out->mean_y = (double)out->sum_y / (double)out->count;
  }
  out->min_x = h_acc->min_x;
  out->max_x = h_acc->max_x;
  out->min_y = h_acc->min_y;
  out->max_y = h_acc->max_y;
  if (present)
    for (int64_t j = 0; j < k; ++j) present[j] = upresent[(size_t)uidx[(size_t)j]];
  return GS_OK;
}

// gs_fit_batched, and the batched image call (img: `points` is the
// context's feature buffer, which the run fills).
static gs_status batched_entry(gs_ctx* ctx, const void* points, gs_dtype dtype,
                               const int64_t* offsets, int B, int32_t* labels, double* modes,
                               int64_t modes_cap, int64_t* mode_offsets, gs_fit_info* infos,
                               const ImgSrc* img) {
  if (!ctx) return GS_E_INVALID;
  ctx->err.clear();
  if (!offsets || !mode_offsets || !infos) return fail(ctx, GS_E_INVALID, "NULL offsets, mode_offsets or infos");
  if (B < 1 || B > kMaxBatch) return fail(ctx, GS_E_INVALID, "B out of range");
  if (B > 1 && ctx->d > kMaxD) return fail(ctx, GS_E_INVALID, "batched runs need d <= 8");
  if (B > 1 && ctx->update == GS_UPDATE_SEQUENTIAL)
    return fail(ctx, GS_E_INVALID, "the sequential update runs on one point set only (B = 1)");
  if (offsets[0] != 0) return fail(ctx, GS_E_INVALID, "offsets[0] must be 0");
  for (int i = 0; i < B; ++i)
    if (offsets[i + 1] < offsets[i]) return fail(ctx, GS_E_INVALID, "offsets must not decrease");
  const int64_t n = offsets[B];
  if (n >= (1ll << 31)) return fail(ctx, GS_E_INVALID, "n out of range");
  if (dtype != GS_IN_F64 && dtype != GS_IN_F32) return fail(ctx, GS_E_INVALID, "bad dtype");
  if (modes_cap < 0 || (modes_cap > 0 && !modes))
    return fail(ctx, GS_E_INVALID, "modes is NULL with modes_cap > 0");
  if (n > 0 && (!points || !labels)) return fail(ctx, GS_E_INVALID, "NULL points or labels");
  std::memset(infos, 0, sizeof(gs_fit_info) * (size_t)B);
  for (int i = 0; i <= B; ++i) mode_offsets[i] = 0;
  ctx->tm.reset();
  std::memset(&ctx->last_times, 0, sizeof(ctx->last_times));
  if (n == 0) {
    for (int i = 0; i < B; ++i) infos[i].converged = 1;
    return GS_OK;
  }
  if (B == 1) {
    int64_t k = 0;
    gs_status st = fit_entry(ctx, points, dtype, n, labels, modes, modes_cap, &k, &infos[0], img);
    mode_offsets[1] = k;
    return st;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(ctx, GS_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorName(ce));
  if (ctx->device != dev) {
    ctx->release_device();
    ctx->device = dev;
  }
  FitArgs a;
  a.d = ctx->d;
  a.h = ctx->h;
  a.max_iter = ctx->max_iter;
  a.stream = ctx->stream;
  a.points = points;
  a.f32 = dtype == GS_IN_F32;
  a.n = n;
  a.labels = labels;
  a.modes = modes;
  a.modes_cap = modes_cap;
  a.tune = ctx->tune;
  a.mixed = ctx->prec == GS_FP32_MIXED;
  a.B = B;
  a.offsets = offsets;
  a.infos = infos;
  a.mode_offsets = mode_offsets;
  set_image(a, img);
  gs_fit_info total;
  std::memset(&total, 0, sizeof(total));
  int64_t k = 0;
  return fit_pipeline(a, ctx->ws, nullptr, &k, &total, nullptr, &ctx->err);
}

gs_status gs_fit_batched(gs_ctx* ctx, const void* points, gs_dtype dtype, const int64_t* offsets,
                         int B, int32_t* labels, double* modes, int64_t modes_cap,
                         int64_t* mode_offsets, gs_fit_info* infos) {
  return batched_entry(ctx, points, dtype, offsets, B, labels, modes, modes_cap, mode_offsets,
                       infos, nullptr);
}

gs_status gs_fit_sweep(gs_ctx* ctx, const void* points, gs_dtype dtype, int64_t n,
                       const double* hs, int B, int32_t* labels, double* modes,
                       int64_t modes_cap, int64_t* mode_offsets, gs_fit_info* infos) {
  if (!ctx) return GS_E_INVALID;
  ctx->err.clear();
  if (!hs || !mode_offsets || !infos) return fail(ctx, GS_E_INVALID, "NULL hs, mode_offsets or infos");
  if (B < 1 || B > kMaxBatch) return fail(ctx, GS_E_INVALID, "B out of range");
  for (int i = 0; i < B; ++i)
    if (!(hs[i] > 0) || !std::isfinite(hs[i])) return fail(ctx, GS_E_INVALID, "h not finite and > 0");
  if (n < 0 || n * (int64_t)B >= (1ll << 31)) return fail(ctx, GS_E_INVALID, "B x n out of range");
  if (dtype != GS_IN_F64 && dtype != GS_IN_F32) return fail(ctx, GS_E_INVALID, "bad dtype");
  if (modes_cap < 0 || (modes_cap > 0 && !modes))
    return fail(ctx, GS_E_INVALID, "modes is NULL with modes_cap > 0");
  if (n > 0 && (!points || !labels)) return fail(ctx, GS_E_INVALID, "NULL points or labels");
  if (ctx->prec != GS_FP64 || ctx->update != GS_UPDATE_PARALLEL)
    return fail(ctx, GS_E_INVALID, "a bandwidth sweep runs in GS_FP64 with the parallel update");
  if (ctx->d > kMaxD) return fail(ctx, GS_E_INVALID, "a bandwidth sweep needs d <= 8");
  std::memset(infos, 0, sizeof(gs_fit_info) * (size_t)B);
  for (int i = 0; i <= B; ++i) mode_offsets[i] = 0;
  ctx->tm.reset();
  std::memset(&ctx->last_times, 0, sizeof(ctx->last_times));
  if (n == 0) {
    for (int i = 0; i < B; ++i) infos[i].converged = 1;
    return GS_OK;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(ctx, GS_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorName(ce));
  if (ctx->device != dev) {
    ctx->release_device();
    ctx->device = dev;
  }
  FitArgs a;
  a.d = ctx->d;
  a.h = hs[0];
  a.max_iter = ctx->max_iter;
  a.stream = ctx->stream;
  a.points = points;
  a.f32 = dtype == GS_IN_F32;
  a.labels = labels;
  a.modes = modes;
  a.modes_cap = modes_cap;
  a.tune = ctx->tune;
  if (B == 1) {
    // one bandwidth: the plain run with that h
    a.n = n;
    int64_t k = 0;
    gs_status st = fit_pipeline(a, ctx->ws, nullptr, &k, &infos[0], nullptr, &ctx->err);
    mode_offsets[1] = k;
    return st;
  }
  std::vector<int64_t> offsets((size_t)B + 1);
  for (int i = 0; i <= B; ++i) offsets[(size_t)i] = (int64_t)i * n;
  a.n = n * B;
  a.B = B;
  a.offsets = offsets.data();
  a.infos = infos;
  a.mode_offsets = mode_offsets;
  a.sweep_h = hs;
  a.n0 = (uint32_t)n;
  gs_fit_info total;
  std::memset(&total, 0, sizeof(total));
  int64_t k = 0;
  return fit_pipeline(a, ctx->ws, nullptr, &k, &total, nullptr, &ctx->err);
}

}  // extern "C"
