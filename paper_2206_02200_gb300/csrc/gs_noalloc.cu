// gs_noalloc.cu -- gs_fit_noalloc: the GridShift run of gs_fit with every
// piece of device scratch carved out of one file-scope static device array, for
// callers that must not allocate device or pinned memory (see the declaration
// in include/gridshift.h).  The steps and kernels are the ones gs_fit runs
// (gs_driver.cu); only the source of the buffers differs.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/gridshift.h"
#include "gs_driver.h"

using namespace gs;

namespace {

// The static scratch.  Every GPU that loads this library holds it until the
// process exits.  Host code must not use the symbol itself as a device
// address: every call obtains the address with cudaGetSymbolAddress, with the
// calling device current.  The address belongs to the context that is current
// then; it is not kept between calls, because a device reset (or another
// context made current on the same device) moves the array.
constexpr size_t kScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr size_t kThrMax = 8192;   // face-table entries (sum over axes of span + 1)
constexpr size_t kProbeMax = 6561; // 3^8 neighbour offsets

std::mutex g_mu;  // serialises calls: they share g_scratch and the host buffers below
int64_t g_words[kThrMax + 2 * kProbeMax];
DevFlags g_hflags;
LoopResult g_hres;

// Bump allocator over the static scratch (256-byte aligned pieces).
struct Carve {
  unsigned char* base;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    const size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    return reinterpret_cast<T*>(base + off);
  }
};

BinTable carve_bin_table(Carve& c, uint32_t cap, uint32_t lmax, int d) {
  BinTable t;
  t.key = c.take<uint64_t>(cap);
  t.cnt = c.take<uint32_t>(cap);
  t.off = c.take<uint32_t>(cap);
  t.id = c.take<uint32_t>(cap);
  t.acc = c.take<uint64_t>((size_t)cap * d * 4);
  t.list = c.take<uint32_t>(lmax);
  t.cap = cap;
  return t;
}

LevelTable carve_level_table(Carve& c, uint32_t cap, uint32_t lmax, int d) {
  LevelTable t;
  t.key = c.take<uint64_t>(cap);
  t.id = c.take<uint32_t>(cap);
  t.row = c.take<ulonglong2>((size_t)cap * (d + 1));
  t.acc = c.take<uint64_t>((size_t)cap * d * 4);
  t.list = c.take<uint32_t>(lmax);
  t.cap = cap;
  return t;
}

// Lays out every buffer of one run for at most M cells (tables of 2M slots)
// and n points from `base` (null: sizes only); returns the bytes used.
size_t layout(unsigned char* base, int64_t n, int d, int max_iter, uint32_t M, size_t thr_words,
              int nprobe, Bufs* out) {
  Carve c{base};
  Bufs tmp;
  Bufs& B = out ? *out : tmp;
  const uint32_t cap = 2 * M;
  B.flags = c.take<DevFlags>(1);
  B.st = c.take<IterState>(max_iter + 2);
  B.res = c.take<LoopResult>(1);
  B.bar = c.take<GridBar>(1);
  B.thr = c.take<int64_t>(thr_words);
  B.dtab = c.take<uint64_t>(2 * (size_t)nprobe);
  B.slot0 = c.take<uint32_t>(n);
  B.perm = c.take<uint32_t>(n);
  B.blocksum = c.take<uint32_t>(kMaxLoopGrid);
  B.t0 = carve_bin_table(c, cap, M, d);
  B.t0_maxcells = M;
  for (int i = 0; i < 3; ++i) B.tab[i] = carve_level_table(c, cap, M, d);
  B.capAB = cap;
  for (int i = 0; i < 2; ++i) {
    B.cells[i].key = c.take<uint64_t>(M);
    B.cells[i].cnt = c.take<uint32_t>(M);
    B.pslot[i] = c.take<uint32_t>(M);
  }
  B.qlist = c.take<uint32_t>((size_t)M * 3);
  B.forest = c.take<uint32_t>((size_t)M * (max_iter + 1));
  B.forest2 = c.take<uint32_t>((size_t)M * (max_iter + 1));
  B.labslot = c.take<uint32_t>(cap);
  B.rank = c.take<uint32_t>(M);
  B.filter = c.take<uint32_t>(2 * kFilterWords);
  B.skey = c.take<uint64_t>(M);
  B.skey2 = c.take<uint64_t>(M);
  B.sval = c.take<uint32_t>(M);
  B.sval2 = c.take<uint32_t>(M);
  B.shist = c.take<uint32_t>(radix_hist_words(M));
  return c.used;
}

cudaError_t clear_bin_table(const BinTable& t, int d, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(t.key, 0xFF, sizeof(uint64_t) * t.cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.cnt, 0, sizeof(uint32_t) * t.cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.acc, 0, sizeof(uint64_t) * t.cap * d * 4, s);
  return e;
}

cudaError_t clear_level_table(const LevelTable& t, int d, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(t.key, 0xFF, sizeof(uint64_t) * t.cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.row, 0, sizeof(ulonglong2) * t.cap * (d + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.acc, 0, sizeof(uint64_t) * t.cap * d * 4, s);
  return e;
}

// The workspace of one call: everything is laid out at once in prepare(), for
// the largest cell bound that fits; nothing is allocated.
struct StaticWorkspace : public Workspace {
  unsigned char* base;
  Bufs laid;
  explicit StaticWorkspace(unsigned char* b) : base(b) {}

  DevFlags* host_flags() override { return &g_hflags; }
  LoopResult* host_result() override { return &g_hres; }
  gs_status host_words(size_t words, int64_t** out, std::string*) override {
    if (words > kThrMax + 2 * kProbeMax) return GS_E_SCRATCH;
    *out = g_words;
    return GS_OK;
  }
  gs_status begin(Bufs& b, std::string*) override {
    b.flags = reinterpret_cast<DevFlags*>(base);  // where layout() puts them
    return GS_OK;
  }
  size_t plan_thr_cap() const override { return kThrMax; }

  gs_status prepare(int64_t n, int d, int max_iter, size_t thr_words, int nprobe,
                    uint64_t m_bound, cudaStream_t s, Bufs& b, std::string*) override {
    if (thr_words > kThrMax || (size_t)nprobe > kProbeMax) return GS_E_SCRATCH;
    // the largest cell bound M (a power of two, at most what the data can
    // need) whose workspace fits the scratch
    uint32_t M = 64;
    while (M < m_bound && M < (1u << 30)) M <<= 1;
    while (M > 64 && layout(nullptr, n, d, max_iter, M, thr_words, nprobe, nullptr) > kScratchBytes)
      M >>= 1;
    if (layout(nullptr, n, d, max_iter, M, thr_words, nprobe, nullptr) > kScratchBytes)
      return GS_E_SCRATCH;
    layout(base, n, d, max_iter, M, thr_words, nprobe, &laid);
    // the scratch keeps the previous call's contents: clear what must start
    // empty or zero
    if (clear_bin_table(laid.t0, d, s) != cudaSuccess) return GS_E_CUDA;
    for (int i = 0; i < 3; ++i)
      if (clear_level_table(laid.tab[i], d, s) != cudaSuccess) return GS_E_CUDA;
    b = laid;
    return GS_OK;
  }
  gs_status regrow_bin(int, cudaStream_t, Bufs&, std::string*) override { return GS_E_SCRATCH; }
  gs_status levels(uint32_t m0, int, int, cudaStream_t, Bufs& b, std::string*) override {
    if (m0 > laid.t0_maxcells) return GS_E_SCRATCH;
    b = laid;
    return GS_OK;
  }
  gs_status sort_space(uint32_t, Bufs& b, std::string*) override {
    b = laid;
    return GS_OK;
  }
  gs_status batch_space(int, Bufs&, uint32_t**, std::string*) override { return GS_E_INVALID; }
  void mark_dirty(bool) override {}
  void note_cells(uint32_t) override {}
  gs_status shift_rows(uint32_t, int, Bufs&, std::string*) override { return GS_E_INVALID; }
  gs_status sweep_space(int, Bufs&, std::string*) override { return GS_E_INVALID; }
};

}  // namespace

extern "C" gs_status gs_fit_noalloc(int d, double h, int max_iter, void* cuda_stream,
                                    const void* points, gs_dtype dtype, int64_t n,
                                    int32_t* labels, double* modes, int64_t modes_cap,
                                    int64_t* k_out, gs_fit_info* info) {
  if (!k_out) return GS_E_INVALID;
  *k_out = 0;
  if (d < 1 || d > kMaxD || !(h > 0) || !std::isfinite(h) || max_iter < 0 || max_iter > 100000)
    return GS_E_INVALID;
  if (n < 0 || n >= (1ll << 31)) return GS_E_INVALID;
  if (dtype != GS_IN_F64 && dtype != GS_IN_F32) return GS_E_INVALID;
  if (modes_cap < 0 || (modes_cap > 0 && !modes)) return GS_E_INVALID;
  if (n > 0 && (!points || !labels)) return GS_E_INVALID;
  gs_fit_info inf;
  std::memset(&inf, 0, sizeof(inf));
  if (n == 0) {
    inf.converged = 1;
    if (info) *info = inf;
    return GS_OK;
  }
  // the per-point arrays (cell slot and counting-sort position) alone must fit
  if ((size_t)n * 2 * sizeof(uint32_t) + (size_t(1) << 20) > kScratchBytes) return GS_E_SCRATCH;

  std::lock_guard<std::mutex> lock(g_mu);
  // set-up, on every call: the device address of the static scratch in the
  // context current on this thread (a lookup; nothing is allocated)
  void* scratch = nullptr;
  if (cudaGetSymbolAddress(&scratch, g_scratch) != cudaSuccess || !scratch) return GS_E_CUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  FitArgs a;
  a.d = d;
  a.h = h;
  a.max_iter = max_iter;
  a.stream = s;
  a.points = points;
  a.f32 = dtype == GS_IN_F32;
  a.n = n;
  a.labels = labels;
  a.modes = modes;
  a.modes_cap = modes_cap;
  StaticWorkspace ws(static_cast<unsigned char*>(scratch));
  gs_status st = fit_pipeline(a, ws, nullptr, k_out, &inf, nullptr, nullptr);
  // no work of this call may still run when the next one reuses the scratch
  if (st != GS_OK) cudaStreamSynchronize(s);
  if (info) *info = inf;
  return st;
}
