// gs_api.cu -- host side of the C ABI declared in include/gridshift.h: argument
// checks, the per-call plan (packed keys, face tables, fixed-point windows),
// the device workspace and the order of kernel launches of one GridShift run.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gridshift.h"
#include "gs_kernels.h"

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

// Device storage of a hash table (see gs::Table).
struct TableBuf {
  DBuf<uint64_t> key;
  DBuf<uint32_t> id, cnt, list;
  DBuf<uint64_t> acc;
  uint32_t cap = 0;
  int d = 0;
  // Allocates capacity c (power of two) for d-dimensional sums and a list of
  // up to lmax cells; a new or regrown table is cleared.
  cudaError_t ensure(uint32_t c, int dd, uint32_t lmax, cudaStream_t s) {
    cudaError_t e;
    if (c > cap || dd != d) {
      key.release(); id.release(); cnt.release(); acc.release();
      if ((e = key.ensure(c)) != cudaSuccess) return e;
      if ((e = id.ensure(c)) != cudaSuccess) return e;
      if ((e = cnt.ensure(c)) != cudaSuccess) return e;
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
    if ((e = cudaMemsetAsync(cnt.p, 0, sizeof(uint32_t) * cnt.cap, s)) != cudaSuccess) return e;
    return cudaMemsetAsync(acc.p, 0, sizeof(uint64_t) * acc.cap, s);
  }
  Table view() const { return Table{key.p, id.p, cnt.p, acc.p, list.p, cap}; }
  void release() {
    key.release(); id.release(); cnt.release(); acc.release(); list.release();
    cap = 0;
  }
};

struct CellBuf {
  DBuf<uint64_t> key;
  DBuf<uint32_t> cnt;
  DBuf<double> cs;
  cudaError_t ensure(uint32_t m, int d) {
    cudaError_t e;
    if ((e = key.ensure(m)) != cudaSuccess) return e;
    if ((e = cnt.ensure(m)) != cudaSuccess) return e;
    return cs.ensure((size_t)m * d);
  }
  Cells view() const { return Cells{key.p, cnt.p, cs.p}; }
  void release() { key.release(); cnt.release(); cs.release(); }
};

uint32_t pow2_at_least(uint64_t v, uint32_t lo) {
  uint64_t c = lo;
  while (c < v && c < (1ull << 31)) c <<= 1;
  return (uint32_t)c;
}

int64_t ord_of(double x) {
  if (x == 0.0) x = 0.0;
  int64_t s;
  std::memcpy(&s, &x, 8);
  return s ^ ((s >> 63) & 0x7FFFFFFFFFFFFFFFll);
}

double from_ord(int64_t o) {
  int64_t s = o ^ ((o >> 63) & 0x7FFFFFFFFFFFFFFFll);
  double x;
  std::memcpy(&x, &s, 8);
  return x;
}

// The least double t with t >= q * h (exactly); the error of the rounded
// product q * h is itself a double, obtained exactly by one fused multiply-add.
double face(int64_t q, double h) {
  double qd = (double)q;
  double p = qd * h;
  double r = std::fma(qd, h, -p);
  if (r > 0) p = std::nextafter(p, INFINITY);
  return p;
}

// floor(x / h) of the exact quotient: the q with face(q) <= x < face(q + 1).
int64_t floor_div(double x, double h) {
  int64_t q = (int64_t)std::floor(x / h);
  for (int i = 0; i < 4 && face(q, h) > x; ++i) --q;
  for (int i = 0; i < 4 && face(q + 1, h) <= x; ++i) ++q;
  return q;
}

int bitlen(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

// CUDA events around the launch groups of one call (opt-in, gs_set_timing).
struct PhaseTimer {
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
  void release() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    phase.clear();
    used = 0;
  }
};

}  // namespace

struct gs_ctx {
  int d = 0;
  double h = 0;
  int max_iter = 0;
  gs_precision prec = GS_FP64;
  cudaStream_t stream = nullptr;
  int device = -1;
  std::string err;
  bool timing = false;
  bool dirty = false;  // a call stopped between binning and its end: tables need clearing
  PhaseTimer tm;
  gs_phase_times last_times{};
  int64_t launches = 0;  // kernels launched by the current call

  DBuf<DevFlags> flags;
  DBuf<IterState> st;
  DBuf<int64_t> thr;
  DBuf<uint64_t> dtab;
  DBuf<uint32_t> slot0;
  TableBuf t0, tab[2];
  CellBuf cells[2];
  DBuf<double> sp;
  DBuf<uint64_t> nkey;
  DBuf<uint32_t> pslot, forest, forest2, labslot, rank;
  DBuf<uint64_t> skey, skey2;
  DBuf<uint32_t> sval, sval2, shist;

  DevFlags* h_flags = nullptr;  // pinned
  IterState* h_st = nullptr;    // pinned, max_iter + 2 entries
  int64_t* h_thr = nullptr;     // pinned staging of thr + dtab
  size_t h_thr_cap = 0;

  void release_device() {
    flags.release(); st.release(); thr.release(); dtab.release(); slot0.release();
    t0.release(); tab[0].release(); tab[1].release(); cells[0].release(); cells[1].release();
    sp.release(); nkey.release(); pslot.release(); forest.release(); forest2.release();
    labslot.release(); rank.release(); skey.release(); skey2.release(); sval.release();
    sval2.release(); shist.release();
    tm.release();
    if (h_flags) cudaFreeHost(h_flags);
    if (h_st) cudaFreeHost(h_st);
    if (h_thr) cudaFreeHost(h_thr);
    h_flags = nullptr;
    h_st = nullptr;
    h_thr = nullptr;
    h_thr_cap = 0;
  }
};

namespace {

gs_status fail(gs_ctx* c, gs_status s, const std::string& msg) {
  c->err = msg;
  return s;
}

gs_status cuda_fail(gs_ctx* c, cudaError_t e, const char* where) {
  c->err = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? GS_E_NOMEM : GS_E_CUDA;
}

#define GS_CU(call, where)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

// A kernel launch: counted, and checked like any runtime call.
#define GS_LAUNCH(call, where, nk) \
  do {                             \
    GS_CU(call, where);            \
    ctx->launches += (nk);         \
  } while (0)

// Start and end of a timed phase (events on the call's stream, if timing is on).
#define GS_PH_BEGIN(ph)                                   \
  do {                                                    \
    if (ctx->timing) {                                    \
      GS_CU(ctx->tm.record(s), "cudaEventRecord");        \
      ctx->tm.phase.push_back(ph);                        \
    }                                                     \
  } while (0)
#define GS_PH_END(ph) \
  do {                \
    if (ctx->timing) GS_CU(ctx->tm.record(s), "cudaEventRecord"); \
  } while (0)

// Host plan of one call: packed-key layout, face tables and fixed-point windows.
gs_status make_plan(gs_ctx* ctx, const DevFlags& fl, int64_t n, Plan& P,
                    std::vector<int64_t>& thr, std::vector<uint64_t>& dtab, uint64_t& span_prod,
                    int& total_bits) {
  const int d = ctx->d;
  const double h = ctx->h;
  std::memset(&P, 0, sizeof(P));
  P.d = d;
  int bits[kMaxD];
  int clog2n = 0;
  while ((1ll << clog2n) < n) ++clog2n;
  span_prod = 1;
  thr.clear();
  for (int a = 0; a < d; ++a) {
    double lo = from_ord(fl.min_ord[a]), hi = from_ord(fl.max_ord[a]);
    if (!(std::fabs(lo / h) < 4.0e15) || !(std::fabs(hi / h) < 4.0e15))
      return fail(ctx, GS_E_KEYRANGE, "a coordinate divided by h exceeds 2^52");
    // The key box of the data, widened by one cell on each side: centroids are
    // convex combinations of the points (Eq. 1, Eq. 3) and leave the data's box
    // by at most a few roundings, never by a whole cell.
    int64_t kmin = floor_div(lo, h) - 1, kmax = floor_div(hi, h) + 1;
    int64_t span = kmax - kmin + 1;
    if (span > (1ll << 22))
      return fail(ctx, GS_E_KEYRANGE, "more than 2^22 cells along one axis");
    P.kmin[a] = kmin;
    P.span[a] = (int)span;
    bits[a] = bitlen((uint64_t)span + 1);
    P.thr_off[a] = (int)thr.size();
    for (int64_t j = 0; j <= span; ++j) thr.push_back(ord_of(face(kmin + j, h)));
    span_prod = span_prod > (1ull << 40) ? span_prod : span_prod * (uint64_t)span;
    double ma;
    uint64_t mb = fl.maxabs[a];
    std::memcpy(&ma, &mb, 8);
    int e = 0;
    if (ma > 0) std::frexp(ma, &e);  // ma < 2^e
    P.L[a] = e + clog2n - 126;
  }
  total_bits = 0;
  for (int a = d - 1; a >= 0; --a) {
    P.off[a] = total_bits;
    total_bits += bits[a];
  }
  if (total_bits > 63) return fail(ctx, GS_E_KEYRANGE, "packed cell key needs more than 63 bits");
  int np = 1;
  for (int a = 0; a < d; ++a) np *= 3;
  P.nprobe = np;
  P.center = (np - 1) / 2;
  dtab.resize(np);
  for (int p = 0; p < np; ++p) {
    int64_t delta = 0;
    int rest = p;
    for (int a = d - 1; a >= 0; --a) {  // axis 0 is the slowest digit
      int v = rest % 3 - 1;
      rest /= 3;
      delta += (int64_t)v * (int64_t)(1ull << P.off[a]);
    }
    dtab[p] = (uint64_t)delta;
  }
  return GS_OK;
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
  if (d < 1 || d > kMaxD || !(h > 0) || !std::isfinite(h) || max_iter < 0 || max_iter > 100000)
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
  if (p != GS_FP64) return fail(ctx, GS_E_INVALID, "only GS_FP64 is implemented");
  ctx->prec = p;
  return GS_OK;
}

gs_status gs_set_stream(gs_ctx* ctx, void* cuda_stream) {
  if (!ctx) return GS_E_INVALID;
  ctx->stream = (cudaStream_t)cuda_stream;
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

gs_status gs_fit(gs_ctx* ctx, const void* points, gs_dtype dtype, int64_t n, int32_t* labels,
                 double* modes, int64_t modes_cap, int64_t* k_out, gs_fit_info* info) {
  if (!ctx) return GS_E_INVALID;
  ctx->err.clear();
  if (!k_out) return fail(ctx, GS_E_INVALID, "k_out is NULL");
  if (n < 0 || n >= (1ll << 31)) return fail(ctx, GS_E_INVALID, "n out of range");
  if (dtype != GS_IN_F64 && dtype != GS_IN_F32) return fail(ctx, GS_E_INVALID, "bad dtype");
  if (modes_cap < 0 || (modes_cap > 0 && !modes))
    return fail(ctx, GS_E_INVALID, "modes is NULL with modes_cap > 0");
  if (n > 0 && (!points || !labels)) return fail(ctx, GS_E_INVALID, "NULL points or labels");
  gs_fit_info inf;
  std::memset(&inf, 0, sizeof(inf));
  *k_out = 0;
  ctx->launches = 0;
  ctx->tm.used = 0;
  ctx->tm.phase.clear();
  std::memset(&ctx->last_times, 0, sizeof(ctx->last_times));
  if (n == 0) {
    inf.converged = 1;
    if (info) *info = inf;
    return GS_OK;
  }
  const int d = ctx->d;
  const bool f32 = dtype == GS_IN_F32;
  cudaStream_t s = ctx->stream;
  int dev = 0;
  GS_CU(cudaGetDevice(&dev), "cudaGetDevice");
  if (ctx->device != dev) {
    ctx->release_device();
    ctx->device = dev;
  }
  const int max_iter = ctx->max_iter;

  // pinned host mirrors
  if (!ctx->h_flags) GS_CU(cudaMallocHost((void**)&ctx->h_flags, sizeof(DevFlags)), "cudaMallocHost");
  if (!ctx->h_st)
    GS_CU(cudaMallocHost((void**)&ctx->h_st, sizeof(IterState) * (max_iter + 2)), "cudaMallocHost");
  GS_CU(ctx->flags.ensure(1), "alloc flags");
  GS_CU(ctx->st.ensure(max_iter + 2), "alloc state");

  // a0: key range, fixed-point window, finiteness
  DevFlags* hf = ctx->h_flags;
  std::memset(hf, 0, sizeof(DevFlags));
  for (int a = 0; a < kMaxD; ++a) {
    hf->min_ord[a] = INT64_MAX;
    hf->max_ord[a] = INT64_MIN;
  }
  GS_CU(cudaMemcpyAsync(ctx->flags.p, hf, sizeof(DevFlags), cudaMemcpyHostToDevice, s), "H2D flags");
  GS_PH_BEGIN(GS_PHASE_RANGE);
  GS_LAUNCH(launch_range(points, f32, n, d, ctx->flags.p, s), "k_range", 1);
  GS_PH_END(GS_PHASE_RANGE);
  GS_CU(cudaMemcpyAsync(hf, ctx->flags.p, sizeof(DevFlags), cudaMemcpyDeviceToHost, s), "D2H flags");
  GS_CU(cudaStreamSynchronize(s), "sync range");
  if (hf->bad) return fail(ctx, GS_E_INVALID, "non-finite input coordinate");

  Plan P;
  std::vector<int64_t> thr;
  std::vector<uint64_t> dtab;
  uint64_t span_prod = 0;
  int total_bits = 0;
  gs_status ps = make_plan(ctx, *hf, n, P, thr, dtab, span_prod, total_bits);
  if (ps != GS_OK) return ps;

  // upload face table and neighbour offsets through pinned staging
  size_t words = thr.size() + dtab.size();
  if (words > ctx->h_thr_cap) {
    if (ctx->h_thr) cudaFreeHost(ctx->h_thr);
    ctx->h_thr = nullptr;
    ctx->h_thr_cap = 0;
    GS_CU(cudaMallocHost((void**)&ctx->h_thr, sizeof(int64_t) * words), "cudaMallocHost");
    ctx->h_thr_cap = words;
  }
  std::memcpy(ctx->h_thr, thr.data(), sizeof(int64_t) * thr.size());
  std::memcpy(ctx->h_thr + thr.size(), dtab.data(), sizeof(uint64_t) * dtab.size());
  GS_CU(ctx->thr.ensure(thr.size()), "alloc thr");
  GS_CU(ctx->dtab.ensure(dtab.size()), "alloc dtab");
  GS_CU(cudaMemcpyAsync(ctx->thr.p, ctx->h_thr, sizeof(int64_t) * thr.size(),
                        cudaMemcpyHostToDevice, s), "H2D thr");
  GS_CU(cudaMemcpyAsync(ctx->dtab.p, ctx->h_thr + thr.size(), sizeof(uint64_t) * dtab.size(),
                        cudaMemcpyHostToDevice, s), "H2D dtab");

  // i: binning into T0 (retried with a larger table if the cells overflow it)
  GS_CU(ctx->slot0.ensure(n), "alloc slot0");
  GS_CU(cudaMemsetAsync(ctx->st.p, 0, sizeof(IterState) * (max_iter + 2), s), "memset state");
  uint64_t m_bound = (uint64_t)n < span_prod ? (uint64_t)n : span_prod;
  uint32_t cap0 = pow2_at_least(2 * m_bound, 1024);
  if (ctx->t0.cap > cap0 && ctx->t0.d == d) cap0 = ctx->t0.cap;
  if (ctx->dirty) {
    if (ctx->t0.cap) GS_CU(ctx->t0.clear(s), "clear T0");
    if (ctx->tab[0].cap) GS_CU(ctx->tab[0].clear(s), "clear table A");
    if (ctx->tab[1].cap) GS_CU(ctx->tab[1].clear(s), "clear table B");
  }
  ctx->dirty = true;
  uint32_t m0 = 0;
  for (int attempt = 0;; ++attempt) {
    uint32_t maxcells = cap0 / 2;
    GS_CU(ctx->t0.ensure(cap0, d, maxcells, s), "alloc T0");
    GS_PH_BEGIN(GS_PHASE_BIN);
    GS_LAUNCH(launch_bin(points, f32, n, P, ctx->thr.p, ctx->t0.view(), cap0 - 1, maxcells,
                         ctx->slot0.p, ctx->flags.p, s), "k_bin", 1);
    GS_PH_END(GS_PHASE_BIN);
    GS_CU(cudaMemcpyAsync(hf, ctx->flags.p, sizeof(DevFlags), cudaMemcpyDeviceToHost, s), "D2H flags");
    GS_CU(cudaStreamSynchronize(s), "sync bin");
    const uint32_t regrow = kErrOverflow | kErrTableFull;
    if (hf->err & ~regrow) {
      ctx->t0.clear(s);
      return fail(ctx, GS_E_INTERNAL, "binning hit a device bound (fixed-point window)");
    }
    if (!(hf->err & regrow)) {
      m0 = hf->m0;
      break;
    }
    if (attempt >= 4 || cap0 >= (1u << 31)) {
      ctx->t0.clear(s);
      return fail(ctx, GS_E_INTERNAL, "binning table overflow");
    }
    GS_CU(ctx->t0.clear(s), "clear T0");
    cap0 <<= 2;
    hf->err = 0;
    hf->m0 = 0;
    GS_CU(cudaMemcpyAsync(ctx->flags.p, hf, sizeof(DevFlags), cudaMemcpyHostToDevice, s), "H2D flags");
  }
  inf.m0 = m0;

  // workspace of the cell levels
  uint32_t capAB = pow2_at_least(2ull * m0, 64);
  GS_CU(ctx->tab[0].ensure(capAB, d, m0, s), "alloc table A");
  GS_CU(ctx->tab[1].ensure(capAB, d, m0, s), "alloc table B");
  GS_CU(ctx->cells[0].ensure(m0, d), "alloc cells");
  GS_CU(ctx->cells[1].ensure(m0, d), "alloc cells");
  GS_CU(ctx->sp.ensure((size_t)m0 * d), "alloc sp");
  GS_CU(ctx->nkey.ensure(m0), "alloc nkey");
  GS_CU(ctx->pslot.ensure(m0), "alloc pslot");
  GS_CU(ctx->forest.ensure((size_t)m0 * (max_iter + 1)), "alloc forest");
  GS_CU(ctx->forest2.ensure((size_t)m0 * (max_iter + 1)), "alloc forest");
  GS_CU(ctx->labslot.ensure(cap0), "alloc labslot");
  GS_CU(ctx->rank.ensure(m0), "alloc rank");

  GS_PH_BEGIN(GS_PHASE_CELLS0);
  GS_LAUNCH(launch_compact0(P, ctx->t0.view(), ctx->cells[0].view(), ctx->tab[0].view(), capAB,
                            m0, ctx->st.p, ctx->flags.p, s), "k_compact0", 1);
  GS_PH_END(GS_PHASE_CELLS0);

  // ii-v: update steps
  int t = 0;
  uint32_t m_t = m0;
  bool converged = false;
  int64_t cell_iters = 0;
  for (;;) {
    Table G = ctx->tab[t & 1].view(), M = ctx->tab[(t + 1) & 1].view();
    Cells c = ctx->cells[t & 1].view(), nx = ctx->cells[(t + 1) & 1].view();
    GS_PH_BEGIN(GS_PHASE_GATHER);
    GS_LAUNCH(launch_gather(P, ctx->thr.p, ctx->dtab.p, G, c, ctx->sp.p, ctx->nkey.p, ctx->st.p,
                            t, m_t, ctx->flags.p, s), "k_gather", 1);
    GS_PH_END(GS_PHASE_GATHER);
    GS_CU(cudaMemcpyAsync(ctx->h_st + t, ctx->st.p + t, sizeof(IterState), cudaMemcpyDeviceToHost, s),
          "D2H state");
    GS_CU(cudaStreamSynchronize(s), "sync gather");
    m_t = ctx->h_st[t].m;
    if (!ctx->h_st[t].has_nb) {
      converged = true;
      break;
    }
    if (t == max_iter) break;
    GS_PH_BEGIN(GS_PHASE_MERGE);
    GS_LAUNCH(launch_merge(P, c, ctx->sp.p, ctx->nkey.p, M, ctx->pslot.p, ctx->st.p, t, m_t,
                           ctx->flags.p, s), "k_merge", 1);
    GS_LAUNCH(launch_compact(P, M, nx, ctx->st.p, t, m_t, ctx->flags.p, s), "k_compact", 1);
    GS_LAUNCH(launch_finish(G, M, ctx->pslot.p, ctx->forest.p, ctx->st.p, t, m_t, s), "k_finish",
              1);
    GS_PH_END(GS_PHASE_MERGE);
    cell_iters += m_t;
    ++t;
  }
  const int T = t;
  GS_PH_BEGIN(GS_PHASE_LABELS);
  GS_LAUNCH(launch_final_level(ctx->tab[T & 1].view(), ctx->forest.p, ctx->st.p, T, m_t, s),
            "k_final_level", 1);
  GS_CU(cudaMemcpyAsync(ctx->h_st + T, ctx->st.p + T, sizeof(IterState), cudaMemcpyDeviceToHost, s),
        "D2H state");
  GS_CU(cudaStreamSynchronize(s), "sync final");
  const uint32_t k = ctx->h_st[T].m;
  const uint32_t baseT = ctx->h_st[T].base;
  const uint32_t nodes = baseT + k;

  // pointer jumping: every node reaches its final cell
  uint32_t* root = ctx->forest.p;
  uint32_t* other = ctx->forest2.p;
  for (int hop = 1; hop < T; hop <<= 1) {
    GS_LAUNCH(launch_jump(root, other, nodes, s), "k_jump", 1);
    uint32_t* tmp = root;
    root = other;
    other = tmp;
  }
  // number the final cells by ascending key
  Cells fin = ctx->cells[T & 1].view();
  GS_CU(ctx->skey.ensure(k), "alloc sort");
  GS_CU(ctx->skey2.ensure(k), "alloc sort");
  GS_CU(ctx->sval.ensure(k), "alloc sort");
  GS_CU(ctx->sval2.ensure(k), "alloc sort");
  GS_CU(ctx->shist.ensure(radix_hist_words(k)), "alloc sort");
  GS_LAUNCH(launch_iota_keys(fin, ctx->skey.p, ctx->sval.p, k, s), "k_iota_keys", 1);
  GS_LAUNCH(radix_sort(ctx->skey.p, ctx->sval.p, ctx->skey2.p, ctx->sval2.p, ctx->shist.p, k,
                       total_bits, s), "radix_sort", radix_sort_launches(k, total_bits));
  GS_LAUNCH(launch_rank(ctx->sval.p, ctx->rank.p, k, s), "k_rank", 1);
  GS_LAUNCH(launch_label_slots(ctx->t0.list.p, root, ctx->rank.p, baseT, ctx->labslot.p, m0, s),
            "k_label_slots", 1);
  GS_LAUNCH(launch_labels(ctx->slot0.p, ctx->labslot.p, labels, n, s), "k_labels", 1);
  if ((int64_t)k <= modes_cap)
    GS_LAUNCH(launch_modes(fin, ctx->rank.p, modes, k, d, s), "k_modes", 1);
  GS_PH_END(GS_PHASE_LABELS);
  GS_CU(cudaMemcpyAsync(hf, ctx->flags.p, sizeof(DevFlags), cudaMemcpyDeviceToHost, s), "D2H flags");
  GS_CU(cudaStreamSynchronize(s), "sync end");
  if (hf->err) return fail(ctx, GS_E_INTERNAL, "an update step hit a device bound");
  ctx->dirty = false;

  if (ctx->timing) {
    for (size_t i = 0; i < ctx->tm.phase.size(); ++i) {
      float ms = 0.f;
      GS_CU(cudaEventElapsedTime(&ms, ctx->tm.pool[2 * i], ctx->tm.pool[2 * i + 1]),
            "cudaEventElapsedTime");
      ctx->last_times.ms[ctx->tm.phase[i]] += ms;
      ctx->last_times.count[ctx->tm.phase[i]] += 1;
    }
  }
  inf.iterations = T;
  inf.converged = converged ? 1 : 0;
  inf.launches = ctx->launches;
  inf.k = k;
  inf.inexact = (int64_t)hf->inexact;
  inf.cell_iters = cell_iters;
  *k_out = k;
  if (info) *info = inf;
  if ((int64_t)k > modes_cap) return fail(ctx, GS_E_CAPACITY, "modes_cap < number of clusters");
  return GS_OK;
}

}  // extern "C"
