// gs_noalloc.cu -- gs_fit_noalloc: the GridShift pipeline of gs_fit with every
// piece of device scratch carved out of one file-scope static device array, for
// callers that must not allocate device or pinned memory (see the declaration
// in include/gridshift.h).  The kernels are the ones gs_fit launches.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/gridshift.h"
#include "gs_kernels.h"

using namespace gs;

namespace {

// The static scratch.  Every GPU that loads this library holds it until the
// process exits.  Host code must not use the symbol itself as a device
// address: the address is obtained once per device with cudaGetSymbolAddress.
constexpr size_t kScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
constexpr int kThrMax = 8192;  // face-table entries (sum over axes of span + 1)
constexpr int kProbeMax = 6561;  // 3^8 neighbour offsets

std::mutex g_mu;  // serialises calls: they share g_scratch and the host buffers below
unsigned char* g_dev_ptr[kMaxDevices] = {};
int64_t g_thr[kThrMax];
uint64_t g_dtab[kProbeMax];

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

// Least double >= q * h: the rounding error of q * h is exact under one fma.
double face(int64_t q, double h) {
  double qd = (double)q;
  double p = qd * h;
  if (std::fma(qd, h, -p) > 0) p = std::nextafter(p, INFINITY);
  return p;
}

int64_t floor_div(double x, double h) {
  int64_t q = (int64_t)std::floor(x / h);
  for (int i = 0; i < 4 && face(q, h) > x; ++i) --q;
  for (int i = 0; i < 4 && face(q + 1, h) <= x; ++i) ++q;
  return q;
}

int bitlen(uint64_t v) {
  int b = 0;
  for (; v; v >>= 1) ++b;
  return b;
}

// Bump allocator over the static scratch (256-byte aligned pieces).
struct Carve {
  unsigned char* base;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    return reinterpret_cast<T*>(base + off);
  }
};

// Views of every workspace array of one call, for at most M cells (lookup
// tables of 2M slots) and n points.
struct Work {
  DevFlags* flags;
  IterState* st;
  int64_t* thr;
  uint64_t* dtab;
  uint32_t* slot0;
  Table t0, tab[2];
  Cells cells[2];
  double* sp;
  uint64_t* nkey;
  uint32_t *pslot, *forest, *forest2, *labslot, *rank;
  uint64_t *skey, *skey2;
  uint32_t *sval, *sval2, *shist;
};

Table carve_table(Carve& c, uint32_t cap, uint32_t lmax, int d) {
  Table t;
  t.key = c.take<uint64_t>(cap);
  t.id = c.take<uint32_t>(cap);
  t.cnt = c.take<uint32_t>(cap);
  t.acc = c.take<uint64_t>((size_t)cap * d * 4);
  t.list = c.take<uint32_t>(lmax);
  t.cap = cap;
  return t;
}

size_t layout(unsigned char* base, int64_t n, int d, int max_iter, uint32_t M, int thr_words,
              int nprobe, Work* w) {
  Carve c{base};
  Work tmp;
  Work& W = w ? *w : tmp;
  const uint32_t cap = 2 * M;
  W.flags = c.take<DevFlags>(1);
  W.st = c.take<IterState>(max_iter + 2);
  W.thr = c.take<int64_t>(thr_words);
  W.dtab = c.take<uint64_t>(nprobe);
  W.slot0 = c.take<uint32_t>(n);
  W.t0 = carve_table(c, cap, M, d);
  W.tab[0] = carve_table(c, cap, M, d);
  W.tab[1] = carve_table(c, cap, M, d);
  for (int b = 0; b < 2; ++b) {
    W.cells[b].key = c.take<uint64_t>(M);
    W.cells[b].cnt = c.take<uint32_t>(M);
    W.cells[b].cs = c.take<double>((size_t)M * d);
  }
  W.sp = c.take<double>((size_t)M * d);
  W.nkey = c.take<uint64_t>(M);
  W.pslot = c.take<uint32_t>(M);
  W.forest = c.take<uint32_t>((size_t)M * (max_iter + 1));
  W.forest2 = c.take<uint32_t>((size_t)M * (max_iter + 1));
  W.labslot = c.take<uint32_t>(cap);
  W.rank = c.take<uint32_t>(M);
  W.skey = c.take<uint64_t>(M);
  W.skey2 = c.take<uint64_t>(M);
  W.sval = c.take<uint32_t>(M);
  W.sval2 = c.take<uint32_t>(M);
  W.shist = c.take<uint32_t>(radix_hist_words(M));
  return c.used;
}

cudaError_t clear_table(const Table& t, int d, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(t.key, 0xFF, sizeof(uint64_t) * t.cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.cnt, 0, sizeof(uint32_t) * t.cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.acc, 0, sizeof(uint64_t) * t.cap * d * 4, s);
  return e;
}

gs_status run(int d, double h, int max_iter, cudaStream_t s, const void* points, bool f32,
              int64_t n, int32_t* labels, double* modes, int64_t modes_cap, int64_t* k_out,
              gs_fit_info* inf, unsigned char* base) {
#define NA_CU(call)                                                           \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return e_ == cudaErrorMemoryAllocation ? GS_E_NOMEM : GS_E_CUDA;        \
  } while (0)
#define NA_LAUNCH(call, nk) \
  do {                      \
    NA_CU(call);            \
    inf->launches += (nk);  \
  } while (0)

  // a0: key range, fixed-point window, finiteness (the flags live at the
  // start of the scratch; their host copy is plain stack memory)
  DevFlags hf;
  std::memset(&hf, 0, sizeof(hf));
  for (int a = 0; a < kMaxD; ++a) {
    hf.min_ord[a] = INT64_MAX;
    hf.max_ord[a] = INT64_MIN;
  }
  DevFlags* dflags = reinterpret_cast<DevFlags*>(base);
  NA_CU(cudaMemcpyAsync(dflags, &hf, sizeof(hf), cudaMemcpyHostToDevice, s));
  NA_LAUNCH(launch_range(points, f32, n, d, dflags, s), 1);
  NA_CU(cudaMemcpyAsync(&hf, dflags, sizeof(hf), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaStreamSynchronize(s));
  if (hf.bad) return GS_E_INVALID;

  // plan: packed keys, face table, fixed-point windows
  Plan P;
  std::memset(&P, 0, sizeof(P));
  P.d = d;
  int bits[kMaxD];
  int clog2n = 0;
  while ((1ll << clog2n) < n) ++clog2n;
  uint64_t span_prod = 1;
  int thr_words = 0;
  for (int a = 0; a < d; ++a) {
    double lo = from_ord(hf.min_ord[a]), hi = from_ord(hf.max_ord[a]);
    if (!(std::fabs(lo / h) < 4.0e15) || !(std::fabs(hi / h) < 4.0e15)) return GS_E_KEYRANGE;
    int64_t kmin = floor_div(lo, h) - 1, kmax = floor_div(hi, h) + 1;
    int64_t span = kmax - kmin + 1;
    if (span > (1ll << 22)) return GS_E_KEYRANGE;
    if (thr_words + span + 1 > kThrMax) return GS_E_SCRATCH;
    P.kmin[a] = kmin;
    P.span[a] = (int)span;
    bits[a] = bitlen((uint64_t)span + 1);
    P.thr_off[a] = thr_words;
    for (int64_t j = 0; j <= span; ++j) g_thr[thr_words++] = ord_of(face(kmin + j, h));
    span_prod = span_prod > (1ull << 40) ? span_prod : span_prod * (uint64_t)span;
    double ma;
    uint64_t mb = hf.maxabs[a];
    std::memcpy(&ma, &mb, 8);
    int e = 0;
    if (ma > 0) std::frexp(ma, &e);
    P.L[a] = e + clog2n - 126;
  }
  int total_bits = 0;
  for (int a = d - 1; a >= 0; --a) {
    P.off[a] = total_bits;
    total_bits += bits[a];
  }
  if (total_bits > 63) return GS_E_KEYRANGE;
  int np = 1;
  for (int a = 0; a < d; ++a) np *= 3;
  P.nprobe = np;
  P.center = (np - 1) / 2;
  for (int p = 0; p < np; ++p) {
    int64_t delta = 0;
    int rest = p;
    for (int a = d - 1; a >= 0; --a) {
      int v = rest % 3 - 1;
      rest /= 3;
      delta += (int64_t)v * (int64_t)(1ull << P.off[a]);
    }
    g_dtab[p] = (uint64_t)delta;
  }

  // the largest cell bound M (a power of two) whose workspace fits the scratch
  uint64_t want = (uint64_t)n < span_prod ? (uint64_t)n : span_prod;
  uint32_t M = 64;
  while (M < want && M < (1u << 30)) M <<= 1;
  while (M > 64 && layout(nullptr, n, d, max_iter, M, thr_words, np, nullptr) > kScratchBytes)
    M >>= 1;
  if (layout(nullptr, n, d, max_iter, M, thr_words, np, nullptr) > kScratchBytes)
    return GS_E_SCRATCH;
  Work W;
  layout(base, n, d, max_iter, M, thr_words, np, &W);

  // clear what must start at zero: the scratch keeps the previous call's contents
  NA_CU(cudaMemcpyAsync(W.thr, g_thr, sizeof(int64_t) * thr_words, cudaMemcpyHostToDevice, s));
  NA_CU(cudaMemcpyAsync(W.dtab, g_dtab, sizeof(uint64_t) * np, cudaMemcpyHostToDevice, s));
  NA_CU(cudaMemsetAsync(W.st, 0, sizeof(IterState) * (max_iter + 2), s));
  NA_CU(clear_table(W.t0, d, s));
  NA_CU(clear_table(W.tab[0], d, s));
  NA_CU(clear_table(W.tab[1], d, s));
  hf.err = 0;
  hf.m0 = 0;
  NA_CU(cudaMemcpyAsync(W.flags, &hf, sizeof(hf), cudaMemcpyHostToDevice, s));

  // i: binning (at most M cells fit)
  NA_LAUNCH(launch_bin(points, f32, n, P, W.thr, W.t0, 2 * M - 1, M, W.slot0, W.flags, s), 1);
  NA_CU(cudaMemcpyAsync(&hf, W.flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaStreamSynchronize(s));
  if (hf.err & (kErrOverflow | kErrTableFull)) return GS_E_SCRATCH;
  if (hf.err) return GS_E_INTERNAL;
  const uint32_t m0 = hf.m0;
  inf->m0 = m0;
  NA_LAUNCH(launch_compact0(P, W.t0, W.cells[0], W.tab[0], 2 * M, m0, W.st, W.flags, s), 1);

  // ii-v: update steps
  IterState hs;
  int t = 0;
  uint32_t m_t = m0;
  bool converged = false;
  for (;;) {
    Table G = W.tab[t & 1], Mt = W.tab[(t + 1) & 1];
    Cells c = W.cells[t & 1], nx = W.cells[(t + 1) & 1];
    NA_LAUNCH(launch_gather(P, W.thr, W.dtab, G, c, W.sp, W.nkey, W.st, t, m_t, W.flags, s), 1);
    NA_CU(cudaMemcpyAsync(&hs, W.st + t, sizeof(hs), cudaMemcpyDeviceToHost, s));
    NA_CU(cudaStreamSynchronize(s));
    m_t = hs.m;
    if (!hs.has_nb) {
      converged = true;
      break;
    }
    if (t == max_iter) break;
    NA_LAUNCH(launch_merge(P, c, W.sp, W.nkey, Mt, W.pslot, W.st, t, m_t, W.flags, s), 1);
    NA_LAUNCH(launch_compact(P, Mt, nx, W.st, t, m_t, W.flags, s), 1);
    NA_LAUNCH(launch_finish(G, Mt, W.pslot, W.forest, W.st, t, m_t, s), 1);
    inf->cell_iters += m_t;
    ++t;
  }
  const int T = t;
  NA_LAUNCH(launch_final_level(W.tab[T & 1], W.forest, W.st, T, m_t, s), 1);
  NA_CU(cudaMemcpyAsync(&hs, W.st + T, sizeof(hs), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaStreamSynchronize(s));
  const uint32_t k = hs.m, baseT = hs.base, nodes = baseT + k;

  // labels and modes
  uint32_t* root = W.forest;
  uint32_t* other = W.forest2;
  for (int hop = 1; hop < T; hop <<= 1) {
    NA_LAUNCH(launch_jump(root, other, nodes, s), 1);
    uint32_t* tmp = root;
    root = other;
    other = tmp;
  }
  Cells fin = W.cells[T & 1];
  NA_LAUNCH(launch_iota_keys(fin, W.skey, W.sval, k, s), 1);
  NA_LAUNCH(radix_sort(W.skey, W.sval, W.skey2, W.sval2, W.shist, k, total_bits, s),
            radix_sort_launches(k, total_bits));
  NA_LAUNCH(launch_rank(W.sval, W.rank, k, s), 1);
  NA_LAUNCH(launch_label_slots(W.t0.list, root, W.rank, baseT, W.labslot, m0, s), 1);
  NA_LAUNCH(launch_labels(W.slot0, W.labslot, labels, n, s), 1);
  if ((int64_t)k <= modes_cap) NA_LAUNCH(launch_modes(fin, W.rank, modes, k, d, s), 1);
  NA_CU(cudaMemcpyAsync(&hf, W.flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
  NA_CU(cudaStreamSynchronize(s));
  if (hf.err) return GS_E_INTERNAL;
  inf->iterations = T;
  inf->converged = converged ? 1 : 0;
  inf->k = k;
  inf->inexact = (int64_t)hf.inexact;
  *k_out = k;
  if ((int64_t)k > modes_cap) return GS_E_CAPACITY;
  return GS_OK;
#undef NA_CU
#undef NA_LAUNCH
}

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
  // the per-point slot array alone must fit
  if ((size_t)n * sizeof(uint32_t) + (size_t(1) << 20) > kScratchBytes) return GS_E_SCRATCH;

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GS_E_CUDA;
  if (!g_dev_ptr[dev]) {
    // set-up on this device, once: the device address of the static scratch
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return GS_E_CUDA;
    g_dev_ptr[dev] = static_cast<unsigned char*>(p);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  gs_status st = run(d, h, max_iter, s, points, dtype == GS_IN_F32, n, labels, modes, modes_cap,
                     k_out, &inf, g_dev_ptr[dev]);
  // no work of this call may still run when the next one reuses the scratch
  if (st != GS_OK) cudaStreamSynchronize(s);
  if (info) *info = inf;
  return st;
}
