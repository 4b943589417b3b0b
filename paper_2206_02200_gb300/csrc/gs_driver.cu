// gs_driver.cu -- host-side order of one GridShift run (Sec. 2.1, Algorithm 1):
// key range of the input, the per-call plan (packed keys, exact cell faces,
// fixed-point windows), binning (step i), then one cooperative launch for the
// update steps ii-v, the labels and the modes.  Buffers come from a Workspace.
#include <cmath>
#include <cstring>

#include "gs_driver.h"

namespace gs {

InstState inst_views(uint32_t* base, int B) {
  InstState I;
  const size_t b = (size_t)B;
  I.cell_iters = reinterpret_cast<unsigned long long*>(base);  // first: 8-byte aligned
  uint32_t* p = base + 2 * b;
  I.done[0] = p; p += b;
  I.done[1] = p; p += b;
  I.nbf[0] = p; p += b;
  I.nbf[1] = p; p += b;
  I.mt[0] = p; p += b;
  I.mt[1] = p; p += b;
  I.iters = reinterpret_cast<int32_t*>(p); p += b;
  I.conv = reinterpret_cast<int32_t*>(p); p += b;
  I.m0 = p; p += b;
  I.k = p; p += b;
  I.koff = p;
  return I;
}

uint32_t pow2_at_least(uint64_t v, uint32_t lo) {
  uint64_t c = lo;
  while (c < v && c < (1ull << 31)) c <<= 1;
  return (uint32_t)c;
}

namespace {

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
  for (; v; v >>= 1) ++b;
  return b;
}

gs_status fail(std::string* err, gs_status s, const char* msg) {
  if (err) *err = msg;
  return s;
}

gs_status cuda_fail(std::string* err, cudaError_t e, const char* where) {
  if (err) *err = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? GS_E_NOMEM : GS_E_CUDA;
}

// Packed-key layout and fixed-point windows from the key range (Sec. 2.1 i):
// per axis the data's key box widened by one cell each side (centroids are
// convex combinations of the points, Eq. 1 and Eq. 3, and leave that box by a
// few roundings at most), packed axis 0 most significant.
gs_status make_plan(int d, double h, int64_t n, int B, const DevFlags& fl, Plan& P,
                    size_t& thr_words, uint64_t& span_prod, int& total_bits, std::string* err) {
  std::memset(&P, 0, sizeof(P));
  P.d = d;
  P.inv_h = (float)(1.0 / h);
  P.h32 = (float)h;
  int bits[kMaxD];
  int clog2n = 0;
  while ((1ll << clog2n) < n) ++clog2n;
  span_prod = 1;
  thr_words = 0;
  for (int a = 0; a < d; ++a) {
    const double lo = from_ord(fl.min_ord[a]), hi = from_ord(fl.max_ord[a]);
    if (!(std::fabs(lo / h) < 4.0e15) || !(std::fabs(hi / h) < 4.0e15))
      return fail(err, GS_E_KEYRANGE, "a coordinate divided by h exceeds 2^52");
    const int64_t kmin = floor_div(lo, h) - 1, kmax = floor_div(hi, h) + 1;
    const int64_t span = kmax - kmin + 1;
    if (span > (1ll << 22)) return fail(err, GS_E_KEYRANGE, "more than 2^22 cells along one axis");
    P.kmin[a] = kmin;
    P.span[a] = (int)span;
    bits[a] = bitlen((uint64_t)span + 1);
    P.thr_off[a] = (int)thr_words;
    thr_words += (size_t)span + 1;
    span_prod = span_prod > (1ull << 40) ? span_prod : span_prod * (uint64_t)span;
    double ma;
    const uint64_t mb = fl.maxabs[a];
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
  // batched runs: the instance index in the field above all axes (it is
  // never probed, so cells of different instances never meet)
  P.inst_off = total_bits;
  if (B > 1) total_bits += bitlen((uint64_t)(B - 1));
  if (total_bits > 63) return fail(err, GS_E_KEYRANGE, "packed cell key needs more than 63 bits");
  int np = 1;
  for (int a = 0; a < d; ++a) np *= 3;
  P.nprobe = np;
  P.center = (np - 1) / 2;
  return GS_OK;
}

// Face tables (order codes of the least doubles >= q h) and the packed-key
// offsets of the 3^d neighbours v in {-1,0,1}^d (axis 0 the slowest digit).
void fill_tables(const Plan& P, double h, int64_t* thr, uint64_t* dtab, uint32_t* vpack) {
  for (int a = 0; a < P.d; ++a)
    for (int64_t j = 0; j <= P.span[a]; ++j) thr[P.thr_off[a] + j] = ord_of(face(P.kmin[a] + j, h));
  for (int p = 0; p < P.nprobe; ++p) {
    int64_t delta = 0;
    uint32_t vp = 0;
    int rest = p;
    for (int a = P.d - 1; a >= 0; --a) {
      const int v = rest % 3 - 1;
      rest /= 3;
      delta += (int64_t)v * (int64_t)(1ull << P.off[a]);
      vp |= (uint32_t)(v + 1) << (2 * a);
    }
    dtab[p] = (uint64_t)delta;
    vpack[p] = vp;
  }
}

}  // namespace

#define GS_CU(call, where)                                     \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail(err, e_, where);   \
  } while (0)
#define GS_ST(call)                     \
  do {                                  \
    gs_status s_ = (call);              \
    if (s_ != GS_OK) return s_;         \
  } while (0)
#define GS_LAUNCH(call, where, nk)      \
  do {                                  \
    GS_CU(call, where);                 \
    info->launches += (nk);             \
  } while (0)
#define GS_T_BEGIN(ph) \
  do { if (timer) GS_CU(timer->begin(ph, s), "cudaEventRecord"); } while (0)
#define GS_T_END() \
  do { if (timer) GS_CU(timer->end(s), "cudaEventRecord"); } while (0)

gs_status fit_pipeline(const FitArgs& a, Workspace& ws, EventTimer* timer, int64_t* k_out,
                       gs_fit_info* info, double* inkernel_ms, std::string* err) {
  const int d = a.d;
  const cudaStream_t s = a.stream;
  const int64_t n = a.n;
  Bufs b;
  GS_ST(ws.begin(b, err));

  // a0: key range, fixed-point window, finiteness
  DevFlags* hf = ws.host_flags();
  std::memset(hf, 0, sizeof(DevFlags));
  for (int i = 0; i < kMaxD; ++i) {
    hf->min_ord[i] = INT64_MAX;
    hf->max_ord[i] = INT64_MIN;
  }
  GS_CU(cudaMemcpyAsync(b.flags, hf, sizeof(DevFlags), cudaMemcpyHostToDevice, s), "H2D flags");
  GS_T_BEGIN(GS_PHASE_RANGE);
  GS_LAUNCH(launch_range(a.points, a.f32, n, d, b.flags, s), "k_range", 1);
  GS_T_END();
  GS_CU(cudaMemcpyAsync(hf, b.flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, s), "D2H flags");
  GS_CU(cudaStreamSynchronize(s), "sync range");
  if (hf->bad) return fail(err, GS_E_INVALID, "non-finite input coordinate");

  Plan P;
  size_t thr_words = 0;
  uint64_t span_prod = 0;
  int total_bits = 0;
  GS_ST(make_plan(d, a.h, n, a.B, *hf, P, thr_words, span_prod, total_bits, err));
  const uint64_t m_bound = (uint64_t)n < span_prod ? (uint64_t)n : span_prod;
  GS_ST(ws.prepare(n, d, a.max_iter, thr_words, P.nprobe, m_bound, s, b, err));

  // face table and neighbour offsets, through host staging
  // (dtab holds nprobe offsets, then nprobe 32-bit packed offset vectors)
  int64_t* stage = nullptr;
  GS_ST(ws.host_words(thr_words + 2 * P.nprobe, &stage, err));
  fill_tables(P, a.h, stage, reinterpret_cast<uint64_t*>(stage + thr_words),
              reinterpret_cast<uint32_t*>(stage + thr_words + P.nprobe));
  GS_CU(cudaMemcpyAsync(b.thr, stage, sizeof(int64_t) * thr_words, cudaMemcpyHostToDevice, s),
        "H2D thr");
  GS_CU(cudaMemcpyAsync(b.dtab, stage + thr_words, sizeof(uint64_t) * 2 * P.nprobe,
                        cudaMemcpyHostToDevice, s), "H2D dtab");
  GS_CU(cudaMemsetAsync(b.st, 0, sizeof(IterState) * (a.max_iter + 2), s), "memset state");
  GS_CU(cudaMemsetAsync(b.bar, 0, sizeof(GridBar), s), "memset barrier");
  uint32_t* hinst = nullptr;
  if (a.B > 1) {
    // batched: instance offsets, cleared per-instance state
    GS_ST(ws.batch_space(a.B, b, &hinst, err));
    GS_CU(cudaMemcpyAsync(b.offsets, a.offsets, sizeof(int64_t) * (a.B + 1),
                          cudaMemcpyHostToDevice, s), "H2D offsets");
    GS_CU(cudaMemsetAsync(b.inst, 0, sizeof(uint32_t) * inst_words(a.B), s), "memset instances");
  }

  // i: binning, then at once the loop kernel: the level workspace is sized
  // for the binning table's cell bound, so no host round trip separates
  // them.  If binning overflows the table, the loop kernel returns at its
  // start and both run again with a larger table.
  ws.mark_dirty(true);
  const int grid = loop_grid(d, a.mixed);
  if (grid <= 0) return fail(err, GS_E_CUDA, "no co-resident grid for the loop kernel");
  LoopArgs L;
  LoopResult* hr = ws.host_result();
  for (int attempt = 0;; ++attempt) {
    GS_ST(ws.levels(b.t0_maxcells, d, a.max_iter, s, b, err));
    std::memset(&L, 0, sizeof(L));
    L.P = P;
    L.pts = a.points;
    L.f32 = a.f32;
    L.perm = b.perm;
    L.blocksum = b.blocksum;
    L.thr = b.thr;
    L.dtab = b.dtab;
    L.vpack = reinterpret_cast<const uint32_t*>(b.dtab + P.nprobe);
    L.T0 = b.t0;
    for (int i = 0; i < 3; ++i) L.tab[i] = b.tab[i];
    L.capAB = b.capAB;
    L.cells[0] = b.cells[0];
    L.cells[1] = b.cells[1];
    L.pslot[0] = b.pslot[0];
    L.pslot[1] = b.pslot[1];
    L.filter[0] = b.filter;
    L.filter[1] = b.filter + kFilterWords;
    L.forest = b.forest;
    L.forest2 = b.forest2;
    L.labslot = b.labslot;
    L.rank = b.rank;
    L.slot0 = b.slot0;
    L.labels = a.labels;
    L.n = n;
    L.modes = a.modes;
    L.modes_cap = a.modes_cap;
    L.st = b.st;
    L.fl = b.flags;
    L.bar = b.bar;
    L.res = b.res;
    L.max_iter = a.max_iter;
    L.rank_max = kRankMax;
    L.B = a.B;
    L.mixed = a.mixed;
    if (a.B > 1) L.I = inst_views(b.inst, a.B);
    GS_CU(cudaMemsetAsync(b.filter, 0, sizeof(uint32_t) * 2 * kFilterWords, s), "memset filters");
    GS_CU(cudaMemsetAsync(b.res, 0, sizeof(LoopResult), s), "memset result");
    GS_T_BEGIN(GS_PHASE_BIN);
    GS_LAUNCH(launch_bin(a.points, a.f32, n, P, b.thr, b.t0, b.t0.cap - 1, b.t0_maxcells, b.slot0,
                         b.flags, b.offsets, a.B, s), "k_bin", 1);
    GS_T_END();
    GS_T_BEGIN(GS_PHASE_LOOP);
    GS_LAUNCH(launch_loop(L, grid, s), "k_loop", 1);
    GS_T_END();
    GS_CU(cudaMemcpyAsync(hr, b.res, sizeof(LoopResult), cudaMemcpyDeviceToHost, s), "D2H result");
    GS_CU(cudaMemcpyAsync(hf, b.flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, s), "D2H flags");
    GS_CU(cudaStreamSynchronize(s), "sync loop");
    const uint32_t regrow = kErrOverflow | kErrTableFull;
    if (!(hf->err & regrow) || !hr->bin_failed) break;
    if (attempt >= 4) return fail(err, GS_E_INTERNAL, "binning table overflow");
    GS_ST(ws.regrow_bin(d, s, b, err));
    hf->err = 0;
    hf->m0 = 0;
    GS_CU(cudaMemcpyAsync(b.flags, hf, sizeof(DevFlags), cudaMemcpyHostToDevice, s), "H2D flags");
  }
  const uint32_t m0 = hf->m0;
  info->m0 = m0;
  ws.note_cells(m0);
  if (hf->err & kErrBarrier) return fail(err, GS_E_INTERNAL, "a grid barrier of the loop timed out");
  if (hf->err) return fail(err, GS_E_INTERNAL, "an update step hit a device bound");
  const uint32_t k = hr->k;
  const int T = hr->iterations;

  if (hr->need_sort) {
    // number the final cells by a radix sort of their keys
    GS_ST(ws.sort_space(k, b, err));
    const Cells fin = b.cells[T & 1];
    GS_T_BEGIN(GS_PHASE_SORT);
    GS_LAUNCH(launch_iota_keys(fin, b.skey, b.sval, k, s), "k_iota_keys", 1);
    GS_LAUNCH(radix_sort(b.skey, b.sval, b.skey2, b.sval2, b.shist, k, total_bits, s),
              "radix_sort", radix_sort_launches(k, total_bits));
    GS_LAUNCH(launch_rank(b.sval, b.rank, k, s), "k_rank", 1);
    GS_LAUNCH(launch_label_tail(L, m0, k, hr->base, T, s), "label tail", kLabelTailLaunches);
    GS_T_END();
  }
  if (a.B > 1)
    GS_CU(cudaMemcpyAsync(hinst, b.inst, sizeof(uint32_t) * inst_words(a.B),
                          cudaMemcpyDeviceToHost, s), "D2H instances");
  if (hr->need_sort || a.B > 1) GS_CU(cudaStreamSynchronize(s), "sync labels");
  ws.mark_dirty(false);

  info->iterations = T;
  info->converged = hr->converged;
  info->k = k;
  info->inexact = (int64_t)hf->inexact;
  info->face_rechecks = (int64_t)hf->rechecks;
  info->cell_iters = (int64_t)hr->cell_iters;
  if (inkernel_ms) {
    for (int i = 0; i < kLoopPhases; ++i) inkernel_ms[i] = (double)hr->ns[i] * 1e-6;
    for (int i = 0; i < kClockSteps; ++i)
      for (int c = 0; c < 2; ++c)
        inkernel_ms[kLoopPhases + 2 * i + c] = i < T ? (double)hr->step_ns[i][c] * 1e-6 : 0.0;
  }
  *k_out = k;
  if (a.B > 1) {
    // per-instance results (the host copy of InstState, same layout)
    const InstState H = inst_views(hinst, a.B);
    int64_t run = 0;
    for (int i = 0; i < a.B; ++i) {
      gs_fit_info& fi = a.infos[i];
      std::memset(&fi, 0, sizeof(fi));
      fi.iterations = H.iters[i];
      fi.converged = H.conv[i];
      fi.m0 = H.m0[i];
      fi.k = H.k[i];
      fi.inexact = info->inexact;
      fi.cell_iters = (int64_t)H.cell_iters[i];
      fi.launches = info->launches;
      fi.face_rechecks = info->face_rechecks;
      a.mode_offsets[i] = run;
      run += H.k[i];
    }
    a.mode_offsets[a.B] = run;
  }
  if ((int64_t)k > a.modes_cap) return fail(err, GS_E_CAPACITY, "modes_cap < number of clusters");
  return GS_OK;
}

}  // namespace gs
