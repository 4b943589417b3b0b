// gs_driver.cu -- host-side order of one GridShift run (Sec. 2.1, Algorithm 1):
// key range of the input, the per-call plan (packed keys, exact cell faces,
// fixed-point windows), binning (step i), then one cooperative launch for the
// update steps ii-v, the labels and the modes.  Buffers come from a Workspace.
#include <cmath>
#include <cstring>
#include <vector>

#include "gs_driver.h"
#include "gs_planner.cuh"

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

gs_status fail(std::string* err, gs_status s, const char* msg) {
  if (err) *err = msg;
  return s;
}

gs_status cuda_fail(std::string* err, cudaError_t e, const char* where) {
  if (err) *err = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? GS_E_NOMEM : GS_E_CUDA;
}

// The error of a plan status other than kPlanOK.
gs_status plan_fail(std::string* err, uint32_t st) {
  switch (st) {
    case kPlanNonFinite: return fail(err, GS_E_INVALID, "non-finite input coordinate");
    case kPlanRangeH: return fail(err, GS_E_KEYRANGE, "a coordinate divided by h exceeds 2^52");
    case kPlanSpan: return fail(err, GS_E_KEYRANGE, "more than 2^22 cells along one axis");
    case kPlanBits: return fail(err, GS_E_KEYRANGE, "packed cell key needs more than 63 bits");
    default: return fail(err, GS_E_INTERNAL, "invalid plan");
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
// Bandwidth sweep: the plan of every instance from the key range of the
// shared points, made on the host (one round trip after k_range).  Each
// instance decides floor(x / h_b) against its own faces (SweepPlan); the
// packed-key layout is shared, each axis field as wide as the largest span,
// so the neighbour offsets are too.  The fixed-point units depend only on the
// points and on n0 (every sum of an instance has at most n0 terms), so they
// are shared as well.  Lays out the workspace, uploads the face tables, the
// offsets and the per-instance plans, and clears the loop kernel's start
// state (which the key-range kernel clears in other runs).
static gs_status sweep_prepare(const FitArgs& a, Workspace& ws, Bufs& b, DevFlags* hf,
                               int nprobe, gs_fit_info* info, std::string* err) {
  const int d = a.d, B = a.B;
  const cudaStream_t s = a.stream;
  GS_LAUNCH(launch_range(a.points, a.f32, (int64_t)a.n0, d, b.flags, nullptr, s), "k_range", 1);
  GS_CU(cudaMemcpyAsync(hf, b.flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, s), "D2H flags");
  GS_CU(cudaStreamSynchronize(s), "sync key range");
  if (hf->bad) return plan_fail(err, kPlanNonFinite);
  std::vector<SweepPlan> sp((size_t)B);
  Plan P;
  std::memset(&P, 0, sizeof(P));
  uint64_t thr_words = 0;
  for (int i = 0; i < B; ++i) {
    Plan Pi;
    std::memset(&Pi, 0, sizeof(Pi));
    for (int ax = 0; ax < d; ++ax) {
      const uint32_t st = plan_axis(ax, a.sweep_h[i], (int64_t)a.n0, *hf, Pi);
      if (st != kPlanOK) return plan_fail(err, st);
    }
    SweepPlan& S = sp[(size_t)i];
    std::memset(&S, 0, sizeof(S));
    for (int ax = 0; ax < d; ++ax) {
      S.kmin[ax] = Pi.kmin[ax];
      S.span[ax] = Pi.span[ax];
      S.thr_off[ax] = (int)thr_words;
      thr_words += (uint64_t)Pi.span[ax] + 1;
      if (Pi.span[ax] > P.span[ax]) P.span[ax] = Pi.span[ax];
      P.L[ax] = Pi.L[ax];
    }
    S.inv_h = (float)(1.0 / a.sweep_h[i]);
    if (thr_words >= (1ull << 31))
      return fail(err, GS_E_KEYRANGE, "the sweep's face tables exceed 2^31 entries");
  }
  PlanSizes z;
  const uint32_t st = plan_finish(d, a.sweep_h[0], B, P, z);
  if (st != kPlanOK) return plan_fail(err, st);
  // instance 0's decisions in the shared plan (the sweep's kernels use sp)
  for (int ax = 0; ax < d; ++ax) {
    P.kmin[ax] = sp[0].kmin[ax];
    P.thr_off[ax] = sp[0].thr_off[ax];
  }
  P.inv_h = sp[0].inv_h;
  z.thr_words = thr_words;
  GS_ST(ws.prepare(a.n, d, a.max_iter, thr_words, nprobe, (uint64_t)a.n, s, b, err));
  GS_ST(ws.levels(b.t0_maxcells, d, a.max_iter, s, b, err));
  GS_ST(ws.sweep_space(B, b, err));
  const size_t plan_words = (sizeof(SweepPlan) * (size_t)B + 7) / 8;
  int64_t* stage = nullptr;
  GS_ST(ws.host_words(thr_words + 2 * (size_t)nprobe + plan_words, &stage, err));
  for (int i = 0; i < B; ++i)
    for (int ax = 0; ax < d; ++ax)
      for (int j = 0; j <= sp[(size_t)i].span[ax]; ++j)
        stage[sp[(size_t)i].thr_off[ax] + j] =
            plan_ord_of(plan_face(sp[(size_t)i].kmin[ax] + j, a.sweep_h[i]));
  uint64_t* hd = reinterpret_cast<uint64_t*>(stage + thr_words);
  uint32_t* hv = reinterpret_cast<uint32_t*>(hd + nprobe);
  for (int p = 0; p < nprobe; ++p) plan_probe(P, p, hd + p, hv + p);
  int64_t* hp = stage + thr_words + 2 * (size_t)nprobe;
  std::memcpy(hp, sp.data(), sizeof(SweepPlan) * (size_t)B);
  GS_CU(cudaMemcpyAsync(b.thr, stage, sizeof(int64_t) * thr_words, cudaMemcpyHostToDevice, s),
        "H2D thr");
  GS_CU(cudaMemcpyAsync(b.dtab, hd, sizeof(uint64_t) * 2 * nprobe, cudaMemcpyHostToDevice, s),
        "H2D dtab");
  GS_CU(cudaMemcpyAsync(b.sweep, hp, sizeof(SweepPlan) * (size_t)B, cudaMemcpyHostToDevice, s),
        "H2D sweep plans");
  GS_CU(cudaMemsetAsync(b.filter, 0, sizeof(uint32_t) * 2 * kFilterWords, s), "memset filters");
  GS_CU(cudaMemsetAsync(b.res, 0, sizeof(LoopResult), s), "memset result");
  GS_CU(cudaMemsetAsync(b.st, 0, sizeof(IterState) * (a.max_iter + 2), s), "memset state");
  GS_CU(cudaMemsetAsync(b.bar, 0, sizeof(GridBar), s), "memset barrier");
  hf->plan = P;
  hf->plan_sizes = z;
  hf->plan_status = kPlanOK;
  hf->err = 0;
  hf->m0 = 0;
  GS_CU(cudaMemcpyAsync(b.flags, hf, sizeof(DevFlags), cudaMemcpyHostToDevice, s), "H2D flags");
  return GS_OK;
}

#define GS_T_BEGIN(ph) \
  do { if (timer) GS_CU(timer->begin(ph, s), "cudaEventRecord"); } while (0)
#define GS_T_END() \
  do { if (timer) GS_CU(timer->end(s), "cudaEventRecord"); } while (0)

gs_status fit_pipeline(const FitArgs& a, Workspace& ws, EventTimer* timer, int64_t* k_out,
                       gs_fit_info* info, double* inkernel_ms, std::string* err) {
  const int d = a.d;
  const cudaStream_t s = a.stream;
  const int64_t n = a.n;
  if (a.sequential && (a.mixed || a.B > 1))
    return fail(err, GS_E_INVALID, "the sequential update runs in GS_FP64 on one point set only");
  if (a.sweep_h && (a.mixed || a.sequential || a.B < 2 || a.n0 == 0 ||
                    (int64_t)a.n0 * a.B != a.n))
    return fail(err, GS_E_INVALID, "a bandwidth sweep runs B > 1 instances of n0 points in GS_FP64");
  if (a.img && (a.sweep_h || a.f32 || a.img_feat != a.points || (a.img_xy && !a.img_tab)))
    return fail(err, GS_E_INVALID, "image features are float64 points of one fit");
  Bufs b;
  GS_ST(ws.begin(b, err));

  // a0: key range, fixed-point window, finiteness, then the plan on the
  // device (k_range's last block); the face table gets the workspace's
  // device-side capacity
  DevFlags* hf = ws.host_flags();
  std::memset(hf, 0, sizeof(DevFlags));
  for (int i = 0; i < kMaxD; ++i) {
    hf->min_ord[i] = INT64_MAX;
    hf->max_ord[i] = INT64_MIN;
  }
  GS_CU(cudaMemcpyAsync(b.flags, hf, sizeof(DevFlags), cudaMemcpyHostToDevice, s), "H2D flags");
  const size_t thr_cap = ws.plan_thr_cap();
  int nprobe = 1;
  for (int i = 0; i < d; ++i) nprobe *= 3;
  if (a.sweep_h) {
    GS_ST(sweep_prepare(a, ws, b, hf, nprobe, info, err));
  } else {
    GS_ST(ws.prepare(n, d, a.max_iter, thr_cap, nprobe, (uint64_t)n, s, b, err));
    GS_ST(ws.levels(b.t0_maxcells, d, a.max_iter, s, b, err));
    GS_T_BEGIN(GS_PHASE_RANGE);
    PlanJob job;
    job.h = a.h;
    job.B = a.B;
    job.thr = b.thr;
    job.thr_cap = thr_cap;
    job.dtab = b.dtab;
    job.filters = reinterpret_cast<uint4*>(b.filter);
    job.filter_vec = 2 * kFilterWords / 4;
    job.st = b.st;
    job.n_st = (uint32_t)(a.max_iter + 2);
    job.bar = b.bar;
    job.res = b.res;
    // the key range, then (in its last block) the plan: no host round trip
    // before binning.  An image's features are built first, their key range
    // published from the pixels, and the key-range kernel only plans.
    if (a.img) {
      if (a.img_xy)
        GS_LAUNCH(launch_axis_products(a.img_width, n / a.img_width, a.img_s, a.img_tab, s),
                  "k_axis_products", 1);
      GS_LAUNCH(launch_image_features(a.img, n, a.img_width, a.img_C, a.img_xy, a.img_tab,
                                      a.img_feat, b.flags, s), "k_image_features", 1);
    }
    GS_LAUNCH(launch_range(a.points, a.f32, n, d, b.flags, &job, s, a.img == nullptr), "k_range",
              1);
    GS_T_END();
  }
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
  // start and both run again with a larger table; if the face table did not
  // fit the device-side capacity, neither ran, and the host makes the plan
  // and runs them again.
  ws.mark_dirty(true);
  const int grid = a.sequential ? loop_grid_seq(d) : loop_grid(d, a.mixed);
  if (grid <= 0) return fail(err, GS_E_CUDA, "no co-resident grid for the loop kernel");
  LoopArgs L;
  LoopResult* hr = ws.host_result();
  bool host_planned = false;
  for (int attempt = 0;; ++attempt) {
    if (attempt > 0) {
      // a second binning (larger table, or the host's plan): the level
      // workspace for its cell bound, and the start state the key-range
      // kernel cleared
      GS_ST(ws.levels(b.t0_maxcells, d, a.max_iter, s, b, err));
      GS_CU(cudaMemsetAsync(b.filter, 0, sizeof(uint32_t) * 2 * kFilterWords, s),
            "memset filters");
      GS_CU(cudaMemsetAsync(b.res, 0, sizeof(LoopResult), s), "memset result");
      GS_CU(cudaMemsetAsync(b.st, 0, sizeof(IterState) * (a.max_iter + 2), s), "memset state");
      GS_CU(cudaMemsetAsync(b.bar, 0, sizeof(GridBar), s), "memset barrier");
    }
    if (a.sequential) GS_ST(ws.shift_rows(b.capAB, d, b, err));
    std::memset(&L, 0, sizeof(L));
    L.P.d = d;  // the loop kernel reads the plan from b.flags
    L.pts = a.points;
    L.f32 = a.f32;
    L.perm = b.perm;
    L.blocksum = b.blocksum;
    L.thr = b.thr;
    L.dtab = b.dtab;
    L.vpack = reinterpret_cast<const uint32_t*>(b.dtab + nprobe);
    L.T0 = b.t0;
    for (int i = 0; i < 3; ++i) L.tab[i] = b.tab[i];
    L.capAB = b.capAB;
    L.cells[0] = b.cells[0];
    L.cells[1] = b.cells[1];
    L.pslot[0] = b.pslot[0];
    L.pslot[1] = b.pslot[1];
    L.filter[0] = b.filter;
    L.filter[1] = b.filter + kFilterWords;
    L.qlist = b.qlist;
    L.ptab = b.ptab;
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
    L.srow = a.sequential ? b.srow : nullptr;
    L.seq_aux = a.sequential ? b.seq_aux : nullptr;
    L.sweep = a.sweep_h ? b.sweep : nullptr;
    L.tune = a.tune;
    L.n0 = a.sweep_h ? a.n0 : 0;
    if (a.B > 1) L.I = inst_views(b.inst, a.B);
    GS_T_BEGIN(GS_PHASE_BIN);
    GS_LAUNCH(launch_bin(a.points, a.f32, n, d, b.thr, b.t0, b.t0.cap - 1, b.t0_maxcells,
                         b.slot0, b.flags, b.offsets, a.B, L.sweep, L.n0,
                         a.tune.bin_list != 0, a.tune.bin_sums != 0, s), "k_bin", 1);
    GS_T_END();
    // step i, second pass (unless binning formed the sums): the exact cell
    // sums through a counting sort (as launches of their own for large runs,
    // else inside the loop kernel)
    const bool split = n >= (int64_t)a.tune.split_min;
    if (split && !a.tune.bin_sums) {
      GS_T_BEGIN(GS_PHASE_K_OFFSETS);
      GS_LAUNCH(launch_prep_offsets(L, s), "k_prep_offsets", kPrepOffsetsLaunches);
      GS_T_END();
      GS_T_BEGIN(GS_PHASE_K_SCATTER);
      GS_LAUNCH(launch_prep_scatter(L, s), "k_prep_scatter", 1);
      GS_T_END();
      GS_T_BEGIN(GS_PHASE_K_SUMS);
      GS_LAUNCH(launch_prep_sums(L, s), "k_prep_sums", 1);
      GS_T_END();
    }
    GS_T_BEGIN(GS_PHASE_LOOP);
    GS_LAUNCH(a.sequential ? launch_loop_seq(L, grid, s) : launch_loop(L, grid, s), "k_loop", 1);
    GS_T_END();
    if (split) {
      GS_T_BEGIN(GS_PHASE_LABELS_OUT);
      GS_LAUNCH(launch_labels_out(L, s), "k_labels_out", 1);
      GS_T_END();
    }
    GS_CU(cudaMemcpyAsync(hr, b.res, sizeof(LoopResult), cudaMemcpyDeviceToHost, s), "D2H result");
    GS_CU(cudaMemcpyAsync(hf, b.flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, s), "D2H flags");
    GS_CU(cudaStreamSynchronize(s), "sync loop");
    if (hf->plan_status != kPlanOK) {
      if (hf->plan_status != kPlanTable || host_planned) {
        if (a.plan_status_out) *a.plan_status_out = hf->plan_status;
        return plan_fail(err, hf->plan_status);
      }
      // the face table is larger than the device-side capacity: the plan,
      // face table and offsets from the host, then binning and the loop
      Plan P;
      PlanSizes z;
      const uint32_t st = plan_from_range(d, a.h, n, a.B, *hf, P, z);
      if (st != kPlanOK) {
        if (a.plan_status_out) *a.plan_status_out = st;
        return plan_fail(err, st);
      }
      const uint64_t m_bound = (uint64_t)n < z.span_prod ? (uint64_t)n : z.span_prod;
      GS_ST(ws.prepare(n, d, a.max_iter, z.thr_words, nprobe, m_bound, s, b, err));
      int64_t* stage = nullptr;
      GS_ST(ws.host_words(z.thr_words + 2 * (size_t)nprobe, &stage, err));
      for (uint64_t j = 0; j < z.thr_words; ++j) stage[j] = plan_face_entry(P, a.h, j);
      uint64_t* hd = reinterpret_cast<uint64_t*>(stage + z.thr_words);
      uint32_t* hv = reinterpret_cast<uint32_t*>(hd + nprobe);
      for (int p = 0; p < nprobe; ++p) plan_probe(P, p, hd + p, hv + p);
      GS_CU(cudaMemcpyAsync(b.thr, stage, sizeof(int64_t) * z.thr_words, cudaMemcpyHostToDevice,
                            s), "H2D thr");
      GS_CU(cudaMemcpyAsync(b.dtab, hd, sizeof(uint64_t) * 2 * nprobe, cudaMemcpyHostToDevice, s),
            "H2D dtab");
      hf->plan = P;
      hf->plan_sizes = z;
      hf->plan_status = kPlanOK;
      hf->err = 0;
      hf->m0 = 0;
      GS_CU(cudaMemcpyAsync(b.flags, hf, sizeof(DevFlags), cudaMemcpyHostToDevice, s), "H2D flags");
      host_planned = true;
      continue;
    }
    const uint32_t regrow = kErrOverflow | kErrTableFull;
    if (!(hf->err & regrow) || !hr->bin_failed) break;
    if (attempt >= 4) return fail(err, GS_E_INTERNAL, "binning table overflow");
    GS_ST(ws.regrow_bin(d, s, b, err));
    hf->err = 0;
    hf->m0 = 0;
    GS_CU(cudaMemcpyAsync(b.flags, hf, sizeof(DevFlags), cudaMemcpyHostToDevice, s), "H2D flags");
  }
  // the plan the kernels ran with, for the kernels after the loop
  L.P = hf->plan;
  const int total_bits = hf->plan_sizes.total_bits;
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
