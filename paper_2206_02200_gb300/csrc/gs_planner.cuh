// gs_planner.cuh -- the per-call plan (Sec. 2.1 i: how floor(x / h) keys are
// packed, the exact cell faces, the fixed-point windows) from the key range
// of the input.  The same code runs on the device (in the last block of the
// key-range kernel, so no host round trip separates the range and binning)
// and on the host (when the face table is larger than the device-side
// capacity).
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "gs_plan.h"

namespace gs {

// Order code of a double: a signed integer whose order is the order of the
// values (-0 is taken as +0).
__host__ __device__ inline int64_t plan_ord_of(double x) {
  if (x == 0.0) x = 0.0;
  int64_t s;
  memcpy(&s, &x, 8);
  return s ^ ((s >> 63) & 0x7FFFFFFFFFFFFFFFll);
}

__host__ __device__ inline double plan_from_ord(int64_t o) {
  const int64_t s = o ^ ((o >> 63) & 0x7FFFFFFFFFFFFFFFll);
  double x;
  memcpy(&x, &s, 8);
  return x;
}

// The least double t with t >= q * h (exactly); the error of the rounded
// product q * h is itself a double, obtained exactly by one fused multiply-add.
__host__ __device__ inline double plan_face(int64_t q, double h) {
  const double qd = (double)q;
  double p = qd * h;
  const double r = fma(qd, h, -p);
  if (r > 0) p = nextafter(p, INFINITY);
  return p;
}

// floor(x / h) of the exact quotient: the q with face(q) <= x < face(q + 1).
__host__ __device__ inline int64_t plan_floor_div(double x, double h) {
  int64_t q = (int64_t)floor(x / h);
  for (int i = 0; i < 4 && plan_face(q, h) > x; ++i) --q;
  for (int i = 0; i < 4 && plan_face(q + 1, h) <= x; ++i) ++q;
  return q;
}

__host__ __device__ inline int plan_bitlen(uint64_t v) {
  int b = 0;
  for (; v; v >>= 1) ++b;
  return b;
}

// Axis a of the plan from the key range in fl (its min_ord, max_ord,
// maxabs): the data's key box along the axis widened by one cell each side
// (centroids are convex combinations of the points, Eq. 1 and Eq. 3, and
// leave that box by a few roundings at most), and the fixed-point unit 2^L
// that holds n coordinate sums exactly.  Returns a plan status.
__host__ __device__ inline uint32_t plan_axis(int a, double h, int64_t n, const DevFlags& fl,
                                              Plan& P) {
  int clog2n = 0;
  while ((1ll << clog2n) < n) ++clog2n;
  const double lo = plan_from_ord(fl.min_ord[a]), hi = plan_from_ord(fl.max_ord[a]);
  if (!(fabs(lo / h) < 4.0e15) || !(fabs(hi / h) < 4.0e15)) return kPlanRangeH;
  const int64_t kmin = plan_floor_div(lo, h) - 1, kmax = plan_floor_div(hi, h) + 1;
  const int64_t span = kmax - kmin + 1;
  if (span > (1ll << 22)) return kPlanSpan;
  P.kmin[a] = kmin;
  P.span[a] = (int)span;
  double ma;
  const uint64_t mb = fl.maxabs[a];
  memcpy(&ma, &mb, 8);
  int e = 0;
  if (ma > 0) frexp(ma, &e);  // ma < 2^e
  P.L[a] = e + clog2n - 126;
  return kPlanOK;
}

// The rest of the plan once every axis has its span: the packed-key layout
// (axis 0 most significant; B > 1 adds the instance field above the axes),
// the face-table offsets and the neighbour count.  z receives the face-table
// length, the product of the spans and the key width.  Returns a plan status.
__host__ __device__ inline uint32_t plan_finish(int d, double h, int B, Plan& P, PlanSizes& z) {
  P.d = d;
  P.inv_h = (float)(1.0 / h);
  P.h32 = (float)h;
  z.span_prod = 1;
  z.thr_words = 0;
  for (int a = 0; a < d; ++a) {
    P.thr_off[a] = (int)z.thr_words;
    z.thr_words += (uint64_t)P.span[a] + 1;
    z.span_prod = z.span_prod > (1ull << 40) ? z.span_prod : z.span_prod * (uint64_t)P.span[a];
  }
  int total = 0;
  for (int a = d - 1; a >= 0; --a) {
    P.off[a] = total;
    total += plan_bitlen((uint64_t)P.span[a] + 1);
  }
  // batched runs: the instance index in the field above all axes (it is
  // never probed, so cells of different instances never meet)
  P.inst_off = total;
  if (B > 1) total += plan_bitlen((uint64_t)(B - 1));
  z.total_bits = total;
  if (total > 63) return kPlanBits;
  int np = 1;
  for (int a = 0; a < d; ++a) np *= 3;
  P.nprobe = np;
  P.center = (np - 1) / 2;
  return kPlanOK;
}

// The whole plan (Sec. 2.1 i) from the key range in fl, one axis after the
// other.  Returns a plan status.
__host__ __device__ inline uint32_t plan_from_range(int d, double h, int64_t n, int B,
                                                    const DevFlags& fl, Plan& P, PlanSizes& z) {
  memset(&P, 0, sizeof(P));
  for (int a = 0; a < d; ++a) {
    const uint32_t st = plan_axis(a, h, n, fl, P);
    if (st != kPlanOK) return st;
  }
  return plan_finish(d, h, B, P, z);
}

// Entry j of the face table: the order code of the least double >= q h for
// the cell index q it stands for (axis a's entries start at thr_off[a]).
__host__ __device__ inline int64_t plan_face_entry(const Plan& P, double h, uint64_t j) {
  int a = 0;
  while (a + 1 < P.d && j >= (uint64_t)P.thr_off[a + 1]) ++a;
  return plan_ord_of(plan_face(P.kmin[a] + (int64_t)(j - (uint64_t)P.thr_off[a]), h));
}

// Neighbour offset p in {-1,0,1}^d (axis 0 the slowest digit): its packed-key
// offset, and the offset vector as 2 bits per axis (v_a + 1 at bit 2a).
__host__ __device__ inline void plan_probe(const Plan& P, int p, uint64_t* delta, uint32_t* vpack) {
  int64_t dl = 0;
  uint32_t vp = 0;
  int rest = p;
  for (int a = P.d - 1; a >= 0; --a) {
    const int v = rest % 3 - 1;
    rest /= 3;
    dl += (int64_t)v * (int64_t)(1ull << P.off[a]);
    vp |= (uint32_t)(v + 1) << (2 * a);
  }
  *delta = (uint64_t)dl;
  *vpack = vp;
}

}  // namespace gs
