// Host build of the library's planner (paper_2206_02200_gb300/csrc/gs_planner.cuh:
// the exact cell faces and floor(x / h) decisions of Sec. 2.1 i, the packed-key
// layout and the neighbour offsets), for tests/test_planner_host.py.  Reads
// one query per line from stdin and prints one answer per line:
//   F x h        -> plan_floor_div(x, h)
//   A q h        -> plan_face(q, h) as a hex float
//   O x          -> plan_ord_of(x)
//   L d B s_0 .. s_{d-1} -> plan_finish status, total key bits, then for every
//                   probe p: its packed-key offset and 2-bit offset vector
//   P d h n B (lo hi maxabs) x d -> plan_from_range from the key range: status,
//                   then per axis "kmin span L thr_off", then the face-table length
// Doubles are read and written as C99 hex floats.
#define __host__
#define __device__
#include <cinttypes>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../paper_2206_02200_gb300/csrc/gs_planner.cuh"

int main() {
  char op[8];
  while (std::scanf("%7s", op) == 1) {
    if (std::strcmp(op, "F") == 0) {
      char xs[64], hs[64];
      if (std::scanf("%63s %63s", xs, hs) != 2) return 2;
      std::printf("%" PRId64 "\n", gs::plan_floor_div(std::strtod(xs, nullptr),
                                                     std::strtod(hs, nullptr)));
    } else if (std::strcmp(op, "A") == 0) {
      long long q;
      char hs[64];
      if (std::scanf("%lld %63s", &q, hs) != 2) return 2;
      std::printf("%a\n", gs::plan_face((int64_t)q, std::strtod(hs, nullptr)));
    } else if (std::strcmp(op, "O") == 0) {
      char xs[64];
      if (std::scanf("%63s", xs) != 1) return 2;
      std::printf("%" PRId64 "\n", gs::plan_ord_of(std::strtod(xs, nullptr)));
    } else if (std::strcmp(op, "L") == 0) {
      int d, B;
      if (std::scanf("%d %d", &d, &B) != 2 || d < 1 || d > gs::kMaxD) return 2;
      gs::Plan P;
      std::memset(&P, 0, sizeof(P));
      for (int a = 0; a < d; ++a)
        if (std::scanf("%d", &P.span[a]) != 1) return 2;
      gs::PlanSizes z;
      const uint32_t st = gs::plan_finish(d, 1.0, B, P, z);
      std::printf("%u %d", st, z.total_bits);
      if (st == gs::kPlanOK) {
        for (int p = 0; p < P.nprobe; ++p) {
          uint64_t delta;
          uint32_t vp;
          gs::plan_probe(P, p, &delta, &vp);
          std::printf(" %" PRIu64 ":%u", delta, vp);
        }
        for (int a = 0; a < d; ++a) std::printf(" off%d=%d", a, P.off[a]);
      }
      std::printf("\n");
    } else if (std::strcmp(op, "P") == 0) {
      int d, B;
      char hs[64];
      long long n;
      if (std::scanf("%d %63s %lld %d", &d, hs, &n, &B) != 4 || d < 1 || d > gs::kMaxD) return 2;
      gs::DevFlags fl;
      std::memset(&fl, 0, sizeof(fl));
      for (int a = 0; a < d; ++a) {
        char ls[64], us[64], ms[64];
        if (std::scanf("%63s %63s %63s", ls, us, ms) != 3) return 2;
        fl.min_ord[a] = gs::plan_ord_of(std::strtod(ls, nullptr));
        fl.max_ord[a] = gs::plan_ord_of(std::strtod(us, nullptr));
        const double m = std::strtod(ms, nullptr);
        std::memcpy(&fl.maxabs[a], &m, 8);
      }
      gs::Plan P;
      gs::PlanSizes z;
      std::memset(&z, 0, sizeof(z));
      const uint32_t st = gs::plan_from_range(d, std::strtod(hs, nullptr), n, B, fl, P, z);
      std::printf("%u", st);
      if (st == gs::kPlanOK) {
        for (int a = 0; a < d; ++a)
          std::printf(" %lld %d %d %d", (long long)P.kmin[a], P.span[a], P.L[a], P.thr_off[a]);
        std::printf(" %llu", (unsigned long long)z.thr_words);
      }
      std::printf("\n");
    } else {
      return 2;
    }
  }
  return 0;
}
