// Host build of the library's exact-arithmetic helpers
// (paper_2206_02200_gb300/csrc/gs_device.cuh: float64 <-> 128-bit fixed point,
// rounding of exact sums and of exact quotients to float64), for
// tests/test_device_math_host.py; key_index comes with the face table the
// planner (gs_planner.cuh) builds; the hash table's insert and lookup run on
// one thread.  The CUDA names the headers use get host meanings below.
// Queries on stdin, one answer line each (integers in hex, two 64-bit halves
// for a 128-bit value, float64 results as their bit patterns):
//   T bits L        -> to_fixed: hi lo inexact err
//   R hi lo L       -> round_fixed: bits
//   Q hi lo L       -> round_to_double: hi lo err
//   V hi lo D L     -> div_round: bits inexact
//   W f32bits       -> f32_bits_to_f64_bits: bits
//   I u32           -> u32_to_f64_bits: bits
//   K h kmin span x -> key_index over the face table of cells kmin .. kmin+span-1
//                      (h and x as C99 hex floats): the cell's index
//   H cap n k_1 .. k_n m a_1 .. a_m -> a table of cap slots: per insert of k_i
//                      "slot won", then per lookup of a_j its slot (or
//                      ffffffff), then the error word
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#define __device__
#define __host__
#define __forceinline__ inline
#define __restrict__ __restrict

struct ulonglong2 {
  unsigned long long x, y;
};

static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
static inline int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }
static inline int __popc(unsigned x) { return __builtin_popcount(x); }
static inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b) {
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
static inline double __longlong_as_double(long long v) {
  double d;
  std::memcpy(&d, &v, 8);
  return d;
}
static inline long long __double_as_longlong(double d) {
  long long v;
  std::memcpy(&v, &d, 8);
  return v;
}
static inline unsigned __float_as_uint(float f) {
  unsigned u;
  std::memcpy(&u, &f, 4);
  return u;
}
static inline float __uint_as_float(unsigned u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
static inline long long __float2ll_rd(float f) { return (long long)std::floor(f); }
template <class T>
static inline T __ldg(const T* p) { return *p; }
template <class T>
static inline T __ldcg(const T* p) { return *p; }
// atomics with their single-thread meaning (the hash table checks run on one
// thread); warp shuffles are declared only (nothing checked here calls them)
template <class T, class U>
T atomicAdd(T* p, U v) {
  const T old = *p;
  *p = old + (T)v;
  return old;
}
template <class T, class U, class V>
T atomicCAS(T* p, U c, V v) {
  const T old = *p;
  if (old == (T)c) *p = (T)v;
  return old;
}
template <class T, class U>
T atomicOr(T* p, U v) {
  const T old = *p;
  *p = old | (T)v;
  return old;
}
template <class T>
T __shfl_xor_sync(unsigned mask, T v, int lane, int width = 32);

#include "../paper_2206_02200_gb300/csrc/gs_device.cuh"
#include "../paper_2206_02200_gb300/csrc/gs_planner.cuh"

#include <cstdlib>
#include <vector>

using gs::u128;

static u128 read128(unsigned long long hi, unsigned long long lo) {
  return ((u128)hi << 64) | lo;
}

static unsigned long long bits_of(double d) { return (unsigned long long)__double_as_longlong(d); }

int main() {
  char op[8];
  while (std::scanf("%7s", op) == 1) {
    unsigned long long hi = 0, lo = 0, b = 0;
    int L = 0;
    unsigned inexact = 0, err = 0;
    if (std::strcmp(op, "T") == 0) {
      if (std::scanf("%llx %d", &b, &L) != 2) return 2;
      const u128 V = gs::to_fixed(b, L, inexact, err);
      std::printf("%llx %llx %u %u\n", (unsigned long long)(V >> 64), (unsigned long long)V,
                  inexact, err);
    } else if (std::strcmp(op, "R") == 0) {
      if (std::scanf("%llx %llx %d", &hi, &lo, &L) != 3) return 2;
      std::printf("%llx\n", bits_of(gs::round_fixed(read128(hi, lo), L, inexact)));
    } else if (std::strcmp(op, "Q") == 0) {
      if (std::scanf("%llx %llx %d", &hi, &lo, &L) != 3) return 2;
      const u128 V = gs::round_to_double(read128(hi, lo), L, err);
      std::printf("%llx %llx %u\n", (unsigned long long)(V >> 64), (unsigned long long)V, err);
    } else if (std::strcmp(op, "V") == 0) {
      unsigned D = 0;
      if (std::scanf("%llx %llx %u %d", &hi, &lo, &D, &L) != 4 || D == 0) return 2;
      const double q = gs::div_round(read128(hi, lo), D, L, inexact);
      std::printf("%llx %u\n", bits_of(q), inexact);
    } else if (std::strcmp(op, "W") == 0) {
      unsigned f = 0;
      if (std::scanf("%x", &f) != 1) return 2;
      std::printf("%llx\n", (unsigned long long)gs::f32_bits_to_f64_bits(f));
    } else if (std::strcmp(op, "I") == 0) {
      unsigned v = 0;
      if (std::scanf("%x", &v) != 1) return 2;
      std::printf("%llx\n", (unsigned long long)gs::u32_to_f64_bits(v));
    } else if (std::strcmp(op, "K") == 0) {
      char hs[64], xs[64];
      long long kmin = 0;
      int span = 0;
      if (std::scanf("%63s %lld %d %63s", hs, &kmin, &span, xs) != 4 || span < 1) return 2;
      const double h = std::strtod(hs, nullptr), x = std::strtod(xs, nullptr);
      std::vector<int64_t> thr((size_t)span + 1);
      for (int j = 0; j <= span; ++j) thr[(size_t)j] = gs::plan_ord_of(gs::plan_face(kmin + j, h));
      std::printf("%d\n", gs::key_index(thr.data(), span, (int64_t)kmin, (float)(1.0 / h),
                                        bits_of(x)));
    } else if (std::strcmp(op, "H") == 0) {
      unsigned cap = 0;
      int n = 0, m = 0;
      if (std::scanf("%u %d", &cap, &n) != 2 || cap < 4 || (cap & (cap - 1)) || n < 0) return 2;
      // 32-byte aligned key array, all slots empty
      std::vector<ulonglong2> store((size_t)cap / 2 + 2);
      uint64_t* keys = reinterpret_cast<uint64_t*>(
          (reinterpret_cast<uintptr_t>(store.data()) + 31) & ~(uintptr_t)31);
      for (unsigned i = 0; i < cap; ++i) keys[i] = gs::kEmpty;
      uint32_t err = 0;
      for (int i = 0; i < n; ++i) {
        unsigned long long k = 0;
        if (std::scanf("%llx", &k) != 1) return 2;
        bool won = false;
        const uint32_t sl = gs::table_insert(keys, cap - 1, k, won, &err);
        std::printf("%x %d ", sl, won ? 1 : 0);
      }
      if (std::scanf("%d", &m) != 1 || m < 0) return 2;
      for (int j = 0; j < m; ++j) {
        unsigned long long k = 0;
        if (std::scanf("%llx", &k) != 1) return 2;
        const uint64_t q[1] = {k};
        const bool v[1] = {true};
        uint32_t sl[1];
        gs::table_find_many<1>(keys, cap - 1, q, v, sl);
        std::printf("%x ", sl[0]);
      }
      std::printf("%u\n", err);
    } else {
      return 2;
    }
  }
  return 0;
}
