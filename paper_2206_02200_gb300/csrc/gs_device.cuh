// gs_device.cuh -- device-side building blocks of the GridShift library:
// exact fixed-point arithmetic, the packed-key hash table and the integer-only
// cell-key decision.  Included by the kernel translation units only.
//
// Why fixed point: every sum of the method (cell sums of Sec. 2.1 i and Eq. 3-4,
// neighbourhood sums of Eq. 1-2) is formed exactly as a two's-complement 128-bit
// integer in units of 2^L (L chosen per coordinate so that n * max|x| < 2^(L+126))
// and rounded once to float64.  The result is independent of the order of the
// additions, so atomics give deterministic results, and no float64 instruction
// is needed on the per-point path.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gs_plan.h"

namespace gs {

typedef unsigned __int128 u128;

constexpr uint64_t kEmpty = ~0ull;      // empty hash slot (packed keys use <= 63 bits)
constexpr uint32_t kNone = 0xFFFFFFFFu; // "no cell"
constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// float64 bit helpers (integer instructions only)

// Maps a double to an int64 whose signed order is the numeric order of the
// doubles (finite values; -0.0 is mapped like +0.0).
__device__ __forceinline__ int64_t ord_of_bits(uint64_t b) {
  if (b == 0x8000000000000000ull) b = 0;
  int64_t s = (int64_t)b;
  return s ^ ((s >> 63) & 0x7FFFFFFFFFFFFFFFll);
}

// The float64 bit pattern of an unsigned 32-bit integer (exact: every such
// integer is a double), built with integer instructions: the leading one at
// bit e gives the exponent 1023 + e and the bits below it the fraction.
__device__ __forceinline__ uint64_t u32_to_f64_bits(uint32_t v) {
  if (v == 0) return 0;
  const int e = 31 - __clz(v);
  const uint64_t mant = ((uint64_t)v << (52 - e)) & 0xFFFFFFFFFFFFFull;
  return ((uint64_t)(1023 + e) << 52) | mant;
}

// Exact float32 -> float64 widening on the bit patterns (finite inputs).
__device__ __forceinline__ uint64_t f32_bits_to_f64_bits(uint32_t f) {
  uint64_t sign = (uint64_t)(f >> 31) << 63;
  uint32_t e = (f >> 23) & 0xFF;
  uint32_t m = f & 0x7FFFFF;
  if (e == 0) {
    if (m == 0) return sign;
    // subnormal float: value = m * 2^-149 with the leading one at bit p
    int p = 31 - __clz(m);
    uint64_t mant = ((uint64_t)m << (52 - p)) & 0xFFFFFFFFFFFFFull;
    return sign | ((uint64_t)(p - 149 + 1023) << 52) | mant;
  }
  if (e == 0xFF) return sign | (0x7FFull << 52) | ((uint64_t)m << 29);
  return sign | ((uint64_t)(e - 127 + 1023) << 52) | ((uint64_t)m << 29);
}

template <typename T>
__device__ __forceinline__ uint64_t load_bits(const T* p);
template <>
__device__ __forceinline__ uint64_t load_bits<double>(const double* p) {
  return (uint64_t)__double_as_longlong(__ldg(p));
}
template <>
__device__ __forceinline__ uint64_t load_bits<float>(const float* p) {
  return f32_bits_to_f64_bits((uint32_t)__float_as_uint(__ldg(p)));
}

// ---------------------------------------------------------------------------
// Exact fixed point

// v (float64 bits) as a two's-complement integer in units of 2^L.  Sets
// *inexact when v has nonzero bits below 2^L, *err when |v| >= 2^(L+126).
__device__ __forceinline__ u128 to_fixed(uint64_t b, int L, unsigned& inexact, unsigned& err) {
  uint64_t neg = b >> 63;
  int e = (int)((b >> 52) & 0x7FF);
  uint64_t M = b & 0xFFFFFFFFFFFFFull;
  if (e == 0) {
    if (M == 0) return 0;
    e = 1;
  } else {
    M |= 1ull << 52;
  }
  int s = e - 1075 - L;  // v = M * 2^(e-1075) = M * 2^s units
  u128 V;
  if (s >= 0) {
    if (s > 73) { err = 1; return 0; }
    V = (u128)M << s;
  } else {
    int r = -s;
    if (r >= 64) {
      inexact = 1;
      V = 0;
    } else {
      if (M & ((1ull << r) - 1)) inexact = 1;
      V = (u128)(M >> r);
    }
  }
  return neg ? (u128)0 - V : V;
}

__device__ __forceinline__ bool is_neg(u128 V) { return (int64_t)(uint64_t)(V >> 64) < 0; }

// Bits [pos, pos + 64) of the little-endian 32-bit limb vector w (pos >= 0).
template <int NL>
__device__ __forceinline__ uint64_t limb_bits64(const uint32_t (&w)[NL], int pos) {
  int i = pos >> 5, sh = pos & 31;
  uint64_t lo = 0, mid = 0, hi = 0;
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    if (k == i) lo = w[k];
    if (k == i + 1) mid = w[k];
    if (k == i + 2) hi = w[k];
  }
  u128 v = (u128)lo | ((u128)mid << 32) | ((u128)hi << 64);
  return (uint64_t)(v >> sh);
}

// True if any bit below position pos (pos >= 0) of w is set.
template <int NL>
__device__ __forceinline__ bool limb_any_below(const uint32_t (&w)[NL], int pos) {
  bool any = false;
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    int base = k * 32;
    if (base + 32 <= pos) {
      any |= (w[k] != 0);
    } else if (base < pos) {
      any |= ((w[k] & ((1u << (pos - base)) - 1u)) != 0);
    }
  }
  return any;
}

// Rounds (-1)^neg * (W + f) * 2^e0 to the nearest float64, ties to even, where
// W is the unsigned integer held in the limbs w and f in [0, 1) is nonzero iff
// sticky_in.  Sets inexact when f could decide the rounding but is unknown.
template <int NL>
__device__ double round_limbs(const uint32_t (&w)[NL], int e0, bool neg, bool sticky_in,
                              unsigned& inexact) {
  int top = -1;
#pragma unroll
  for (int k = 0; k < NL; ++k)
    if (w[k] != 0) top = k;
  if (top < 0) {
    if (sticky_in) inexact = 1;
    return neg ? -0.0 : 0.0;
  }
  uint32_t wt = 0;
#pragma unroll
  for (int k = 0; k < NL; ++k)
    if (k == top) wt = w[k];
  int P = top * 32 + 31 - __clz(wt);  // position of the leading one
  int rp = P - 52;                    // position of the result's last bit
  if (rp + e0 < -1074) rp = -1074 - e0;
  uint64_t sig;
  bool guard = false, sticky = sticky_in;
  if (rp <= 0) {
    if (sticky_in) inexact = 1;
    sig = limb_bits64<NL>(w, 0) << (-rp);
  } else {
    int nb = P - rp + 1;  // <= 53
    sig = limb_bits64<NL>(w, rp);
    if (nb < 64) sig &= (1ull << nb) - 1;
    guard = (limb_bits64<NL>(w, rp - 1) & 1ull) != 0;
    sticky = sticky || limb_any_below<NL>(w, rp - 1);
  }
  if (guard && (sticky || (sig & 1ull))) sig += 1;
  if (sig >> 53) {
    sig >>= 1;
    rp += 1;
  }
  int e2 = rp + e0;  // value = sig * 2^e2
  uint64_t bits;
  if (sig >> 52) {
    bits = ((uint64_t)(e2 + 52 + 1023) << 52) | (sig & 0xFFFFFFFFFFFFFull);
  } else {
    bits = sig;  // subnormal: e2 == -1074
  }
  if (neg) bits |= 1ull << 63;
  return __longlong_as_double((long long)bits);
}

// Round the exact value V * 2^L (V two's complement) to float64.
__device__ __forceinline__ double round_fixed(u128 V, int L, unsigned& inexact) {
  bool neg = is_neg(V);
  u128 mag = neg ? (u128)0 - V : V;
  uint32_t w[4] = {(uint32_t)mag, (uint32_t)(mag >> 32), (uint32_t)(mag >> 64),
                   (uint32_t)(mag >> 96)};
  return round_limbs<4>(w, L, neg, false, inexact);
}

// V (units of 2^L, two's complement) rounded to the nearest value a float64
// holds (ties to even), still in units of 2^L: the value round_fixed gives,
// converted back by to_fixed, computed on the integer directly (keep the 53
// bits from the leading one, or the bits from 2^-1074 up where that is
// lower, and round on the rest).  Sets err where to_fixed would: a result of
// 2^126 or more.
__device__ __forceinline__ u128 round_to_double(u128 V, int L, unsigned& err) {
  const bool neg = is_neg(V);
  u128 mag = neg ? (u128)0 - V : V;
  if (mag == 0) return 0;
  const uint64_t hi = (uint64_t)(mag >> 64), lo = (uint64_t)mag;
  const int P = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  int rp = P - 52;  // the last bit kept
  if (rp < -1074 - L) rp = -1074 - L;
  if (rp > 0) {
    const u128 keep = mag >> rp;
    const u128 rem = mag - (keep << rp);
    const u128 half = (u128)1 << (rp - 1);
    const bool up = rem > half || (rem == half && ((uint64_t)keep & 1u));
    mag = (keep + (up ? 1u : 0u)) << rp;
  }
  if ((uint64_t)(mag >> 64) >> 62) err = 1;
  return neg ? (u128)0 - mag : mag;
}

// Round the exact quotient (N * 2^L) / D to float64 (D >= 1).  Long division
// of N * 2^64 by D in 32-bit digits, from the top; once three digits below
// the leading nonzero one are known (at least 65 quotient bits), the rest only
// matters as a sticky bit: nonzero iff the partial remainder is.  Each digit
// is estimated with a 64-bit reciprocal of D and corrected exactly.
__device__ __forceinline__ double div_round(u128 N, uint32_t D, int L, unsigned& inexact) {
  bool neg = is_neg(N);
  u128 mag = neg ? (u128)0 - N : N;
  uint32_t w[6] = {0u, 0u, (uint32_t)mag, (uint32_t)(mag >> 32), (uint32_t)(mag >> 64),
                   (uint32_t)(mag >> 96)};
  uint32_t q[6] = {0u, 0u, 0u, 0u, 0u, 0u};
  const uint64_t r = ~0ull / D;  // floor((2^64 - 1) / D) <= 2^64 / D
  uint64_t rem = 0;
  int lead = -1;  // index of the leading nonzero quotient digit
  bool sticky = false;
#pragma unroll
  for (int k = 5; k >= 0; --k) {
    if (lead >= 0 && lead - k >= 3) {
      sticky = sticky || w[k] != 0u;
      continue;
    }
    uint64_t cur = (rem << 32) | w[k];  // cur < D * 2^32
    uint64_t qq = __umul64hi(cur, r);  // qq <= cur / D < qq + 3
    uint64_t rr = cur - qq * D;
    if (rr >= D) { rr -= D; ++qq; }
    if (rr >= D) { rr -= D; ++qq; }
    q[k] = (uint32_t)qq;
    rem = rr;
    if (lead < 0 && qq != 0) lead = k;
  }
  sticky = sticky || rem != 0;
  return round_limbs<6>(q, L - 64, neg, sticky, inexact);
}

// Sum of four 64-bit limb accumulators (limb k holds a sum of 32-bit pieces of
// weight 2^(32k)) as a two's-complement 128-bit value.
__device__ __forceinline__ u128 limbs_value(const uint64_t* acc) {
  return (u128)acc[0] + ((u128)acc[1] << 32) + ((u128)acc[2] << 64) + ((u128)acc[3] << 96);
}

// acc += V exactly (mod 2^128); every limb receives a value below 2^32, so a
// limb cannot overflow before 2^32 additions.
__device__ __forceinline__ void atomic_add_fixed(uint64_t* acc, u128 V) {
  uint32_t p0 = (uint32_t)V, p1 = (uint32_t)(V >> 32), p2 = (uint32_t)(V >> 64),
           p3 = (uint32_t)(V >> 96);
  if (p0) atomicAdd((unsigned long long*)&acc[0], (unsigned long long)p0);
  if (p1) atomicAdd((unsigned long long*)&acc[1], (unsigned long long)p1);
  if (p2) atomicAdd((unsigned long long*)&acc[2], (unsigned long long)p2);
  if (p3) atomicAdd((unsigned long long*)&acc[3], (unsigned long long)p3);
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int o) {
  uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
  lo = __shfl_xor_sync(kFull, lo, o);
  hi = __shfl_xor_sync(kFull, hi, o);
  return (u128)lo | ((u128)hi << 64);
}

// ---------------------------------------------------------------------------
// Hash table over packed keys: open addressing over buckets of kBucket = 4
// slots (32 bytes of keys, one DRAM/L2 sector), linear probing from bucket to
// bucket, capacity a power of two >= 4.  The home bucket is Fibonacci
// (multiplicative) hashing: the top log2(buckets) bits of key * 2^64/phi,
// which depend on every bit of the key.  Within a bucket, inserts fill slots
// in order, so once the inserts of a phase are done the occupied slots of a
// bucket are a prefix and a lookup can stop at the first bucket holding an
// empty slot.  The key array must be 32-byte aligned.

constexpr uint32_t kBucket = 4;

__device__ __host__ __forceinline__ uint32_t home_bucket(uint64_t key, uint32_t bmask) {
#ifdef __CUDA_ARCH__
  const int b = __popc(bmask);
#else
  const int b = __builtin_popcount(bmask);
#endif
  return b == 0 ? 0u : (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - b));
}

// Longest probe sequence: an insert that finds no free slot within
// kMaxProbeBuckets buckets of the key's home fails (kErrTableFull), so every
// stored key lies within that many buckets of its home and a lookup may stop
// there.  At the load factors used (<= 1/2) sequences this long do not occur
// in practice; the bound keeps an over-full table from turning into a
// near-endless scan.
constexpr uint32_t kMaxProbeBuckets = 128;

__device__ __forceinline__ uint32_t probe_limit(uint32_t bmask) {
  return bmask < kMaxProbeBuckets ? bmask + 1 : kMaxProbeBuckets;
}

// Index of key in the four keys of a bucket, 4 if absent; *open is set when
// the bucket holds an empty slot (so the key is in no later bucket).
__device__ __forceinline__ uint32_t bucket_match(ulonglong2 lo, ulonglong2 hi, uint64_t key,
                                                 bool* open) {
  *open = lo.x == kEmpty || lo.y == kEmpty || hi.x == kEmpty || hi.y == kEmpty;
  return lo.x == key ? 0u : lo.y == key ? 1u : hi.x == key ? 2u : hi.y == key ? 3u : 4u;
}

// Slot holding key, or kNone, scanning from bucket b (the i0-th bucket of the
// key's sequence).  mask = capacity - 1.
__device__ __forceinline__ uint32_t table_find_from(const uint64_t* keys, uint32_t mask,
                                                    uint64_t key, uint32_t b, uint32_t i0) {
  const uint32_t bmask = mask >> 2;
  const uint32_t lim = probe_limit(bmask);
  for (uint32_t i = i0; i < lim; ++i) {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(keys + (size_t)b * kBucket);
    const ulonglong2 lo = p[0], hi = p[1];
    bool open;
    const uint32_t j = bucket_match(lo, hi, key, &open);
    if (j < kBucket) return b * kBucket + j;
    if (open) return kNone;
    b = (b + 1) & bmask;
  }
  return kNone;
}

// Lookups of U keys at once: the home buckets of all of them are loaded
// before any is examined, so the U loads are in flight together.  valid[u]
// false leaves slot[u] = kNone.
template <int U>
__device__ __forceinline__ void table_find_many(const uint64_t* keys, uint32_t mask,
                                                const uint64_t (&key)[U], const bool (&valid)[U],
                                                uint32_t (&slot)[U]) {
  const uint32_t bmask = mask >> 2;
  uint32_t b[U];
  ulonglong2 lo[U], hi[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    b[u] = home_bucket(key[u], bmask);
    if (valid[u]) {
      const ulonglong2* p = reinterpret_cast<const ulonglong2*>(keys + (size_t)b[u] * kBucket);
      lo[u] = p[0];
      hi[u] = p[1];
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    slot[u] = kNone;
    if (!valid[u]) continue;
    bool open;
    const uint32_t j = bucket_match(lo[u], hi[u], key[u], &open);
    if (j < kBucket) {
      slot[u] = b[u] * kBucket + j;
    } else if (!open) {
      slot[u] = table_find_from(keys, mask, key[u], (b[u] + 1) & bmask, 1);
    }
  }
}

// Slot of key, inserting it if absent; won is set for the inserting thread.
// Returns kNone (and sets kErrTableFull) when no free slot is found.  The
// bucket is read at L2 (the point of coherence), then empty slots are claimed
// in order with compare-and-swap.
__device__ __forceinline__ uint32_t table_insert(uint64_t* keys, uint32_t mask, uint64_t key,
                                                 bool& won, uint32_t* err) {
  const uint32_t bmask = mask >> 2;
  uint32_t b = home_bucket(key, bmask);
  won = false;
  const uint32_t lim = probe_limit(bmask);
  for (uint32_t i = 0; i < lim; ++i) {
    uint64_t* p = keys + (size_t)b * kBucket;
    const ulonglong2 lo = __ldcg(reinterpret_cast<const ulonglong2*>(p));
    const ulonglong2 hi = __ldcg(reinterpret_cast<const ulonglong2*>(p) + 1);
    bool open;
    const uint32_t j = bucket_match(lo, hi, key, &open);
    if (j < kBucket) return b * kBucket + j;
    if (open) {
      const uint64_t seen[kBucket] = {lo.x, lo.y, hi.x, hi.y};
#pragma unroll
      for (uint32_t q = 0; q < kBucket; ++q) {
        if (seen[q] != kEmpty) continue;
        const uint64_t prev = atomicCAS((unsigned long long*)&p[q], (unsigned long long)kEmpty,
                                        (unsigned long long)key);
        if (prev == kEmpty) {
          won = true;
          return b * kBucket + q;
        }
        if (prev == key) return b * kBucket + q;
      }
    }
    b = (b + 1) & bmask;
  }
  atomicOr(err, kErrTableFull);
  return kNone;
}

// Capacity mask of a table that receives at most m distinct keys: load <= 1/4
// where cap_max allows (lookups then rarely leave the home bucket).
__device__ __host__ __forceinline__ uint32_t mask_for(uint32_t m, uint32_t cap_max) {
  uint32_t c = 64;
  while (c < 4u * m && c < cap_max) c <<= 1;
  return c - 1;
}

// ---------------------------------------------------------------------------
// Cell key of one coordinate: the index j in [0, span) with
// thr[j] <= v < thr[j+1], where thr[j] is the order code of the least double
// >= (kmin + j) * h.  That is floor(x / h) - kmin of the exact quotient,
// decided by integer compares.  A float estimate of x / h gives the first
// guess (at most a cell off while |x / h| < 2^20), a few steps correct it, and
// a binary search settles anything further away.

// float with the sign, exponent and leading 23 significand bits of a double
// (0 for magnitudes below the float normal range, +-2^127 above it).
__device__ __forceinline__ float approx_float(uint64_t b) {
  uint32_t sign = (uint32_t)(b >> 63) << 31;
  int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | (254u << 23));
  return __uint_as_float(sign | ((uint32_t)e << 23) | (uint32_t)((b >> 29) & 0x7FFFFF));
}

__device__ __forceinline__ int key_index_search(const int64_t* __restrict__ thr, int span,
                                                int64_t v) {
  int lo = 0, hi = span - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(&thr[mid]) <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int key_index(const int64_t* __restrict__ thr, int span, int64_t kmin,
                                         float inv_h, uint64_t bits) {
  const int64_t v = ord_of_bits(bits);
  const float g = approx_float(bits) * inv_h;
  int idx = 0;
  if (fabsf(g) < 4.0e15f) {
    const long long q = __float2ll_rd(g) - kmin;
    idx = q < 0 ? 0 : (q >= span ? span - 1 : (int)q);
  }
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    if (idx > 0 && v < __ldg(&thr[idx])) {
      --idx;
    } else if (idx < span - 1 && v >= __ldg(&thr[idx + 1])) {
      ++idx;
    } else {
      return idx;
    }
  }
  return key_index_search(thr, span, v);
}

}  // namespace gs
