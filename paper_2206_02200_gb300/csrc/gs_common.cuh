// gs_common.cuh -- launch geometry and small helpers shared by the kernel
// translation units (gs_kernels.cu and the loop kernel's gs_loop*.cu).
#pragma once

#include <cstdio>

#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kLoopBlock = 512;  // threads per block of the loop kernel

inline unsigned grid_for(int64_t work, int per_block = kBlock, unsigned cap = 152u * 32u) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > (int64_t)cap) g = cap;
  return (unsigned)g;
}

#define GS_DISPATCH_D(dval, ...)                  \
  switch (dval) {                                 \
    case 1: { constexpr int D = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int D = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int D = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int D = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int D = 5; __VA_ARGS__; } break; \
    case 6: { constexpr int D = 6; __VA_ARGS__; } break; \
    case 7: { constexpr int D = 7; __VA_ARGS__; } break; \
    case 8: { constexpr int D = 8; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;        \
  }


__device__ __forceinline__ uint64_t bits_of(double v) { return (uint64_t)__double_as_longlong(v); }
__device__ __forceinline__ uint64_t bits_of(float v) {
  return f32_bits_to_f64_bits((uint32_t)__float_as_uint(v));
}

}  // namespace
}  // namespace gs
