// Shared device/host helpers of the GCR library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math_constants.h>

#include "../../include/gcr.h"

#define GCR_FULL 0xffffffffu

namespace gcr {

constexpr int kMaxK = 64;          // largest k supported by the kNN search
constexpr int kMaxD = 4096;        // largest feature dimension
constexpr int kDsfpMaxK = 64;      // largest k of the local propagation (Algorithm 1)
constexpr int kQCap = 32;          // survivors queued per row before a merge

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over the caller's workspace (256-byte aligned slices).
struct Carve {
  char* base;
  size_t off;
  size_t cap;
  __host__ Carve(void* b, size_t c) : base((char*)b), off(0), cap(c) {}
  template <typename T>
  __host__ T* take(size_t count) {
    off = align_up(off, 256);
    T* p = (T*)(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

// Float-float accumulation of sums of squares or products without FP64 arithmetic (GB300's FP64
// rate is 1/64 of FP32): each product is split exactly (a*b = p + pe with an FMA), each addition
// is an exact TwoSum into (hi, lo); the result is accurate to about 2^-46 relative (for sums
// without cancellation), well below the 1e-12 the FP64 tie-break needs from the squared norms.
struct FF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_sq(float x) {
    const float p = x * x;
    const float pe = fmaf(x, x, -p);
    const float s = hi + p;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (p - bp) + pe;
    hi = s;
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    const float s = hi + p;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (p - bp) + pe;
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Rounding of an FP32 value to TF32 (10 explicit mantissa bits): round to nearest, ties away
// from zero, by adding half a unit of the 13th bit to the magnitude and clearing the low 13
// bits (a carry into the exponent gives the next power of two). Finite inputs only.
__device__ __forceinline__ float round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Strict total order used by every top-k structure: larger value first, then smaller index.
__device__ __forceinline__ bool better(float a, int ai, float b, int bi) {
  return a > b || (a == b && ai < bi);
}
__device__ __forceinline__ bool better_d(double a, int ai, double b, int bi) {
  return a > b || (a == b && ai < bi);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GCR_FULL, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GCR_FULL, v, o);
  return v;
}

// Descending bitonic sort of 32 (value, index) pairs held one per lane.
__device__ __forceinline__ void warp_sort32_desc(float& v, int& vi, int lane) {
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      float ov = __shfl_xor_sync(GCR_FULL, v, stride);
      int oi = __shfl_xor_sync(GCR_FULL, vi, stride);
      bool desc = (lane & size) == 0 || size == 32;
      bool lower = (lane & stride) == 0;
      bool take = (lower == desc) ? better(ov, oi, v, vi) : better(v, vi, ov, oi);
      if (take) { v = ov; vi = oi; }
    }
  }
}

// Descending bitonic merge of a bitonic sequence of 32 pairs held one per lane.
__device__ __forceinline__ void warp_merge32_desc(float& v, int& vi, int lane) {
#pragma unroll
  for (int stride = 16; stride > 0; stride >>= 1) {
    float ov = __shfl_xor_sync(GCR_FULL, v, stride);
    int oi = __shfl_xor_sync(GCR_FULL, vi, stride);
    bool lower = (lane & stride) == 0;
    bool take = lower ? better(ov, oi, v, vi) : better(v, vi, ov, oi);
    if (take) { v = ov; vi = oi; }
  }
}

// The lanes of the warp whose dg equals this lane's (dg < 2^bits, bits <= 9, warp-uniform):
// one ballot per bit, ANDed. The same mask as __match_any_sync(GCR_FULL, dg), but on the ALU
// pipe (the pipe of __match_any_sync bounded the radix sorts that rank keys this way).
__device__ __forceinline__ unsigned warp_peers(uint32_t dg, int bits) {
  unsigned peers = GCR_FULL;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    if (b < bits) {
      const bool bit = (dg >> b) & 1u;
      const unsigned m = __ballot_sync(GCR_FULL, bit);
      peers &= bit ? m : ~m;
    }
  }
  return peers;
}

// float -> uint32 whose unsigned order equals the float order (ascending).
__device__ __forceinline__ uint32_t float_to_ordered(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

struct GcrvWs;
size_t gcrv_carve(Carve& c, int64_t F, int d, int C, int ncam, GcrvWs* w);

}  // namespace gcr

#define GCR_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return GCR_E_CUDA;      \
  } while (0)

#define GCR_LAUNCH_CHECK()                         \
  do {                                             \
    cudaError_t _e = cudaGetLastError();           \
    if (_e != cudaSuccess) return GCR_E_CUDA;      \
  } while (0)
