// Segmented sort of the re-ranked distances (one segment per query).
//
// Each query's gallery distances become 64-bit keys (order-preserving bits of the FP32
// distance, gallery index), so one ascending sort yields the ranking with ties broken by the
// smaller gallery index. One CTA per query sorts the whole segment (up to 16384 keys) with a
// bitonic network whose data stay in registers: each thread holds E consecutive keys, so
// strides below E are exchanged inside a thread, strides below 32E through warp shuffles, and
// only the strides of 32E and more (15 of the 105 stages for 16384 keys) go through shared
// memory. The first K keys are written out.
#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

constexpr int kMaxSeg = 16384;

__device__ __forceinline__ void cmp_swap(unsigned long long& lo, unsigned long long& hi, bool asc) {
  const bool sw = asc ? (lo > hi) : (lo < hi);
  if (sw) {
    const unsigned long long t = lo;
    lo = hi;
    hi = t;
  }
}

// In-thread stage with a compile-time stride (keeps the key array in registers).
template <int E, int S>
__device__ __forceinline__ void reg_stage(unsigned long long (&key)[E], int base, int size) {
  if constexpr (S < E) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int j = i ^ S;
      if (j > i) cmp_swap(key[i], key[j], ((base + i) & size) == 0);
    }
  }
}

// Shared-memory position of key e: one padding word every 32 keys, so that the blocked
// (E consecutive keys per thread) and the strided access patterns both avoid bank conflicts.
__device__ __forceinline__ int pad(int e) { return e + (e >> 5); }

template <int E>
__global__ void __launch_bounds__(1024) rank_rows_kernel(const float* __restrict__ D, int ng, int N, int K,
                                                          int32_t* __restrict__ idx_out, float* __restrict__ dist_out) {
  extern __shared__ unsigned long long sk[];
  const int q = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, T = blockDim.x;
  const int base = t * E;
  const float* row = D + (size_t)q * ng;
  // coalesced load into shared memory, then E consecutive keys per thread into registers
  for (int e = t; e < N; e += T)
    sk[pad(e)] = e < ng ? (((unsigned long long)float_to_ordered(row[e]) << 32) | (unsigned)e) : ~0ull;
  __syncthreads();
  unsigned long long key[E];
#pragma unroll
  for (int i = 0; i < E; ++i) key[i] = sk[pad(base + i)];
  __syncthreads();
  const int wide = 32 * E;  // strides at or above this cross warps
  bool in_smem = false;
  for (int size = 2; size <= N; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= wide) {
        if (!in_smem) {
#pragma unroll
          for (int i = 0; i < E; ++i) sk[pad(base + i)] = key[i];
          __syncthreads();
          in_smem = true;
        }
        for (int p = t; p < (N >> 1); p += T) {
          const int lo = 2 * p - (p & (stride - 1));
          const int hi = lo + stride;
          unsigned long long a = sk[pad(lo)], b = sk[pad(hi)];
          cmp_swap(a, b, (lo & size) == 0);
          sk[pad(lo)] = a;
          sk[pad(hi)] = b;
        }
        __syncthreads();
      } else {
        if (in_smem) {
#pragma unroll
          for (int i = 0; i < E; ++i) key[i] = sk[pad(base + i)];
          __syncthreads();
          in_smem = false;
        }
        if (stride >= E) {
          const int ld = stride / E;  // partner lane distance
          const bool lower = (lane & ld) == 0;
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const unsigned long long o = __shfl_xor_sync(GCR_FULL, key[i], ld);
            const bool asc = ((base + i) & size) == 0;
            const bool keep_small = lower == asc;
            key[i] = keep_small ? (o < key[i] ? o : key[i]) : (o > key[i] ? o : key[i]);
          }
        } else if (stride == 1) {
          reg_stage<E, 1>(key, base, size);
        } else if (stride == 2) {
          reg_stage<E, 2>(key, base, size);
        } else if (stride == 4) {
          reg_stage<E, 4>(key, base, size);
        } else {
          reg_stage<E, 8>(key, base, size);
        }
      }
    }
  }
  if (!in_smem) {
#pragma unroll
    for (int i = 0; i < E; ++i) sk[pad(base + i)] = key[i];
    __syncthreads();
  }
  // coalesced output of the first K ranks
  for (int r = t; r < K; r += T) {
    const unsigned long long k = sk[pad(r)];
    idx_out[(size_t)q * K + r] = (int32_t)(k & 0xffffffffu);
    dist_out[(size_t)q * K + r] = ordered_to_float((uint32_t)(k >> 32));
  }
}

}  // namespace

cudaError_t launch_rank_rows(const float* D, int nq, int ng, int K, int32_t* idx_out, float* dist_out,
                             cudaStream_t st) {
  if (ng > kMaxSeg) return cudaErrorInvalidValue;
  int N = 64;
  while (N < ng) N <<= 1;
  const int E = N >= 512 ? 16 : (N >= 128 ? 4 : 2);
  const int threads = N / E;
  const size_t smem = sizeof(unsigned long long) * (N + N / 32);
  cudaError_t e;
  if (E == 16) {
    e = cudaFuncSetAttribute(rank_rows_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    rank_rows_kernel<16><<<nq, threads, smem, st>>>(D, ng, N, K, idx_out, dist_out);
  } else if (E == 4) {
    rank_rows_kernel<4><<<nq, threads, smem, st>>>(D, ng, N, K, idx_out, dist_out);
  } else {
    rank_rows_kernel<2><<<nq, threads, smem, st>>>(D, ng, N, K, idx_out, dist_out);
  }
  (void)e;
  return cudaGetLastError();
}

}  // namespace gcr
