// Segmented sort of the re-ranked distances (one segment per query).
//
// Each query's gallery distances become 64-bit keys (order-preserving bits of the FP32
// distance, gallery index) so that one ascending sort yields the ranking with ties broken
// by the smaller gallery index. One CTA per query sorts its whole segment in shared memory
// (bitonic network, up to 16384 keys = 128 KB) and writes the first K entries.
#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

constexpr int kMaxSeg = 16384;

__global__ void __launch_bounds__(1024) rank_rows_kernel(const float* __restrict__ D, int ng, int N, int K,
                                                          int32_t* __restrict__ idx_out, float* __restrict__ dist_out) {
  extern __shared__ unsigned long long keys[];
  const int q = blockIdx.x;
  const float* row = D + (size_t)q * ng;
  for (int e = threadIdx.x; e < N; e += blockDim.x)
    keys[e] = e < ng ? (((unsigned long long)float_to_ordered(row[e]) << 32) | (unsigned)e) : ~0ull;
  __syncthreads();
  for (int size = 2; size <= N; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (N >> 1); t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const unsigned long long a = keys[lo], b = keys[hi];
        if ((a > b) == asc) { keys[lo] = b; keys[hi] = a; }
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < K; r += blockDim.x) {
    const unsigned long long k = keys[r];
    idx_out[(size_t)q * K + r] = (int32_t)(k & 0xffffffffu);
    dist_out[(size_t)q * K + r] = ordered_to_float((uint32_t)(k >> 32));
  }
}

}  // namespace

cudaError_t launch_rank_rows(const float* D, int nq, int ng, int K, int32_t* idx_out,
                             float* dist_out, cudaStream_t st) {
  if (ng > kMaxSeg) return cudaErrorInvalidValue;
  int N = 2;
  while (N < ng) N <<= 1;
  const size_t smem = sizeof(unsigned long long) * N;
  cudaError_t e = cudaFuncSetAttribute(rank_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = N >= 2048 ? 1024 : (N / 2 < 32 ? 32 : N / 2);
  rank_rows_kernel<<<nq, threads, smem, st>>>(D, ng, N, K, idx_out, dist_out);
  return cudaGetLastError();
}

}  // namespace gcr
