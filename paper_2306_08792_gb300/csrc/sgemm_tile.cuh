// 128 x 128 FP32 tile product on CUDA cores, shared by the similarity GEMM (sgemm.cu)
// and the GCRV Gram / solver products (gcrv.cu).
//
// acc = A_tile . B_tile^T with A, B row-major along K (K contiguous), 256 threads, 8 x 8
// outputs per thread, BK = 8 slices double-buffered through shared memory. Each output is
// one sequential FMA chain over K, which fixes its error bound: gamma_K * sum |a_k b_k|.
#pragma once
#include "common.cuh"

namespace gcr {
namespace simt {

constexpr int BM = 128, BN = 128, BK = 8, PITCH = 132, SP = BN + 1;

struct TileSmem {
  float As[2][BK][PITCH];
  float Bs[2][BK][PITCH];
};

// Loads the BK-slice [k0, k0+8) of 128 rows into registers (one float4 per thread).
__device__ __forceinline__ float4 load_slice(const float* __restrict__ base, int nrows, int d,
                                             int k0, int tid, const int* __restrict__ rowmap) {
  int r = tid >> 1;
  int kk = k0 + ((tid & 1) << 2);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (r < nrows && kk < d) {
    size_t row = rowmap ? (size_t)rowmap[r] : (size_t)r;
    v = *reinterpret_cast<const float4*>(base + row * (size_t)d + kk);
  }
  return v;
}

__device__ __forceinline__ void store_slice(float (*S)[PITCH], float4 v, int tid) {
  int r = tid >> 1;
  int kk = (tid & 1) << 2;
  S[kk + 0][r] = v.x;
  S[kk + 1][r] = v.y;
  S[kk + 2][r] = v.z;
  S[kk + 3][r] = v.w;
}

// acc[i][j] = sum_k A[row_i][k] * B[col_j][k]; rows i = ty*4 + (i&3) + 64*(i>>2), cols alike.
// A rows: abase[(rowmap ? rowmap[r] : r)], r < arows; B rows: bbase[c], c < brows.
__device__ __forceinline__ void tile_mma(TileSmem& sm, const float* __restrict__ abase, int arows,
                                         const int* __restrict__ rowmap,
                                         const float* __restrict__ bbase, int brows, int d,
                                         float acc[8][8]) {
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float4 ra = load_slice(abase, arows, d, 0, tid, rowmap);
  float4 rb = load_slice(bbase, brows, d, 0, tid, nullptr);
  __syncthreads();  // previous users of the staging buffers are done
  store_slice(sm.As[0], ra, tid);
  store_slice(sm.Bs[0], rb, tid);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < d; k0 += BK) {
    const bool more = k0 + BK < d;
    if (more) {
      ra = load_slice(abase, arows, d, k0 + BK, tid, rowmap);
      rb = load_slice(bbase, brows, d, k0 + BK, tid, nullptr);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&sm.As[buf][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&sm.As[buf][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&sm.Bs[buf][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&sm.Bs[buf][kk][64 + tx * 4]);
      float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store_slice(sm.As[buf ^ 1], ra, tid);
      store_slice(sm.Bs[buf ^ 1], rb, tid);
      __syncthreads();
      buf ^= 1;
    }
  }
}

__device__ __forceinline__ int acc_row(int ty, int i) { return ty * 4 + (i & 3) + ((i >> 2) << 6); }
__device__ __forceinline__ int acc_col(int tx, int j) { return tx * 4 + (j & 3) + ((j >> 2) << 6); }


}  // namespace simt
}  // namespace gcr
