// One propagation layer (Eq. 2 / Eq. 9) fused with the row L2 normalisation:
//   X_out[i] = normalise( sum_j M_ij X_in[j] )
// M is the CSR operator built by graph.cu. A row is split into S column slices of 128*VW
// floats, one warp per slice (S warps per row, 8/S rows per 256-thread block); each lane keeps
// VW float4 accumulators, so the register footprint stays small and enough warps are resident
// to keep many gathered rows in flight. Every output element is accumulated in FP32 in the
// operator's column order; the squared norm is summed per warp and then over the row's
// slices (in slice order) through shared memory. The operator's row indices and weights are
// read by all slices of the row. Bandwidth-bound: the algorithmic traffic is the operator
// (8 B per entry) + n*d*4 written + the gathered rows.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

// Rows with more operator entries than this (in-degree hubs) are left to propagate_long_kernel,
// which puts a whole block on each of them.
constexpr int kLongRow = 1024;

template <int VW>
__global__ void __launch_bounds__(256) propagate_kernel(const int* __restrict__ rowptr, const int* __restrict__ len,
                                                        const int* __restrict__ col, const float* __restrict__ val,
                                                        const float* __restrict__ X_in, float* __restrict__ X_out,
                                                        int n, int d, int S, const int* __restrict__ order) {
  __shared__ float part[8];
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int rpb = 8 / S;               // rows per block
  const int rb = wb / S, sl = wb % S;  // row within the block, slice within the row
  const int w = blockIdx.x * rpb + rb;
  const int i = w < n ? (order ? order[w] : w) : 0;
  const bool active = w < n && len[i] <= kLongRow;
  const int base = sl * VW * 128 + lane * 4;  // this lane's first float in the row
  float4 acc[VW];
#pragma unroll
  for (int v = 0; v < VW; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (active) {
    const int beg = rowptr[i], L = len[i];
    for (int e0 = 0; e0 < L; e0 += 32) {
      const int e = e0 + lane;
      const int c = e < L ? col[beg + e] : 0;
      const float wt = e < L ? val[beg + e] : 0.f;
      const int m = min(32, L - e0);
      int t = 0;
      // four entries at a time: their slices are all loaded before any is multiplied, so a lane
      // keeps 4 * VW gathers in flight (the layer is bound by the latency of these gathers);
      // each output element still adds the entries in the operator's order
      for (; t + 4 <= m; t += 4) {
        float4 xa[4][VW];
        float wa[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int cu = __shfl_sync(GCR_FULL, c, t + u);
          wa[u] = __shfl_sync(GCR_FULL, wt, t + u);
          const float* ru = X_in + (size_t)cu * d;
#pragma unroll
          for (int v = 0; v < VW; ++v) {
            const int off = base + v * 128;
            xa[u][v] = off < d ? *reinterpret_cast<const float4*>(ru + off) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < VW; ++v) {
            acc[v].x = fmaf(wa[u], xa[u][v].x, acc[v].x); acc[v].y = fmaf(wa[u], xa[u][v].y, acc[v].y);
            acc[v].z = fmaf(wa[u], xa[u][v].z, acc[v].z); acc[v].w = fmaf(wa[u], xa[u][v].w, acc[v].w);
          }
      }
      for (; t + 2 <= m; t += 2) {
        const int c0 = __shfl_sync(GCR_FULL, c, t), c1 = __shfl_sync(GCR_FULL, c, t + 1);
        const float w0 = __shfl_sync(GCR_FULL, wt, t), w1 = __shfl_sync(GCR_FULL, wt, t + 1);
        const float* r0 = X_in + (size_t)c0 * d;
        const float* r1 = X_in + (size_t)c1 * d;
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          const int off = base + v * 128;
          if (off < d) {
            const float4 x0 = *reinterpret_cast<const float4*>(r0 + off);
            const float4 x1 = *reinterpret_cast<const float4*>(r1 + off);
            acc[v].x = fmaf(w0, x0.x, acc[v].x); acc[v].y = fmaf(w0, x0.y, acc[v].y);
            acc[v].z = fmaf(w0, x0.z, acc[v].z); acc[v].w = fmaf(w0, x0.w, acc[v].w);
            acc[v].x = fmaf(w1, x1.x, acc[v].x); acc[v].y = fmaf(w1, x1.y, acc[v].y);
            acc[v].z = fmaf(w1, x1.z, acc[v].z); acc[v].w = fmaf(w1, x1.w, acc[v].w);
          }
        }
      }
      for (; t < m; ++t) {
        const int c0 = __shfl_sync(GCR_FULL, c, t);
        const float w0 = __shfl_sync(GCR_FULL, wt, t);
        const float* r0 = X_in + (size_t)c0 * d;
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          const int off = base + v * 128;
          if (off < d) {
            const float4 x0 = *reinterpret_cast<const float4*>(r0 + off);
            acc[v].x = fmaf(w0, x0.x, acc[v].x); acc[v].y = fmaf(w0, x0.y, acc[v].y);
            acc[v].z = fmaf(w0, x0.z, acc[v].z); acc[v].w = fmaf(w0, x0.w, acc[v].w);
          }
        }
      }
    }
  }
  float ss = 0.f;
#pragma unroll
  for (int v = 0; v < VW; ++v)
    ss += acc[v].x * acc[v].x + acc[v].y * acc[v].y + acc[v].z * acc[v].z + acc[v].w * acc[v].w;
  ss = warp_sum(ss);
  if (lane == 0) part[wb] = ss;
  __syncthreads();
  float tot = 0.f;
  for (int s = 0; s < S; ++s) tot += part[rb * S + s];
  if (!active) return;
  const float inv = tot > 0.f ? 1.0f / sqrtf(tot) : 0.f;
  float* out = X_out + (size_t)i * d;
#pragma unroll
  for (int v = 0; v < VW; ++v) {
    const int off = base + v * 128;
    if (off < d)
      *reinterpret_cast<float4*>(out + off) =
          make_float4(acc[v].x * inv, acc[v].y * inv, acc[v].z * inv, acc[v].w * inv);
  }
}

// Hub rows (more than kLongRow entries), one 1024-thread block per row: the row's entries are
// cut into 32/S contiguous chunks, each chunk accumulated by S warps (one per column slice),
// and the chunk partials are added in chunk order through shared memory, so the result does not
// depend on scheduling. Blocks find the hub rows among their share of row indices.
template <int VW>
__global__ void __launch_bounds__(1024) propagate_long_kernel(const int* __restrict__ rowptr,
                                                              const int* __restrict__ len,
                                                              const int* __restrict__ col,
                                                              const float* __restrict__ val,
                                                              const float* __restrict__ X_in,
                                                              float* __restrict__ X_out, int n, int d, int S) {
  extern __shared__ float4 partial[];  // [32/S groups][S*VW*32] float4
  __shared__ int list[1024];
  __shared__ int nlist;
  __shared__ float red[32];
  const int t = threadIdx.x, lane = t & 31, wb = t >> 5;
  const int G = 32 / S;                // chunk groups
  const int g = wb / S, sl = wb % S;
  const int row_f4 = S * VW * 32;      // float4 per row covered by the slices
  for (int base = blockIdx.x * 1024; base < n; base += gridDim.x * 1024) {
    if (t == 0) nlist = 0;
    __syncthreads();
    const int r = base + t;
    if (r < n && len[r] > kLongRow) list[atomicAdd(&nlist, 1)] = r;
    __syncthreads();
    const int m = nlist;
    for (int q = 0; q < m; ++q) {
      const int i = list[q];
      const int beg = rowptr[i], L = len[i];
      const int per = (L + G - 1) / G;
      const int e_lo = min(L, g * per), e_hi = min(L, e_lo + per);
      float4 acc[VW];
#pragma unroll
      for (int v = 0; v < VW; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
      const int off0 = sl * VW * 128 + lane * 4;
      for (int e0 = e_lo; e0 < e_hi; e0 += 32) {
        const int e = e0 + lane;
        const int c = e < e_hi ? col[beg + e] : 0;
        const float wt = e < e_hi ? val[beg + e] : 0.f;
        const int mm = min(32, e_hi - e0);
        int u = 0;
        for (; u + 2 <= mm; u += 2) {
          const int c0 = __shfl_sync(GCR_FULL, c, u), c1 = __shfl_sync(GCR_FULL, c, u + 1);
          const float w0 = __shfl_sync(GCR_FULL, wt, u), w1 = __shfl_sync(GCR_FULL, wt, u + 1);
          const float* r0 = X_in + (size_t)c0 * d;
          const float* r1 = X_in + (size_t)c1 * d;
#pragma unroll
          for (int v = 0; v < VW; ++v) {
            const int off = off0 + v * 128;
            if (off < d) {
              const float4 x0 = *reinterpret_cast<const float4*>(r0 + off);
              const float4 x1 = *reinterpret_cast<const float4*>(r1 + off);
              acc[v].x = fmaf(w0, x0.x, acc[v].x); acc[v].y = fmaf(w0, x0.y, acc[v].y);
              acc[v].z = fmaf(w0, x0.z, acc[v].z); acc[v].w = fmaf(w0, x0.w, acc[v].w);
              acc[v].x = fmaf(w1, x1.x, acc[v].x); acc[v].y = fmaf(w1, x1.y, acc[v].y);
              acc[v].z = fmaf(w1, x1.z, acc[v].z); acc[v].w = fmaf(w1, x1.w, acc[v].w);
            }
          }
        }
        for (; u < mm; ++u) {
          const int c0 = __shfl_sync(GCR_FULL, c, u);
          const float w0 = __shfl_sync(GCR_FULL, wt, u);
          const float* r0 = X_in + (size_t)c0 * d;
#pragma unroll
          for (int v = 0; v < VW; ++v) {
            const int off = off0 + v * 128;
            if (off < d) {
              const float4 x0 = *reinterpret_cast<const float4*>(r0 + off);
              acc[v].x = fmaf(w0, x0.x, acc[v].x); acc[v].y = fmaf(w0, x0.y, acc[v].y);
              acc[v].z = fmaf(w0, x0.z, acc[v].z); acc[v].w = fmaf(w0, x0.w, acc[v].w);
            }
          }
        }
      }
#pragma unroll
      for (int v = 0; v < VW; ++v) partial[g * row_f4 + sl * VW * 32 + v * 32 + lane] = acc[v];
      __syncthreads();
      // a lane's accumulator v of slice sl holds float4 sl*VW*32 + v*32 + lane of the row, which
      // is where it was stored: thread t adds up float4 t over the groups in order
      float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
      const int d4 = d >> 2;
      if (t < d4) {
        for (int gg = 0; gg < G; ++gg) {
          const float4 z = partial[gg * row_f4 + t];
          y.x += z.x; y.y += z.y; y.z += z.z; y.w += z.w;
        }
      }
      float ss = y.x * y.x + y.y * y.y + y.z * y.z + y.w * y.w;
      ss = warp_sum(ss);
      if (lane == 0) red[wb] = ss;
      __syncthreads();
      float tot = 0.f;
      for (int k = 0; k < 32; ++k) tot += red[k];
      const float inv = tot > 0.f ? 1.0f / sqrtf(tot) : 0.f;
      if (t < d4)
        reinterpret_cast<float4*>(X_out + (size_t)i * d)[t] = make_float4(y.x * inv, y.y * inv, y.z * inv, y.w * inv);
      __syncthreads();
    }
  }
}

}  // namespace

cudaError_t launch_propagate(const int* rowptr, const int* len, const int* col, const float* val,
                             const float* X_in, float* X_out, int n, int d, const int* order, cudaStream_t st) {
  const int v128 = (d + 127) / 128;  // 128-float units of a row
  if (v128 > 32) return cudaErrorInvalidValue;
  // up to 4 units per warp; the row's slices (1, 2, 4 or 8 warps) divide the 8 warps of a block
  int VW = v128 <= 1 ? 1 : (v128 <= 2 ? 2 : 4);
  int S = 1;
  while (S * VW < v128) S <<= 1;
  dim3 grid((unsigned)((n + (8 / S) - 1) / (8 / S)));
  if (VW == 1) propagate_kernel<1><<<grid, 256, 0, st>>>(rowptr, len, col, val, X_in, X_out, n, d, S, order);
  else if (VW == 2) propagate_kernel<2><<<grid, 256, 0, st>>>(rowptr, len, col, val, X_in, X_out, n, d, S, order);
  else propagate_kernel<4><<<grid, 256, 0, st>>>(rowptr, len, col, val, X_in, X_out, n, d, S, order);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // hub rows: 32 warps per row (S slices x 32/S chunk groups), partials in shared memory
  const size_t smem = (size_t)32 * VW * 32 * sizeof(float4);
  const dim3 lgrid((unsigned)std::max(1, std::min(152, (n + 1023) / 1024)));
  if (VW == 1) {
    propagate_long_kernel<1><<<lgrid, 1024, smem, st>>>(rowptr, len, col, val, X_in, X_out, n, d, S);
  } else if (VW == 2) {
    propagate_long_kernel<2><<<lgrid, 1024, smem, st>>>(rowptr, len, col, val, X_in, X_out, n, d, S);
  } else {
    e = cudaFuncSetAttribute(propagate_long_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    propagate_long_kernel<4><<<lgrid, 1024, smem, st>>>(rowptr, len, col, val, X_in, X_out, n, d, S);
  }
  return cudaGetLastError();
}

}  // namespace gcr
