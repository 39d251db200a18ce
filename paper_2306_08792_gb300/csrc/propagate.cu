// One propagation layer (Eq. 2 / Eq. 9) fused with the row L2 normalisation:
//   X_out[i] = normalise( sum_j M_ij X_in[j] )
// M is the CSR operator built by graph.cu. One warp per row; each lane owns a d/32 slice of
// the output in registers (16-byte loads, FP32 accumulation in the operator's column order),
// so X_in is read once per operator entry and X_out written once. Bandwidth-bound: the
// algorithmic traffic is the operator (8 B per entry) + n*d*4 written + the gathered rows.
#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

template <int VPL>
__global__ void __launch_bounds__(256) propagate_kernel(const int* __restrict__ rowptr, const int* __restrict__ len,
                                                        const int* __restrict__ col, const float* __restrict__ val,
                                                        const float* __restrict__ X_in, float* __restrict__ X_out,
                                                        int n, int d, const int* __restrict__ order) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= n) return;
  const int i = order ? order[w] : w;
  float4 acc[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int beg = rowptr[i], L = len[i];
  for (int e0 = 0; e0 < L; e0 += 32) {
    const int e = e0 + lane;
    const int c = e < L ? col[beg + e] : 0;
    const float w = e < L ? val[beg + e] : 0.f;
    const int m = min(32, L - e0);
    int t = 0;
    for (; t + 2 <= m; t += 2) {
      const int c0 = __shfl_sync(GCR_FULL, c, t), c1 = __shfl_sync(GCR_FULL, c, t + 1);
      const float w0 = __shfl_sync(GCR_FULL, w, t), w1 = __shfl_sync(GCR_FULL, w, t + 1);
      const float* r0 = X_in + (size_t)c0 * d;
      const float* r1 = X_in + (size_t)c1 * d;
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int off = v * 128 + lane * 4;
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
      const float w0 = __shfl_sync(GCR_FULL, w, t);
      const float* r0 = X_in + (size_t)c0 * d;
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int off = v * 128 + lane * 4;
        if (off < d) {
          const float4 x0 = *reinterpret_cast<const float4*>(r0 + off);
          acc[v].x = fmaf(w0, x0.x, acc[v].x); acc[v].y = fmaf(w0, x0.y, acc[v].y);
          acc[v].z = fmaf(w0, x0.z, acc[v].z); acc[v].w = fmaf(w0, x0.w, acc[v].w);
        }
      }
    }
  }
  float ss = 0.f;
#pragma unroll
  for (int v = 0; v < VPL; ++v)
    ss += acc[v].x * acc[v].x + acc[v].y * acc[v].y + acc[v].z * acc[v].z + acc[v].w * acc[v].w;
  ss = warp_sum(ss);
  const float inv = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
  float* out = X_out + (size_t)i * d;
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int off = v * 128 + lane * 4;
    if (off < d)
      *reinterpret_cast<float4*>(out + off) =
          make_float4(acc[v].x * inv, acc[v].y * inv, acc[v].z * inv, acc[v].w * inv);
  }
}

}  // namespace

cudaError_t launch_propagate(const int* rowptr, const int* len, const int* col, const float* val,
                             const float* X_in, float* X_out, int n, int d, const int* order, cudaStream_t st) {
  dim3 grid((n + 7) / 8);
  const int vpl = (d + 127) / 128;
  if (vpl <= 1) propagate_kernel<1><<<grid, 256, 0, st>>>(rowptr, len, col, val, X_in, X_out, n, d, order);
  else if (vpl <= 2) propagate_kernel<2><<<grid, 256, 0, st>>>(rowptr, len, col, val, X_in, X_out, n, d, order);
  else if (vpl <= 4) propagate_kernel<4><<<grid, 256, 0, st>>>(rowptr, len, col, val, X_in, X_out, n, d, order);
  else if (vpl <= 8) propagate_kernel<8><<<grid, 256, 0, st>>>(rowptr, len, col, val, X_in, X_out, n, d, order);
  else if (vpl <= 16) propagate_kernel<16><<<grid, 256, 0, st>>>(rowptr, len, col, val, X_in, X_out, n, d, order);
  else if (vpl <= 32) propagate_kernel<32><<<grid, 256, 0, st>>>(rowptr, len, col, val, X_in, X_out, n, d, order);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace gcr
