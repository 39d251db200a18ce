// Row normalisation (S0) and the per-row statistics used by the certified kNN search.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace gcr {

// X_out[i] = X_in[i] / ||X_in[i]|| with the norm and the scaling in FP64, so that each
// output element is the FP32 rounding of the exact quotient (up to one FP64 rounding).
// One warp per row, 16-byte loads.
__global__ void normalize_kernel(const float* __restrict__ X_in, float* __restrict__ X_out,
                                 int64_t n, int d) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float4* src = reinterpret_cast<const float4*>(X_in + row * d);
  float4* dst = reinterpret_cast<float4*>(X_out + row * d);
  const int d4 = d >> 2;
  double ss = 0.0;
  for (int v = lane; v < d4; v += 32) {
    float4 x = src[v];
    ss += (double)x.x * x.x + (double)x.y * x.y + (double)x.z * x.z + (double)x.w * x.w;
  }
  ss = warp_sum_d(ss);
  const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
  for (int v = lane; v < d4; v += 32) {
    float4 x = src[v];
    dst[v] = make_float4((float)(x.x * inv), (float)(x.y * inv), (float)(x.z * inv), (float)(x.w * inv));
  }
}

// n64[i] = ||x_i||^2 in FP64, n32[i] = its FP32 rounding; with xb != NULL also the BF16
// shadow xb = bf16_rn(x), enrm[i] = ||xb_i - x_i|| and anrm[i] = ||xb_i|| (FP64 sums).
__global__ void row_stats_kernel(const float* __restrict__ X, int n, int d, double* __restrict__ n64,
                                 float* __restrict__ n32, __nv_bfloat16* __restrict__ xb,
                                 float* __restrict__ enrm, float* __restrict__ anrm) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float4* src = reinterpret_cast<const float4*>(X + (size_t)row * d);
  const int d4 = d >> 2;
  double ss = 0.0, ee = 0.0, aa = 0.0;
  for (int v = lane; v < d4; v += 32) {
    float4 x = src[v];
    ss += (double)x.x * x.x + (double)x.y * x.y + (double)x.z * x.z + (double)x.w * x.w;
    if (xb) {
      __nv_bfloat16 b0 = __float2bfloat16_rn(x.x), b1 = __float2bfloat16_rn(x.y);
      __nv_bfloat16 b2 = __float2bfloat16_rn(x.z), b3 = __float2bfloat16_rn(x.w);
      __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(xb + (size_t)row * d + 4 * v);
      o[0] = __halves2bfloat162(b0, b1);
      o[1] = __halves2bfloat162(b2, b3);
      double f0 = __bfloat162float(b0), f1 = __bfloat162float(b1);
      double f2 = __bfloat162float(b2), f3 = __bfloat162float(b3);
      double e0 = f0 - x.x, e1 = f1 - x.y, e2 = f2 - x.z, e3 = f3 - x.w;
      ee += e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3;
      aa += f0 * f0 + f1 * f1 + f2 * f2 + f3 * f3;
    }
  }
  ss = warp_sum_d(ss);
  if (xb) {
    ee = warp_sum_d(ee);
    aa = warp_sum_d(aa);
  }
  if (lane == 0) {
    n64[row] = ss;
    n32[row] = (float)ss;
    if (xb) {
      enrm[row] = (float)(sqrt(ee) * (1.0 + 1e-6));
      anrm[row] = (float)(sqrt(aa) * (1.0 + 1e-6));
    }
  }
}

// One block: min / max reductions over the rows.
__global__ void row_scalars_kernel(const double* __restrict__ n64, const float* __restrict__ enrm,
                                   const float* __restrict__ anrm, int n, RowScalars* __restrict__ sc) {
  double nmin = 1e300, nmax = 0.0, emax = 0.0, amax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v = n64[i];
    nmin = fmin(nmin, v);
    nmax = fmax(nmax, v);
    if (enrm) {
      emax = fmax(emax, (double)enrm[i]);
      amax = fmax(amax, (double)anrm[i]);
    }
  }
  __shared__ double s[4][32];
  for (int o = 16; o > 0; o >>= 1) {
    nmin = fmin(nmin, __shfl_xor_sync(GCR_FULL, nmin, o));
    nmax = fmax(nmax, __shfl_xor_sync(GCR_FULL, nmax, o));
    emax = fmax(emax, __shfl_xor_sync(GCR_FULL, emax, o));
    amax = fmax(amax, __shfl_xor_sync(GCR_FULL, amax, o));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { s[0][w] = nmin; s[1][w] = nmax; s[2][w] = emax; s[3][w] = amax; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    nmin = lane < nw ? s[0][lane] : 1e300;
    nmax = lane < nw ? s[1][lane] : 0.0;
    emax = lane < nw ? s[2][lane] : 0.0;
    amax = lane < nw ? s[3][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      nmin = fmin(nmin, __shfl_xor_sync(GCR_FULL, nmin, o));
      nmax = fmax(nmax, __shfl_xor_sync(GCR_FULL, nmax, o));
      emax = fmax(emax, __shfl_xor_sync(GCR_FULL, emax, o));
      amax = fmax(amax, __shfl_xor_sync(GCR_FULL, amax, o));
    }
    if (lane == 0) {
      sc->nmin = nmin;
      sc->nmax = nmax;
      sc->bmax = sqrt(nmax) * (1.0 + 1e-12);
      sc->emax = emax;
      sc->amax = amax;
    }
  }
}

cudaError_t launch_normalize(const float* X_in, float* X_out, int64_t n, int d, cudaStream_t st) {
  const int wpb = 8;
  dim3 grid((unsigned)((n + wpb - 1) / wpb));
  normalize_kernel<<<grid, wpb * 32, 0, st>>>(X_in, X_out, n, d);
  return cudaGetLastError();
}

cudaError_t launch_row_stats(const float* X, int n, int d, double* n64, float* n32,
                             __nv_bfloat16* xb, float* enrm, float* anrm, RowScalars* sc,
                             cudaStream_t st) {
  const int wpb = 8;
  row_stats_kernel<<<(n + wpb - 1) / wpb, wpb * 32, 0, st>>>(X, n, d, n64, n32, xb, enrm, anrm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  row_scalars_kernel<<<1, 1024, 0, st>>>(n64, xb ? enrm : nullptr, xb ? anrm : nullptr, n, sc);
  return cudaGetLastError();
}

}  // namespace gcr
