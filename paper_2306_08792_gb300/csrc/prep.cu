// Row normalisation (S0) and the per-row statistics used by the certified kNN search.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gcr {

// X_out[i] = X_in[i] / ||X_in[i]||: the squared norm is accumulated exactly (float-float,
// combined in FP64 once per row) and 1/||x|| is formed in FP64, so each output element is the
// FP32 rounding of x * fl32(1/||x||), within one ulp of the exact quotient. One warp per row.
__global__ void normalize_kernel(const float* __restrict__ X_in, float* __restrict__ X_out,
                                 int64_t n, int d) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float4* src = reinterpret_cast<const float4*>(X_in + row * d);
  float4* dst = reinterpret_cast<float4*>(X_out + row * d);
  const int d4 = d >> 2;
  FF acc;
  for (int v = lane; v < d4; v += 32) {
    float4 x = src[v];
    acc.add_sq(x.x); acc.add_sq(x.y); acc.add_sq(x.z); acc.add_sq(x.w);
  }
  const double ss = warp_sum_d(acc.value());
  const float inv = ss > 0.0 ? (float)(1.0 / sqrt(ss)) : 0.f;
  for (int v = lane; v < d4; v += 32) {
    float4 x = src[v];
    dst[v] = make_float4(x.x * inv, x.y * inv, x.z * inv, x.w * inv);
  }
}

// n64[i] = ||x_i||^2 (float-float accumulation, combined in FP64), n32[i] = its FP32 rounding;
// with xr != NULL also the rounded operand copy xr = round(x) (BF16 round-to-nearest-even, or
// TF32 as above, held as FP32), enrm[i] >= ||round(x_i) - x_i|| and anrm[i] >= ||round(x_i)||
// (FP32 sums rounded up by a relative margin that covers their own accumulation error: at most
// (d/32 + 5) * 2^-24 < 1e-3 for d <= 4096). Each difference round(x) - x is exact in FP32.
// The min / max of those over the rows go to sc: every value is non-negative, so the bit
// patterns of the doubles order like the values and 64-bit integer atomics reduce them (sc is
// set to the neutral values by row_scalars_init_kernel first). One warp per row, rows strided
// over the grid so that each block folds many rows before its four atomics.
__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

__global__ void row_scalars_init_kernel(RowScalars* __restrict__ sc) {
  sc->nmin = 1e300;
  sc->nmax = 0.0;
  sc->emax = 0.0;
  sc->amax = 0.0;
}

template <Elt E>
__global__ void __launch_bounds__(256) row_stats_kernel(const float* __restrict__ X, int n, int d,
                                                        double* __restrict__ n64, float* __restrict__ n32,
                                                        void* __restrict__ xr, float* __restrict__ enrm,
                                                        float* __restrict__ anrm, RowScalars* __restrict__ sc) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int d4 = d >> 2;
  double nmin = 1e300, nmax = 0.0, emax = 0.0, amax = 0.0;
  for (int row = blockIdx.x * 8 + wib; row < n; row += gridDim.x * 8) {
    const float4* src = reinterpret_cast<const float4*>(X + (size_t)row * d);
    FF acc;
    float ee = 0.f, aa = 0.f;
    for (int v = lane; v < d4; v += 32) {
      float4 x = src[v];
      acc.add_sq(x.x); acc.add_sq(x.y); acc.add_sq(x.z); acc.add_sq(x.w);
      if (xr) {
        float f0, f1, f2, f3;
        if constexpr (E == Elt::BF16) {
          __nv_bfloat16 b0 = __float2bfloat16_rn(x.x), b1 = __float2bfloat16_rn(x.y);
          __nv_bfloat16 b2 = __float2bfloat16_rn(x.z), b3 = __float2bfloat16_rn(x.w);
          __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(xr) + (size_t)row * d + 4 * v);
          o[0] = __halves2bfloat162(b0, b1);
          o[1] = __halves2bfloat162(b2, b3);
          f0 = __bfloat162float(b0); f1 = __bfloat162float(b1);
          f2 = __bfloat162float(b2); f3 = __bfloat162float(b3);
        } else {
          f0 = round_tf32(x.x); f1 = round_tf32(x.y);
          f2 = round_tf32(x.z); f3 = round_tf32(x.w);
          reinterpret_cast<float4*>(static_cast<float*>(xr) + (size_t)row * d)[v] = make_float4(f0, f1, f2, f3);
        }
        const float e0 = f0 - x.x, e1 = f1 - x.y, e2 = f2 - x.z, e3 = f3 - x.w;  // exact differences
        ee = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, ee))));
        aa = fmaf(f0, f0, fmaf(f1, f1, fmaf(f2, f2, fmaf(f3, f3, aa))));
      }
    }
    const double ss = warp_sum_d(acc.value());
    nmin = fmin(nmin, ss);
    nmax = fmax(nmax, ss);
    if (xr) {
      const float en = sqrtf(warp_sum(ee) * 1.002f) * 1.0001f;
      const float an = sqrtf(warp_sum(aa) * 1.002f) * 1.0001f;
      emax = fmax(emax, (double)en);
      amax = fmax(amax, (double)an);
      if (lane == 0) {
        enrm[row] = en;
        anrm[row] = an;
      }
    }
    if (lane == 0) {
      n64[row] = ss;
      n32[row] = (float)ss;
    }
  }
  // every lane holds its warp's values; fold the block's warps, then one atomic per scalar
  __shared__ double s[4][8];
  if (lane == 0) { s[0][wib] = nmin; s[1][wib] = nmax; s[2][wib] = emax; s[3][wib] = amax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) {
      nmin = fmin(nmin, s[0][w]);
      nmax = fmax(nmax, s[1][w]);
      emax = fmax(emax, s[2][w]);
      amax = fmax(amax, s[3][w]);
    }
    if (nmin < 1e300) atomicMin(reinterpret_cast<unsigned long long*>(&sc->nmin), dbits(nmin));
    atomicMax(reinterpret_cast<unsigned long long*>(&sc->nmax), dbits(nmax));
    if (xr) {
      atomicMax(reinterpret_cast<unsigned long long*>(&sc->emax), dbits(emax));
      atomicMax(reinterpret_cast<unsigned long long*>(&sc->amax), dbits(amax));
    }
  }
}

// Compensated BF16 operands for the re-ranked distances: x = hi + e exactly (e in FP32),
// hi = bf16(x), lo = bf16(e). Queries become [hi | hi | lo], gallery rows [hi | lo | hi], so
// one BF16 product over 3d terms gives hi.hi' + hi.lo' + lo.hi', whose error against x.x'
// is <= ||x|| ||e'-lo'|| + ||e-lo|| ||x'|| + ||e|| ||e'|| + accumulation <= ~3 * 2^-16 for
// unit rows (instead of ~2^-7 for hi.hi' alone).
__global__ void split3_kernel(const float* __restrict__ X, int n, int d, int gallery_order,
                              __nv_bfloat16* __restrict__ out) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)n * d) return;
  const long row = t / d, c = t % d;
  const float x = X[t];
  const __nv_bfloat16 hi = __float2bfloat16_rn(x);
  const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
  __nv_bfloat16* o = out + row * 3 * d;
  o[c] = hi;
  o[d + c] = gallery_order ? lo : hi;
  o[2 * d + c] = gallery_order ? hi : lo;
}

cudaError_t launch_split3(const float* X, int n, int d, int gallery_order, __nv_bfloat16* out, cudaStream_t st) {
  const long total = (long)n * d;
  split3_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(X, n, d, gallery_order, out);
  return cudaGetLastError();
}

cudaError_t launch_normalize(const float* X_in, float* X_out, int64_t n, int d, cudaStream_t st) {
  const int wpb = 8;
  dim3 grid((unsigned)((n + wpb - 1) / wpb));
  normalize_kernel<<<grid, wpb * 32, 0, st>>>(X_in, X_out, n, d);
  return cudaGetLastError();
}

cudaError_t launch_row_stats(const float* X, int n, int d, double* n64, float* n32,
                             void* xr, Elt elt, float* enrm, float* anrm, RowScalars* sc,
                             cudaStream_t st) {
  row_scalars_init_kernel<<<1, 1, 0, st>>>(sc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // 8 rows per block per pass; one wave of 6 blocks (40 registers a thread) on each of the 152 SMs
  const int blocks = std::max(1, std::min((n + 7) / 8, 152 * 6));
  if (elt == Elt::TF32)
    row_stats_kernel<Elt::TF32><<<blocks, 256, 0, st>>>(X, n, d, n64, n32, xr, enrm, anrm, sc);
  else
    row_stats_kernel<Elt::BF16><<<blocks, 256, 0, st>>>(X, n, d, n64, n32, xr, enrm, anrm, sc);
  return cudaGetLastError();
}

}  // namespace gcr
