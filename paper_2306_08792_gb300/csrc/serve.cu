// Re-ranking against a resident gallery (serving form of GCR, Sec. IV-F2: the gallery's graphs
// are computed and stored in advance).
//
// The gallery state holds the layers G_0..G_T of offline GCR on the gallery alone and, per
// layer t < T, the degrees of that layer's gallery graph. A batch of queries then runs, for
// t = 1..T, the certified kNN search against G_{t-1} (column-split streaming pools, merged),
// and one row of the operator per query with the gallery frozen and no query-query edges:
//   symmetric (Eq. 7): y = x_q / D_q + sum_j (w_qj / 2) g_j / sqrt(D_q D_j),
//                      D_q = (1 + sum_j w_qj + 1) / 2
//   asymmetric (Eq. 6): y = x_q / sqrt(r_q) + sum_j w_qj g_j / sqrt(r_q Dc_j), r_q = 1 + sum w
// x_q <- normalise(y); finally the certified top-K of the gallery on G_T. Every step is per
// query row, so a query's result does not depend on the other queries of its batch.
#include "common.cuh"
#include "kernels.h"
#include "pool.cuh"

namespace gcr {
namespace {

// Merges the sorted list held by a warp (b, bi: KP entries, entry p*32 + lane) with the sorted
// KP-entry list at (lv, li) (shared or global memory), keeping the KP best. Chunks of a sorted
// list are sorted, so the merge stops at the first chunk whose best cannot enter.
template <int KP>
__device__ __forceinline__ void merge_list(float (&b)[KP / 32], int (&bi)[KP / 32], const float* lv, const int* li,
                                           int lane) {
  constexpr int P = KP / 32;
#pragma unroll
  for (int c = 0; c < P; ++c) {
    float a = lv[c * 32 + lane];
    int ai = li[c * 32 + lane];
    const float worst = __shfl_sync(GCR_FULL, b[P - 1], 31);
    const int worst_i = __shfl_sync(GCR_FULL, bi[P - 1], 31);
    const float best = __shfl_sync(GCR_FULL, a, 0);
    const int best_i = __shfl_sync(GCR_FULL, ai, 0);
    if (!better(best, best_i, worst, worst_i)) break;
    const float ar = __shfl_sync(GCR_FULL, a, 31 - lane);
    const int ari = __shfl_sync(GCR_FULL, ai, 31 - lane);
    if (better(ar, ari, b[P - 1], bi[P - 1])) { b[P - 1] = ar; bi[P - 1] = ari; }
#pragma unroll
    for (int stride = KP / 2; stride >= 32; stride >>= 1) {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int q2 = p ^ (stride >> 5);
        if (q2 > p && better(b[q2], bi[q2], b[p], bi[p])) {
          float tv = b[p]; b[p] = b[q2]; b[q2] = tv;
          int ti = bi[p]; bi[p] = bi[q2]; bi[q2] = ti;
        }
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) warp_merge32_desc(b[p], bi[p], lane);
  }
}

// Merge S sorted pools per (kind, row) into one: pools [S][kinds][na][KP] -> [kinds][na][KP].
// One block of 8 warps per (kind, row): warp w merges splits w, w + 8, ..., then warp 0 merges
// the 8 partial lists (the strict order makes the result independent of the merge order).
template <int KP>
__global__ void __launch_bounds__(256) merge_splits_kernel(const float* __restrict__ pv, const int* __restrict__ pi,
                                                           int S, int kinds, int na, float* __restrict__ ov,
                                                           int* __restrict__ oi) {
  constexpr int P = KP / 32;
  __shared__ float sv[8][KP];
  __shared__ int si[8][KP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long w = blockIdx.x;  // (kind, row)
  float b[P];
  int bi[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const bool has = warp < S;
    b[p] = has ? pv[((size_t)warp * kinds * na + w) * KP + p * 32 + lane] : -CUDART_INF_F;
    bi[p] = has ? pi[((size_t)warp * kinds * na + w) * KP + p * 32 + lane] : -1;
  }
  for (int s = warp + 8; s < S; s += 8) {
    const size_t base = ((size_t)s * kinds * na + w) * KP;
    merge_list<KP>(b, bi, pv + base, pi + base, lane);
  }
#pragma unroll
  for (int p = 0; p < P; ++p) {
    sv[warp][p * 32 + lane] = b[p];
    si[warp][p * 32 + lane] = bi[p];
  }
  __syncthreads();
  if (warp != 0) return;
  for (int v = 1; v < 8 && v < S; ++v) merge_list<KP>(b, bi, sv[v], si[v], lane);
#pragma unroll
  for (int p = 0; p < P; ++p) {
    ov[w * KP + p * 32 + lane] = b[p];
    oi[w * KP + p * 32 + lane] = bi[p];
  }
}

// One warp per query: the query's row of the operator against the frozen layer, normalised.
template <int VPL>
__global__ void __launch_bounds__(256) query_step_kernel(const float* __restrict__ xq, int b, int d,
                                                         const float* __restrict__ G, const float* __restrict__ deg,
                                                         const int32_t* __restrict__ nbr,
                                                         const float* __restrict__ d2, int k, float gamma,
                                                         int symmetric, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (q >= b) return;
  float wsum = 0.f;
  for (int s = 0; s < k; ++s) {
    const int j = nbr[(size_t)q * k + s];
    if (j >= 0) wsum += expf(-d2[(size_t)q * k + s] / gamma);
  }
  const float Dq = symmetric ? 0.5f * (1.f + wsum + 1.f) : 1.f + wsum;
  const float cself = symmetric ? 1.f / Dq : 1.f / sqrtf(Dq);
  float4 acc[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int off = v * 128 + lane * 4;
    acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (off < d) {
      const float4 x = *reinterpret_cast<const float4*>(xq + (size_t)q * d + off);
      acc[v] = make_float4(cself * x.x, cself * x.y, cself * x.z, cself * x.w);
    }
  }
  for (int s = 0; s < k; ++s) {
    const int j = nbr[(size_t)q * k + s];
    if (j < 0) continue;
    const float w = expf(-d2[(size_t)q * k + s] / gamma);
    const float c = symmetric ? 0.5f * w / sqrtf(Dq * deg[j]) : w / sqrtf(Dq * deg[j]);
    const float* g = G + (size_t)j * d;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      const int off = v * 128 + lane * 4;
      if (off < d) {
        const float4 y = *reinterpret_cast<const float4*>(g + off);
        acc[v].x = fmaf(c, y.x, acc[v].x); acc[v].y = fmaf(c, y.y, acc[v].y);
        acc[v].z = fmaf(c, y.z, acc[v].z); acc[v].w = fmaf(c, y.w, acc[v].w);
      }
    }
  }
  float ss = 0.f;
#pragma unroll
  for (int v = 0; v < VPL; ++v)
    ss += acc[v].x * acc[v].x + acc[v].y * acc[v].y + acc[v].z * acc[v].z + acc[v].w * acc[v].w;
  ss = warp_sum(ss);
  const float inv = ss > 0.f ? 1.f / sqrtf(ss) : 0.f;
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int off = v * 128 + lane * 4;
    if (off < d)
      *reinterpret_cast<float4*>(out + (size_t)q * d + off) =
          make_float4(acc[v].x * inv, acc[v].y * inv, acc[v].z * inv, acc[v].w * inv);
  }
}

// Symmetric degree D = (D_r + D_c) / 2, or D_c for the asymmetric operator.
__global__ void layer_degree_kernel(const float* __restrict__ dr, const float* __restrict__ dc, int n, int symmetric,
                                    float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = symmetric ? 0.5f * (dr[i] + dc[i]) : dc[i];
}

}  // namespace

cudaError_t launch_merge_splits(const float* pv, const int* pi, int S, int kinds, int na, int kp, float* ov, int* oi,
                                cudaStream_t st) {
  dim3 grid((unsigned)((long)kinds * na));  // one block per (kind, row)
  if (kp == 32) merge_splits_kernel<32><<<grid, 256, 0, st>>>(pv, pi, S, kinds, na, ov, oi);
  else if (kp == 64) merge_splits_kernel<64><<<grid, 256, 0, st>>>(pv, pi, S, kinds, na, ov, oi);
  else if (kp == 128) merge_splits_kernel<128><<<grid, 256, 0, st>>>(pv, pi, S, kinds, na, ov, oi);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_query_step(const float* xq, int b, int d, const float* G, const float* deg, const int32_t* nbr,
                              const float* d2, int k, float gamma, int symmetric, float* out, cudaStream_t st) {
  dim3 grid((b + 7) / 8);
  const int vpl = (d + 127) / 128;
  if (vpl <= 1) query_step_kernel<1><<<grid, 256, 0, st>>>(xq, b, d, G, deg, nbr, d2, k, gamma, symmetric, out);
  else if (vpl <= 2) query_step_kernel<2><<<grid, 256, 0, st>>>(xq, b, d, G, deg, nbr, d2, k, gamma, symmetric, out);
  else if (vpl <= 4) query_step_kernel<4><<<grid, 256, 0, st>>>(xq, b, d, G, deg, nbr, d2, k, gamma, symmetric, out);
  else if (vpl <= 8) query_step_kernel<8><<<grid, 256, 0, st>>>(xq, b, d, G, deg, nbr, d2, k, gamma, symmetric, out);
  else if (vpl <= 16) query_step_kernel<16><<<grid, 256, 0, st>>>(xq, b, d, G, deg, nbr, d2, k, gamma, symmetric, out);
  else if (vpl <= 32) query_step_kernel<32><<<grid, 256, 0, st>>>(xq, b, d, G, deg, nbr, d2, k, gamma, symmetric, out);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_layer_degree(const float* dr, const float* dc, int n, int symmetric, float* out, cudaStream_t st) {
  layer_degree_kernel<<<(n + 255) / 256, 256, 0, st>>>(dr, dc, n, symmetric, out);
  return cudaGetLastError();
}

}  // namespace gcr
