// DSFP: decentralized and synchronous feature propagation (Algorithm 1, Sec. III-B).
//
// For image i the local node set is L = {i} u N_i (m = 1 + |N_i| <= kDsfpMaxK + 1 nodes,
// local index 0 is i). Algorithm 1 builds the symmetric local similarity matrix
// A_uv = exp(-||x_u - x_v||^2 / gamma) over every pair of L, its degrees D_u = sum_v A_uv,
// M = D^{-1/2} A D^{-1/2}, and iterates X_{t+1} = M X_t on the m x d local features (each
// iteration followed by the row L2 normalisation, as in the global method). The output for
// image i is its own row of X_T.
//
// Every local row stays a combination of the input rows: X_t = P_t X_0 with P_t an m x m
// matrix, so the iterations run in the m x m space:
//   Y = M P_t,  ||row u of Y X_0||^2 = (Y G Y^T)_uu with G = X_0 X_0^T (the local Gram),
//   P_{t+1} = diag(1 / ||row u||) Y.
// G is also all that A needs (||x_u - x_v||^2 = G_uu + G_vv - 2 G_uv). So one CTA per image
// computes G over d in staged column chunks (the only pass over the m rows besides the
// output), runs the small recurrence, and writes sum_v Y_0v x_v / ||.|| for the last
// iteration's Y, the norm again from G. FP32 throughout; the Gram and the output are plain
// FP32 dot products.
// A chunk is staged row-major (a straight float4 copy); each Gram job (a pair of kTl-row tiles
// and a group of column quads) reads kTl + kTl float4 per quad for its 4 kTl^2 products.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

constexpr int kDsfpThreads = 128;
constexpr int kCh = 128;   // columns per staged chunk
// Gram register tile (kTl x kTl entries per thread and job). 3 x 3 (m = 21 needs no padding
// rows, 28 tile pairs keep 112 of the 128 threads busy) measured 1.78 ms against 1.95 ms for
// 4 x 4 (24 padded rows, 21 tile pairs, 84 busy threads) on 19,281 images of d = 2048.
constexpr int kTl = 3;
constexpr int kTT = kTl * kTl;
constexpr int kMaxGroups = 4;   // column-quad groups per tile pair (measured: 4 beats 6 and 8)

struct DsfpLayout {
  int mp;      // m rounded up to kTl (rows of the staged chunk)
  int cs;      // row stride of the chunk, kCh + 4 (float4-aligned, staggers the banks)
  int tiles;   // mp / kTl
  int tp;      // tile pairs (a <= b)
  int groups;  // column-quad groups per tile pair (<= kMaxGroups)
  int jobs;    // tp * groups (<= 2 * kDsfpThreads)
  size_t chunk_off, parts_off, mat_off, bytes;
};

__host__ __device__ inline DsfpLayout dsfp_layout(int m_max) {
  DsfpLayout L;
  L.mp = (m_max + kTl - 1) / kTl * kTl;
  L.cs = kCh + 4;
  L.tiles = L.mp / kTl;
  L.tp = L.tiles * (L.tiles + 1) / 2;
  // column-quad groups: as many as one job per thread allows (two jobs per thread past 128
  // tile pairs). Consecutive lanes take consecutive quads of the same tile pair, so a warp's
  // float4 reads mostly hit distinct banks (lanes on different 4-row tiles would alias: tiles
  // are 528 floats apart)
  L.groups = L.tp >= kDsfpThreads ? 1 : (kDsfpThreads / L.tp < kMaxGroups ? kDsfpThreads / L.tp : kMaxGroups);
  L.jobs = L.tp * L.groups;
  L.chunk_off = 0;
  L.parts_off = L.chunk_off + sizeof(float) * (size_t)2 * L.mp * L.cs;  // two chunk buffers
  L.mat_off = L.parts_off + sizeof(float) * (size_t)L.jobs * kTl * kTl;
  // G, M, P, Y (each mp x mp), then the row norms and degrees
  L.bytes = L.mat_off + sizeof(float) * ((size_t)4 * L.mp * L.mp + 2 * L.mp);
  return L;
}

// Asynchronous 16-byte global -> shared copy (zero-fill when !valid; src must still be a
// valid address), its group commit and wait.
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Copies columns [c0, c0 + kCh) of the local rows into a chunk buffer (rows >= m and columns
// >= d read as zero).
__device__ __forceinline__ void stage_chunk(float* buf, const float* __restrict__ X, const int* loc, int m, int mp,
                                            int cs, int d, int c0) {
  for (int e = threadIdx.x; e < mp * (kCh / 4); e += kDsfpThreads) {
    const int r = e / (kCh / 4), c4 = (e % (kCh / 4)) * 4;
    const bool ok = r < m && c0 + c4 < d;  // d % 4 == 0: a quad is wholly in or out
    cp_async16(buf + r * cs + c4, ok ? X + (size_t)loc[r] * d + c0 + c4 : X, ok);
  }
}

// grid = n CTAs (one per image), kDsfpThreads threads, dynamic shared memory = layout.bytes.
// Both passes over the local rows (the Gram, then the output row) stream column chunks
// through two buffers: chunk c + 1 is in flight while chunk c is used.
__global__ void __launch_bounds__(kDsfpThreads) dsfp_kernel(const float* __restrict__ X, int n, int d,
                                                            const int32_t* __restrict__ nbr, int k, float gamma,
                                                            int T, int m_max, float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int loc[kDsfpMaxK + 1];
  __shared__ int s_m;
  const DsfpLayout L = dsfp_layout(m_max);
  float* buf0 = reinterpret_cast<float*>(smem + L.chunk_off);   // [2][mp][cs]
  float* parts = reinterpret_cast<float*>(smem + L.parts_off);  // [jobs][kTT]
  float* G = reinterpret_cast<float*>(smem + L.mat_off);         // [mp][mp]
  float* M = G + L.mp * L.mp;
  float* P = M + L.mp * L.mp;
  float* Y = P + L.mp * L.mp;
  float* nrm = Y + L.mp * L.mp;                                  // [mp]
  float* deg = nrm + L.mp;                                       // [mp]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = blockIdx.x;
  const int mp = L.mp, cs = L.cs;
  const int nch = (d + kCh - 1) / kCh;
  const int bufsz = mp * cs;

  if (T == 0) {  // the (already normalised) input row
    for (int c4 = tid; c4 < (d >> 2); c4 += kDsfpThreads)
      reinterpret_cast<float4*>(out + (size_t)i * d)[c4] = reinterpret_cast<const float4*>(X + (size_t)i * d)[c4];
    return;
  }

  // ---- local node set: i, then its valid neighbours in list order
  if (warp == 0) {
    int cnt = 1;
    if (lane == 0) loc[0] = i;
    for (int s0 = 0; s0 < k; s0 += 32) {
      const int s = s0 + lane;
      const int j = s < k ? nbr[(size_t)i * k + s] : -1;
      const unsigned vm = __ballot_sync(GCR_FULL, j >= 0);
      if (j >= 0) loc[cnt + __popc(vm & ((1u << lane) - 1))] = j;
      cnt += __popc(vm);
    }
    if (lane == 0) s_m = cnt;
  }
  __syncthreads();
  const int m = s_m;

  // ---- local Gram G = X_L X_L^T over d
  float acc[2][kTl][kTl];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int a = 0; a < kTl; ++a)
#pragma unroll
      for (int b = 0; b < kTl; ++b) acc[q][a][b] = 0.f;
  // job j = (tile pair j / groups, column-quad group j % groups); thread tid takes jobs tid
  // and tid + 128
  int ta[2], tb[2], tg[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = tid + q * kDsfpThreads;
    int pr = j < L.jobs ? j / L.groups : 0;
    tg[q] = j < L.jobs ? j % L.groups : -1;
    int a = 0;
    while (pr >= L.tiles - a) { pr -= L.tiles - a; ++a; }
    ta[q] = a;
    tb[q] = a + pr;
  }
  stage_chunk(buf0, X, loc, m, mp, cs, d, 0);
  cp_async_commit();
  for (int ci = 0; ci < nch; ++ci) {
    if (ci + 1 < nch) stage_chunk(buf0 + ((ci + 1) & 1) * bufsz, X, loc, m, mp, cs, d, (ci + 1) * kCh);
    cp_async_commit();  // (an empty group on the last chunk keeps the count uniform)
    cp_async_wait_prev();
    __syncthreads();
    const float* chunk = buf0 + (ci & 1) * bufsz;
    const int cw = min(kCh, d - ci * kCh);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (tg[q] < 0) continue;
      const float* ra = chunk + ta[q] * kTl * cs;
      const float* rb = chunk + tb[q] * kTl * cs;
      for (int c4 = tg[q] * 4; c4 < cw; c4 += L.groups * 4) {
        float4 u[kTl], v[kTl];
#pragma unroll
        for (int a = 0; a < kTl; ++a) {
          u[a] = *reinterpret_cast<const float4*>(ra + a * cs + c4);
          v[a] = *reinterpret_cast<const float4*>(rb + a * cs + c4);
        }
#pragma unroll
        for (int a = 0; a < kTl; ++a)
#pragma unroll
          for (int b = 0; b < kTl; ++b) {
            float t = acc[q][a][b];
            t = fmaf(u[a].x, v[b].x, t);
            t = fmaf(u[a].y, v[b].y, t);
            t = fmaf(u[a].z, v[b].z, t);
            t = fmaf(u[a].w, v[b].w, t);
            acc[q][a][b] = t;
          }
      }
    }
    __syncthreads();  // the buffer is refilled by the next iteration's copy
  }
  // the output pass streams the same rows again: its first chunk is in flight during the
  // small m x m algebra below
  stage_chunk(buf0, X, loc, m, mp, cs, d, 0);
  cp_async_commit();

  // fold the column groups in a fixed order (the result does not depend on the schedule)
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int j = tid + q * kDsfpThreads;
    if (j < L.jobs)
#pragma unroll
      for (int a = 0; a < kTl; ++a)
#pragma unroll
        for (int b = 0; b < kTl; ++b) parts[(size_t)j * kTT + a * kTl + b] = acc[q][a][b];
  }
  __syncthreads();
  for (int e2 = tid; e2 < L.tp * kTT; e2 += kDsfpThreads) {
    const int pr = e2 / kTT, e = e2 % kTT;
    int a = 0, r = pr;
    while (r >= L.tiles - a) { r -= L.tiles - a; ++a; }
    const int b = a + r;
    float s = 0.f;
    for (int g = 0; g < L.groups; ++g) s += parts[((size_t)pr * L.groups + g) * kTT + e];
    const int u = a * kTl + e / kTl, v = b * kTl + e % kTl;
    G[u * mp + v] = s;
    G[v * mp + u] = s;
  }
  __syncthreads();

  // ---- A, degrees, M = D^{-1/2} A D^{-1/2} (steps 3 and 5): one warp per row u, lanes
  // over the columns v, row sums by warp reduction
  for (int u = warp; u < m; u += kDsfpThreads / 32) {
    float s = 0.f;
    for (int v = lane; v < m; v += 32) {
      const float d2 = fmaxf(0.f, G[u * mp + u] + G[v * mp + v] - 2.f * G[u * mp + v]);
      const float a = u == v ? 1.f : expf(-d2 / gamma);
      M[u * mp + v] = a;
      s += a;
    }
    s = warp_sum(s);
    if (lane == 0) deg[u] = 1.f / sqrtf(s);
  }
  __syncthreads();
  for (int u = warp; u < m; u += kDsfpThreads / 32)
    for (int v = lane; v < m; v += 32) {
      const float a = M[u * mp + v] * (deg[u] * deg[v]);
      M[u * mp + v] = a;
      Y[u * mp + v] = a;  // Y_1 = M P_0 = M
    }
  __syncthreads();

  // ---- step 6 in the m x m space: per iteration ||row u of Y X_0||^2 = sum_w (Y G)_uw Y_uw,
  // P = diag(1/||row u||) Y, Y <- M P
  for (int t = 1;; ++t) {
    const int rows = t < T ? m : 1;  // the last iteration needs the norm of row 0 only
    for (int u = warp; u < rows; u += kDsfpThreads / 32) {
      float s = 0.f;
      for (int w = lane; w < m; w += 32) {
        float z = 0.f;
        for (int v = 0; v < m; ++v) z = fmaf(Y[u * mp + v], G[v * mp + w], z);
        s = fmaf(z, Y[u * mp + w], s);
      }
      s = warp_sum(s);
      if (lane == 0) nrm[u] = s > 0.f ? 1.f / sqrtf(s) : 0.f;
    }
    __syncthreads();
    if (t == T) break;
    for (int u = warp; u < m; u += kDsfpThreads / 32)
      for (int v = lane; v < m; v += 32) P[u * mp + v] = Y[u * mp + v] * nrm[u];
    __syncthreads();
    for (int u = warp; u < m; u += kDsfpThreads / 32)
      for (int v = lane; v < m; v += 32) {
        float s = 0.f;
        for (int w = 0; w < m; ++w) s = fmaf(M[u * mp + w], P[w * mp + v], s);
        Y[u * mp + v] = s;
      }
    __syncthreads();
  }
  // output weights: row 0 of the last Y, scaled by the norm of that row's combination
  if (tid < m) deg[tid] = Y[tid] * nrm[0];
  __syncthreads();

  // ---- output row i = sum_v w_v x_v, column chunk by column chunk (one column per thread)
  for (int ci = 0; ci < nch; ++ci) {
    if (ci + 1 < nch) stage_chunk(buf0 + ((ci + 1) & 1) * bufsz, X, loc, m, mp, cs, d, (ci + 1) * kCh);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    const float* chunk = buf0 + (ci & 1) * bufsz;
    const int c = ci * kCh + tid;
    if (c < d) {
      float s = 0.f;
      for (int v = 0; v < m; ++v) s = fmaf(deg[v], chunk[v * cs + tid], s);
      out[(size_t)i * d + c] = s;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_dsfp(const float* X, int n, int d, const int32_t* nbr, int k, float gamma, int T, float* out,
                        cudaStream_t st) {
  if (n < 1 || k < 0 || k > kDsfpMaxK || d < 4 || d > kMaxD || d % 4 || T < 0) return cudaErrorInvalidValue;
  const DsfpLayout L = dsfp_layout(k + 1);
  if (L.jobs > 2 * kDsfpThreads) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(dsfp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e != cudaSuccess) return e;
  dsfp_kernel<<<n, kDsfpThreads, L.bytes, st>>>(X, n, d, nbr, k, gamma, T, k + 1, out);
  return cudaGetLastError();
}

}  // namespace gcr
