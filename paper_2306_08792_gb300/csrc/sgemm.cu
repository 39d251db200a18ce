// FP32 similarity GEMM on CUDA cores (the plain FP32 reference path of the kNN search).
//
// s_ij = x_i . x_j (Sec. III-B: on unit rows ||x_i - x_j||^2 = 2 - 2 s_ij, so the k nearest
// samples are the k largest scores) computed in 128 x 128 tiles, 256 threads, 8 x 8
// outputs per thread, each output a plain sequential FMA chain over d. That fixes the
// error bound used by the certified refinement: |s^ - s| <= gamma_d * ||x_i|| ||x_j||,
// gamma_d = d u / (1 - d u), u = 2^-24.
//
// Three epilogues share the tile loop:
//   POOL  one CTA owns 128 rows and sweeps every column tile; the tile goes through
//         shared memory into the streaming per-row pool (global graph: threads 0-127,
//         cross-camera graph: threads 128-255).
//   BAND  one CTA owns a column tile and loops over blocks of gathered rows; every score
//         at or above the row's threshold is appended to that row's band buffer.
//   DIST  one CTA per (row tile, column tile): writes ||x_q||^2 + ||x_g||^2 - 2 s_qg.
#include "common.cuh"
#include "pool.cuh"
#include "kernels.h"

namespace gcr {

namespace {

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

}  // namespace

// ---------------------------------------------------------------------------------- POOL
// grid.x = ceil(n / 128); dynamic smem: S tile + two queues.
template <int KP, bool CROSS>
__global__ void __launch_bounds__(256, 1)
sgemm_pool_kernel(const float* __restrict__ X, int n, int d, const int* __restrict__ cam,
                  float* __restrict__ pool_v, int* __restrict__ pool_i) {
  __shared__ TileSmem sm;
  extern __shared__ __align__(16) unsigned char dyn[];
  float (*S)[SP] = reinterpret_cast<float (*)[SP]>(dyn);
  float* qv = reinterpret_cast<float*>(dyn + sizeof(float) * BM * SP);
  int* qi = reinterpret_cast<int*>(qv + 2 * BM * kQCap);
  __shared__ int cam_tile[BN];

  const int tid = threadIdx.x, lane = tid & 31;
  const int ty = tid >> 4, tx = tid & 15;
  const int row0 = blockIdx.x * BM;
  const int kind = tid >> 7;          // 0: global graph, 1: cross-camera graph
  const int r = tid & 127;            // CTA-local row owned by this thread
  const int row = row0 + r;
  const bool valid = row < n && (kind == 0 || CROSS);
  const int my_cam = (CROSS && row < n) ? cam[row] : 0;
  PoolOwner me;
  pool_init(me, valid);
  const int qrow = kind * BM + r;     // queue row of this owner
  const int sw = qrow & 31;
  float* my_qv = qv + qrow * kQCap;
  int* my_qi = qi + qrow * kQCap;
  float* pv = pool_v + (size_t)kind * n * KP;
  int* pi = pool_i + (size_t)kind * n * KP;
  const int warp_row0 = row0 + (r & ~31);
  const int warp_qrow0 = qrow & ~31;
  const int arows = min(BM, n - row0);

  float acc[8][8];
  for (int col0 = 0; col0 < n; col0 += BN) {
    const int brows = min(BN, n - col0);
    tile_mma(sm, X + (size_t)row0 * d, arows, nullptr, X + (size_t)col0 * d, brows, d, acc);
    __syncthreads();  // every thread is past its reads of S (previous tile)
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) S[acc_row(ty, i)][acc_col(tx, j)] = acc[i][j];
    if (CROSS && tid < BN) cam_tile[tid] = (col0 + tid < n) ? cam[col0 + tid] : -1;
    __syncthreads();
    if (kind == 0 || CROSS) {
      for (int c0 = 0; c0 < brows; c0 += 8) {
        pool_make_room<KP>(8, lane, me, warp_row0, warp_qrow0, qv, qi, pv, pi);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int cc = c0 + c;
          const int j = col0 + cc;
          float v = S[r][cc];
          bool ok = cc < brows && j != row;
          if (CROSS && kind == 1) ok = ok && cam_tile[cc] != my_cam;
          if (ok) pool_push(me, v, j, my_qv, my_qi, sw);
        }
      }
    }
  }
  if (kind == 0 || CROSS) pool_flush<KP>(lane, valid, me, warp_row0, warp_qrow0, qv, qi, pv, pi);
}

// ---------------------------------------------------------------------------------- BAND
// Rows to rescan: band_row[u] (sample index), band_kind[u], band_thr[u], u < *count.
// grid.x = ceil(n / 128) column tiles; each CTA loops over the row blocks.
__global__ void __launch_bounds__(256, 1)
sgemm_band_kernel(const float* __restrict__ X, int n, int d, const int* __restrict__ cam,
                  const int* __restrict__ count, int cap, const int* __restrict__ band_row,
                  const int* __restrict__ band_kind, const float* __restrict__ band_thr,
                  int bcap, int* __restrict__ band_cnt, float* __restrict__ band_v,
                  int* __restrict__ band_i) {
  __shared__ TileSmem sm;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int col0 = blockIdx.x * BN;
  const int brows = min(BN, n - col0);
  const int U = min(*count, cap);
  float acc[8][8];
  for (int u0 = 0; u0 < U; u0 += BM) {
    const int arows = min(BM, U - u0);
    tile_mma(sm, X, arows, band_row + u0, X + (size_t)col0 * d, brows, d, acc);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int ur = acc_row(ty, i);
      if (ur >= arows) continue;
      const int u = u0 + ur;
      const int row = band_row[u];
      const int kind = band_kind[u];
      const float thr = band_thr[u];
      const int rc = cam ? cam[row] : 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int cc = acc_col(tx, j);
        const int col = col0 + cc;
        if (cc >= brows || col == row || acc[i][j] < thr) continue;
        if (kind == 1 && cam[col] == rc) continue;
        int pos = atomicAdd(&band_cnt[u], 1);
        if (pos < bcap) {
          band_v[(size_t)u * bcap + pos] = acc[i][j];
          band_i[(size_t)u * bcap + pos] = col;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------- DIST
// D[q][g] = nq[q] + ng[g] - 2 s_qg (squared Euclidean distance), grid = (ceil(ng/128), ceil(nq/128)).
__global__ void __launch_bounds__(256, 2)
sgemm_dist_kernel(const float* __restrict__ Xq, int nq, const float* __restrict__ Xg, int ng,
                  int d, const float* __restrict__ nrm_q, const float* __restrict__ nrm_g,
                  float* __restrict__ D) {
  __shared__ TileSmem sm;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int q0 = blockIdx.y * BM, g0 = blockIdx.x * BN;
  const int arows = min(BM, nq - q0), brows = min(BN, ng - g0);
  float acc[8][8];
  tile_mma(sm, Xq + (size_t)q0 * d, arows, nullptr, Xg + (size_t)g0 * d, brows, d, acc);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int qr = acc_row(ty, i);
    if (qr >= arows) continue;
    const float a = nrm_q[q0 + qr];
    float* out = D + (size_t)(q0 + qr) * ng + g0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gc = acc_col(tx, j);
      if (gc < brows) out[gc] = a + nrm_g[g0 + gc] - 2.f * acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------------- launchers
size_t sgemm_pool_smem() { return sizeof(float) * BM * SP + 2 * BM * kQCap * (sizeof(float) + sizeof(int)); }

cudaError_t launch_sgemm_pool(const float* X, int n, int d, const int* cam, int kp, bool cross,
                              float* pool_v, int* pool_i, cudaStream_t st) {
  dim3 grid((n + BM - 1) / BM);
  size_t smem = sgemm_pool_smem();
#define GCR_POOL_CASE(KPV, CR)                                                                   \
  {                                                                                              \
    auto fn = sgemm_pool_kernel<KPV, CR>;                                                        \
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                              \
    fn<<<grid, 256, smem, st>>>(X, n, d, cam, pool_v, pool_i);                                   \
    return cudaGetLastError();                                                                   \
  }
  if (kp == 32 && !cross) GCR_POOL_CASE(32, false)
  if (kp == 32 && cross) GCR_POOL_CASE(32, true)
  if (kp == 64 && !cross) GCR_POOL_CASE(64, false)
  if (kp == 64 && cross) GCR_POOL_CASE(64, true)
#undef GCR_POOL_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_sgemm_band(const float* X, int n, int d, const int* cam, const int* count,
                              int cap, const int* band_row, const int* band_kind, const float* band_thr,
                              int bcap, int* band_cnt, float* band_v, int* band_i, cudaStream_t st) {
  dim3 grid((n + BN - 1) / BN);
  sgemm_band_kernel<<<grid, 256, 0, st>>>(X, n, d, cam, count, cap, band_row, band_kind, band_thr, bcap,
                                          band_cnt, band_v, band_i);
  return cudaGetLastError();
}

cudaError_t launch_sgemm_dist(const float* Xq, int nq, const float* Xg, int ng, int d,
                              const float* nrm_q, const float* nrm_g, float* D, cudaStream_t st) {
  dim3 grid((ng + BN - 1) / BN, (nq + BM - 1) / BM);
  sgemm_dist_kernel<<<grid, 256, 0, st>>>(Xq, nq, Xg, ng, d, nrm_q, nrm_g, D);
  return cudaGetLastError();
}

}  // namespace gcr
