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
#include "kernels.h"
#include "pool.cuh"
#include "sgemm_tile.cuh"

namespace gcr {

using namespace simt;

// ---------------------------------------------------------------------------------- POOL
// S = A . B^T; rows of A own pools, columns are the rows of B. grid = (ceil(na / 128), splits):
// split y sweeps column tiles [y * tps, (y + 1) * tps). Pools: [split][kind][na][KP].
// With self_excl (A == B) the diagonal is skipped; the cross-camera graph needs A == B.
template <int KP, bool CROSS>
__global__ void __launch_bounds__(256, 1)
sgemm_pool_kernel(const float* __restrict__ A, int na, const float* __restrict__ B, int nb, int d,
                  const int* __restrict__ cam, int self_excl, int tps, float* __restrict__ pool_v,
                  int* __restrict__ pool_i) {
  __shared__ TileSmem sm;
  extern __shared__ __align__(16) unsigned char dyn[];
  float (*S)[SP] = reinterpret_cast<float (*)[SP]>(dyn);
  float2* q = reinterpret_cast<float2*>(dyn + sizeof(float) * BM * SP);
  __shared__ int cam_tile[BN];

  const int tid = threadIdx.x, lane = tid & 31;
  const int ty = tid >> 4, tx = tid & 15;
  const int row0 = blockIdx.x * BM;
  const int kind = tid >> 7;          // 0: global graph, 1: cross-camera graph
  const int r = tid & 127;            // CTA-local row owned by this thread
  const int row = row0 + r;
  const bool valid = row < na && (kind == 0 || CROSS);
  const int my_cam = (CROSS && row < na) ? cam[row] : 0;
  PoolOwner me;
  pool_init(me, valid);
  const int qrow = kind * BM + r;     // queue row of this owner
  const int sw = qrow & 31;
  float2* my_q = q + qrow * kQCap;
  const int kinds = CROSS ? 2 : 1;
  const size_t pbase = ((size_t)blockIdx.y * kinds + kind) * na * KP;
  float* pv = pool_v + pbase;
  int* pi = pool_i + pbase;
  const int warp_row0 = row0 + (r & ~31);
  const int warp_qrow0 = qrow & ~31;
  const int arows = min(BM, na - row0);
  const int ntiles = (nb + BN - 1) / BN;
  const int t0 = blockIdx.y * tps, t1 = min(ntiles, t0 + tps);

  float acc[8][8];
  for (int t = t0; t < t1; ++t) {
    const int col0 = t * BN;
    const int brows = min(BN, nb - col0);
    tile_mma(sm, A + (size_t)row0 * d, arows, nullptr, B + (size_t)col0 * d, brows, d, acc);
    __syncthreads();  // every thread is past its reads of S (previous tile)
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) S[acc_row(ty, i)][acc_col(tx, j)] = acc[i][j];
    if (CROSS && tid < BN) cam_tile[tid] = (col0 + tid < nb) ? cam[col0 + tid] : -1;
    __syncthreads();
    if (kind == 0 || CROSS) {
      for (int c0 = 0; c0 < brows; c0 += 4) {  // queues fill to 28 of 32 before a merge
        pool_make_room<KP>(4, lane, me, warp_row0, warp_qrow0, q, pv, pi);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int cc = c0 + c;
          const int j = col0 + cc;
          float v = S[r][cc];
          bool ok = cc < brows && !(self_excl && j == row);
          if (CROSS && kind == 1) ok = ok && cam_tile[cc] != my_cam;
          pool_push(me, v, j, ok, my_q, sw);
        }
      }
    }
  }
  if (kind == 0 || CROSS) pool_flush<KP>(lane, valid, me, warp_row0, warp_qrow0, q, pv, pi);
}

// ---------------------------------------------------------------------------------- BAND
// Rows to rescan: band_row[u] (sample index), band_kind[u], band_thr[u], u < *count.
// grid.x = ceil(n / 128) column tiles; each CTA loops over the row blocks.
__global__ void __launch_bounds__(256, 1)
sgemm_band_kernel(const float* __restrict__ X, const float* __restrict__ Bm, int n, int d,
                  const int* __restrict__ cam, int self_excl,
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
    tile_mma(sm, X, arows, band_row + u0, Bm + (size_t)col0 * d, brows, d, acc);
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
        if (cc >= brows || (self_excl && col == row) || acc[i][j] < thr) continue;
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

cudaError_t launch_sgemm_pool(const float* A, int na, const float* B, int nb, int d, const int* cam, int kp,
                              bool cross, int self_excl, int splits, float* pool_v, int* pool_i, cudaStream_t st) {
  const int ntiles = (nb + BN - 1) / BN;
  if (splits < 1) splits = 1;
  if (splits > ntiles) splits = ntiles;
  const int tps = (ntiles + splits - 1) / splits;
  splits = (ntiles + tps - 1) / tps;  // no split is left without a column tile
  dim3 grid((na + BM - 1) / BM, splits);
  size_t smem = sgemm_pool_smem();
#define GCR_POOL_CASE(KPV, CR)                                                                   \
  {                                                                                              \
    auto fn = sgemm_pool_kernel<KPV, CR>;                                                        \
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                              \
    fn<<<grid, 256, smem, st>>>(A, na, B, nb, d, cam, self_excl, tps, pool_v, pool_i);           \
    return cudaGetLastError();                                                                   \
  }
  if (kp == 32 && !cross) GCR_POOL_CASE(32, false)
  if (kp == 32 && cross) GCR_POOL_CASE(32, true)
  if (kp == 64 && !cross) GCR_POOL_CASE(64, false)
  if (kp == 64 && cross) GCR_POOL_CASE(64, true)
  if (kp == 128 && !cross) GCR_POOL_CASE(128, false)
  if (kp == 128 && cross) GCR_POOL_CASE(128, true)
#undef GCR_POOL_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_sgemm_band(const float* X, const float* Bm, int n, int d, const int* cam, int self_excl,
                              const int* count, int cap, const int* band_row, const int* band_kind,
                              const float* band_thr, int bcap, int* band_cnt, float* band_v, int* band_i,
                              cudaStream_t st) {
  dim3 grid((n + BN - 1) / BN);
  sgemm_band_kernel<<<grid, 256, 0, st>>>(X, Bm, n, d, cam, self_excl, count, cap, band_row, band_kind, band_thr,
                                          bcap, band_cnt, band_v, band_i);
  return cudaGetLastError();
}

cudaError_t launch_sgemm_dist(const float* Xq, int nq, const float* Xg, int ng, int d,
                              const float* nrm_q, const float* nrm_g, float* D, cudaStream_t st) {
  dim3 grid((ng + BN - 1) / BN, (nq + BM - 1) / BM);
  sgemm_dist_kernel<<<grid, 256, 0, st>>>(Xq, nq, Xg, ng, d, nrm_q, nrm_g, D);
  return cudaGetLastError();
}

}  // namespace gcr
