// GCRV tracklet profile vectors (Sec. III-D, Eq. 10 and Eq. 17; Algorithm 2 step 1).
//
// For every tracklet c of camera s:
//   mu_c = mean of c's L2-normalised frames                                   (Eq. 10)
//   w_c  = (G_s + lambda n_s I)^{-1} (mu_c - mu_s),  G_s = X_s^T X_s           (Eq. 17)
// where X_s stacks the n_s normalised frames of every tracklet of camera s and mu_s is their
// mean. A camera holding one tracklet gives w = 0; that tracklet keeps mu_c.
//
// Device-side plan (no host synchronisation):
//   1. 1/||x_f|| per frame (frames are normalised on the fly, never copied);
//   2. one block orders the tracklets by camera (stable), pads each camera's block of rows to
//      a multiple of 128 and lays out its frames contiguously in a frame index list;
//   3. tracklet means and camera means;
//   4. per-camera Gram G_s on CUDA cores (upper-triangle 128 x 128 tiles, mirrored), K = the
//      camera's frames, gathered through the frame list;
//   5. conjugate gradients for all right-hand sides at once: each iteration is one
//      (rows of P) x G_s product per camera plus one row-wise update. Since every frame has
//      unit norm, the eigenvalues of G_s lie in [0, n_s], so cond(G_s + lambda n_s I) <=
//      1 + 1/lambda and the iteration count needed for a relative error of 1e-7 follows
//      from the standard CG bound 2 ((sqrt(k)-1)/(sqrt(k)+1))^m.
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "sgemm_tile.cuh"

namespace gcr {
namespace {

using namespace simt;

constexpr int kMaxCams = 64;

__global__ void frame_inv_norm_kernel(const float* __restrict__ F, int64_t nf, int d, float* __restrict__ inv) {
  const int lane = threadIdx.x & 31;
  const int64_t f = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (f >= nf) return;
  const float4* x = reinterpret_cast<const float4*>(F + f * d);
  double ss = 0.0;
  for (int v = lane; v < (d >> 2); v += 32) {
    const float4 a = x[v];
    ss += (double)a.x * a.x + (double)a.y * a.y + (double)a.z * a.z + (double)a.w * a.w;
  }
  ss = warp_sum_d(ss);
  if (lane == 0) inv[f] = ss > 0.0 ? (float)(1.0 / sqrt(ss)) : 0.f;
}

struct Layout {
  int* cam_cnt;       // [kMaxCams] tracklets per camera
  int64_t* cam_nf;    // [kMaxCams] frames per camera (n_s)
  int* blk0;          // [kMaxCams + 1] first 128-row block of each camera
  int* perm;          // [rows_cap] tracklet at each padded row (-1: padding)
  int* pos;           // [C] padded row of each tracklet
  int64_t* fstart;    // [C] start of the tracklet's frames in the frame list
  int64_t* foff;      // [kMaxCams + 1] start of each camera's frames in the frame list
  int* row_cam;       // [rows_cap / 128] camera of each row block
};

// One block of 1024 threads: stable grouping of the tracklets by camera.
__global__ void __launch_bounds__(1024) layout_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ cam,
                                                      int C, int ncam, int rows_cap, Layout L) {
  __shared__ int cnt[kMaxCams];
  __shared__ long long nfr[kMaxCams];
  __shared__ int run[kMaxCams];
  __shared__ long long frun[kMaxCams];
  __shared__ int wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid < kMaxCams) { cnt[tid] = 0; nfr[tid] = 0; run[tid] = 0; frun[tid] = 0; }
  __syncthreads();
  for (int c = tid; c < C; c += blockDim.x) {
    const int s = cam[c];
    atomicAdd(&cnt[s], 1);
    atomicAdd((unsigned long long*)&nfr[s], (unsigned long long)(off[c + 1] - off[c]));
  }
  __syncthreads();
  if (tid == 0) {
    int b = 0;
    long long fo = 0;
    for (int s = 0; s < ncam; ++s) {
      L.blk0[s] = b;
      L.foff[s] = fo;
      L.cam_cnt[s] = cnt[s];
      L.cam_nf[s] = nfr[s];
      for (int q = 0; q < (cnt[s] + 127) / 128; ++q) L.row_cam[b + q] = s;
      b += (cnt[s] + 127) / 128;
      fo += nfr[s];
    }
    L.blk0[ncam] = b;
    L.foff[ncam] = fo;
    for (int q = b; q < rows_cap / 128; ++q) L.row_cam[q] = -1;
  }
  for (int r = tid; r < rows_cap; r += blockDim.x) L.perm[r] = -1;
  __syncthreads();
  // ranks within each camera, chunk by chunk, in tracklet order
  for (int base = 0; base < C; base += blockDim.x) {
    const int c = base + tid;
    const int s = c < C ? cam[c] : -1;
    const long long len = c < C ? (long long)(off[c + 1] - off[c]) : 0;
    for (int q = 0; q < ncam; ++q) {
      const bool f = s == q;
      const unsigned m = __ballot_sync(GCR_FULL, f);
      if (lane == 0) wsum[w] = __popc(m);
      __syncthreads();
      int before = 0;
      for (int i = 0; i < w; ++i) before += wsum[i];
      const int rank = before + __popc(m & ((1u << lane) - 1));
      // frames of earlier tracklets of camera q in this chunk: second pass over the chunk
      __syncthreads();
      if (f) {
        const int row = L.blk0[q] * 128 + run[q] + rank;
        L.perm[row] = c;
        L.pos[c] = row;
      }
      __syncthreads();
      if (tid == 0) {
        int tot = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += wsum[i];
        run[q] += tot;
      }
      __syncthreads();
    }
    (void)len;
  }
  __syncthreads();
  // frame starts: walk each camera's rows in order (one thread per camera; C is small)
  if (tid < ncam) {
    long long fo = L.foff[tid];
    const int r0 = L.blk0[tid] * 128, r1 = r0 + cnt[tid];
    for (int r = r0; r < r1; ++r) {
      const int c = L.perm[r];
      L.fstart[c] = fo;
      fo += off[c + 1] - off[c];
    }
  }
}

__global__ void frame_list_kernel(const int64_t* __restrict__ off, int C, const int64_t* __restrict__ fstart,
                                  int* __restrict__ flist) {
  const int c = blockIdx.x;
  if (c >= C) return;
  const int64_t b = off[c], m = off[c + 1] - b, s = fstart[c];
  for (int64_t t = threadIdx.x; t < m; t += blockDim.x) flist[s + t] = (int)(b + t);
}

// mu[row] = mean of the tracklet's normalised frames (Eq. 10); padded rows are zero.
__global__ void means_kernel(const float* __restrict__ F, int d, const int64_t* __restrict__ off,
                             const float* __restrict__ inv, const int* __restrict__ perm, float* __restrict__ mu) {
  const int row = blockIdx.x;
  const int c = perm[row];
  float* out = mu + (size_t)row * d;
  for (int a = threadIdx.x * 4; a < d; a += blockDim.x * 4) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c >= 0) {
      const int64_t b = off[c], e = off[c + 1];
      for (int64_t f = b; f < e; ++f) {
        const float s = inv[f];
        const float4 x = *reinterpret_cast<const float4*>(F + f * d + a);
        acc.x = fmaf(x.x, s, acc.x); acc.y = fmaf(x.y, s, acc.y);
        acc.z = fmaf(x.z, s, acc.z); acc.w = fmaf(x.w, s, acc.w);
      }
      const float m = 1.0f / (float)(e - b);
      acc.x *= m; acc.y *= m; acc.z *= m; acc.w *= m;
    }
    *reinterpret_cast<float4*>(out + a) = acc;
  }
}

// mu_s = (sum over the camera's tracklets of m_c mu_c) / n_s, in row order (deterministic).
__global__ void cam_means_kernel(const float* __restrict__ mu, int d, const int64_t* __restrict__ off,
                                 const int* __restrict__ perm, Layout L, float* __restrict__ mu_cam) {
  const int s = blockIdx.y;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d) return;
  const int r0 = L.blk0[s] * 128, r1 = r0 + L.cam_cnt[s];
  double acc = 0.0;
  for (int r = r0; r < r1; ++r) {
    const int c = perm[r];
    acc += (double)(off[c + 1] - off[c]) * (double)mu[(size_t)r * d + a];
  }
  const int64_t nf = L.cam_nf[s];
  mu_cam[(size_t)s * d + a] = nf > 0 ? (float)(acc / (double)nf) : 0.f;
}

// G_s = sum over the camera's frames of x^ x^^T, upper-triangle tiles mirrored, plus
// lambda n_s on the diagonal. grid = (d/128 tiles a, d/128 tiles b, camera).
__global__ void __launch_bounds__(256) gram_kernel(const float* __restrict__ F, int d, const float* __restrict__ inv,
                                                   const int* __restrict__ flist, Layout L, float lambda,
                                                   float* __restrict__ G) {
  const int ta = blockIdx.x, tb = blockIdx.y, s = blockIdx.z;
  if (tb < ta) return;
  __shared__ TileSmem sm;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int a0 = ta * BM, b0 = tb * BN;
  const int64_t f0 = L.foff[s], nf = L.cam_nf[s];
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  // slice loader: 8 frames x 128 features; thread t -> frame t/32, features 4*(t%32)
  auto load = [&](int64_t k0, int col0) {
    const int kk = tid >> 5, cc = (tid & 31) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k0 + kk < nf && col0 + cc < d) {
      const int f = flist[f0 + k0 + kk];
      const float sc = inv[f];
      v = *reinterpret_cast<const float4*>(F + (size_t)f * d + col0 + cc);
      v.x *= sc; v.y *= sc; v.z *= sc; v.w *= sc;
    }
    return v;
  };
  auto store = [&](float (*S)[PITCH], float4 v) {
    const int kk = tid >> 5, cc = (tid & 31) * 4;
    *reinterpret_cast<float4*>(&S[kk][cc]) = v;
  };
  float4 ra = load(0, a0), rb = load(0, b0);
  store(sm.As[0], ra);
  store(sm.Bs[0], rb);
  __syncthreads();
  int buf = 0;
  for (int64_t k0 = 0; k0 < nf; k0 += BK) {
    const bool more = k0 + BK < nf;
    if (more) { ra = load(k0 + BK, a0); rb = load(k0 + BK, b0); }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 x0 = *reinterpret_cast<const float4*>(&sm.As[buf][kk][ty * 4]);
      const float4 x1 = *reinterpret_cast<const float4*>(&sm.As[buf][kk][64 + ty * 4]);
      const float4 y0 = *reinterpret_cast<const float4*>(&sm.Bs[buf][kk][tx * 4]);
      const float4 y1 = *reinterpret_cast<const float4*>(&sm.Bs[buf][kk][64 + tx * 4]);
      const float av[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float bv[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      store(sm.As[buf ^ 1], ra);
      store(sm.Bs[buf ^ 1], rb);
      __syncthreads();
      buf ^= 1;
    }
  }
  float* Gs = G + (size_t)s * d * d;
  const float lam_n = lambda * (float)nf;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int a = a0 + acc_row(ty, i);
    if (a >= d) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int b = b0 + acc_col(tx, j);
      if (b >= d) continue;
      const float v = acc[i][j] + (a == b ? lam_n : 0.f);
      Gs[(size_t)a * d + b] = v;
      if (ta != tb) Gs[(size_t)b * d + a] = v;
    }
  }
}

// R = mu_c - mu_s, X = 0, P = R, rr = R.R (one warp per padded row).
__global__ void cg_init_kernel(const float* __restrict__ mu, const float* __restrict__ mu_cam, int d,
                               const int* __restrict__ perm, const int* __restrict__ row_cam, int rows,
                               float* __restrict__ Xs, float* __restrict__ R, float* __restrict__ P,
                               double* __restrict__ rr) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const int s = row_cam[r >> 7];
  const bool live = perm[r] >= 0 && s >= 0;
  double acc = 0.0;
  for (int a = lane * 4; a < d; a += 128) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
      const float4 m = *reinterpret_cast<const float4*>(mu + (size_t)r * d + a);
      const float4 q = *reinterpret_cast<const float4*>(mu_cam + (size_t)s * d + a);
      v = make_float4(m.x - q.x, m.y - q.y, m.z - q.z, m.w - q.w);
    }
    *reinterpret_cast<float4*>(R + (size_t)r * d + a) = v;
    *reinterpret_cast<float4*>(P + (size_t)r * d + a) = v;
    *reinterpret_cast<float4*>(Xs + (size_t)r * d + a) = make_float4(0.f, 0.f, 0.f, 0.f);
    acc += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
  }
  acc = warp_sum_d(acc);
  if (lane == 0) rr[r] = acc;
}

// Q = P (G_s + lambda n_s I) for each camera's 128-row blocks (G_s symmetric, so this is
// the tile product P . G_s^T). grid = (d/128, row blocks).
__global__ void __launch_bounds__(256) cg_apply_kernel(const float* __restrict__ P, const float* __restrict__ G, int d,
                                                       const int* __restrict__ row_cam, float* __restrict__ Q) {
  const int s = row_cam[blockIdx.y];
  if (s < 0) return;
  __shared__ TileSmem sm;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  float acc[8][8];
  tile_mma(sm, P + (size_t)r0 * d, BM, nullptr, G + (size_t)s * d * d + (size_t)c0 * d, min(BN, d - c0), d, acc);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + acc_row(ty, i);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c0 + acc_col(tx, j);
      if (c < d) Q[(size_t)r * d + c] = acc[i][j];
    }
  }
}

// One CG step per row: alpha = rr / p.q; x += alpha p; r -= alpha q; beta = rr'/rr; p = r + beta p.
template <int VPL>
__global__ void __launch_bounds__(256) cg_update_kernel(float* __restrict__ Xs, float* __restrict__ R,
                                                        float* __restrict__ P, const float* __restrict__ Q,
                                                        double* __restrict__ rr, const int* __restrict__ perm,
                                                        int rows, int d) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows || perm[r] < 0) return;
  const double rr0 = rr[r];
  if (!(rr0 > 0.0)) return;
  float4 p[VPL], q[VPL];
  double pq = 0.0;
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int a = v * 128 + lane * 4;
    if (a < d) {
      p[v] = *reinterpret_cast<const float4*>(P + (size_t)r * d + a);
      q[v] = *reinterpret_cast<const float4*>(Q + (size_t)r * d + a);
      pq += (double)p[v].x * q[v].x + (double)p[v].y * q[v].y + (double)p[v].z * q[v].z + (double)p[v].w * q[v].w;
    }
  }
  pq = warp_sum_d(pq);
  if (!(pq > 0.0)) return;
  const float alpha = (float)(rr0 / pq);
  double rr1 = 0.0;
  float4 rv[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int a = v * 128 + lane * 4;
    if (a < d) {
      float4 x = *reinterpret_cast<const float4*>(Xs + (size_t)r * d + a);
      float4 rt = *reinterpret_cast<const float4*>(R + (size_t)r * d + a);
      x.x = fmaf(alpha, p[v].x, x.x); x.y = fmaf(alpha, p[v].y, x.y);
      x.z = fmaf(alpha, p[v].z, x.z); x.w = fmaf(alpha, p[v].w, x.w);
      rt.x = fmaf(-alpha, q[v].x, rt.x); rt.y = fmaf(-alpha, q[v].y, rt.y);
      rt.z = fmaf(-alpha, q[v].z, rt.z); rt.w = fmaf(-alpha, q[v].w, rt.w);
      *reinterpret_cast<float4*>(Xs + (size_t)r * d + a) = x;
      *reinterpret_cast<float4*>(R + (size_t)r * d + a) = rt;
      rv[v] = rt;
      rr1 += (double)rt.x * rt.x + (double)rt.y * rt.y + (double)rt.z * rt.z + (double)rt.w * rt.w;
    }
  }
  rr1 = warp_sum_d(rr1);
  const float beta = (float)(rr1 / rr0);
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int a = v * 128 + lane * 4;
    if (a < d) {
      const float4 np = make_float4(fmaf(beta, p[v].x, rv[v].x), fmaf(beta, p[v].y, rv[v].y),
                                    fmaf(beta, p[v].z, rv[v].z), fmaf(beta, p[v].w, rv[v].w));
      *reinterpret_cast<float4*>(P + (size_t)r * d + a) = np;
    }
  }
  if (lane == 0) rr[r] = rr1;
}

// W[c] = solution row of c, or its mean profile when its camera holds one tracklet.
__global__ void gcrv_out_kernel(const float* __restrict__ Xs, const float* __restrict__ mu, int d, int C,
                                const int32_t* __restrict__ cam, Layout L, float* __restrict__ W) {
  const int c = blockIdx.x;
  if (c >= C) return;
  const int r = L.pos[c];
  const bool single = L.cam_cnt[cam[c]] == 1;
  const float* src = (single ? mu : Xs) + (size_t)r * d;
  for (int a = threadIdx.x * 4; a < d; a += blockDim.x * 4)
    *reinterpret_cast<float4*>(W + (size_t)c * d + a) = *reinterpret_cast<const float4*>(src + a);
}

}  // namespace

// ---------------------------------------------------------------------------------- host
int gcrv_iterations(float lambda) {
  const double kappa = 1.0 + 1.0 / (double)lambda;
  const double rho = (std::sqrt(kappa) - 1.0) / (std::sqrt(kappa) + 1.0);
  if (rho <= 0.0) return 1;
  int m = (int)std::ceil(std::log(5e-8) / std::log(rho)) + 1;
  return m < 1 ? 1 : (m > 400 ? 400 : m);
}

size_t gcrv_carve(Carve& c, int64_t F, int d, int C, int ncam, GcrvWs* w) {
  const int rows_cap = (C + 128 * ncam + 127) / 128 * 128;
  GcrvWs t;
  t.rows_cap = rows_cap;
  t.inv = c.take<float>((size_t)F);
  t.cam_cnt = c.take<int>(kMaxCams);
  t.cam_nf = c.take<int64_t>(kMaxCams);
  t.blk0 = c.take<int>(kMaxCams + 1);
  t.perm = c.take<int>(rows_cap);
  t.pos = c.take<int>(C);
  t.fstart = c.take<int64_t>(C);
  t.foff = c.take<int64_t>(kMaxCams + 1);
  t.row_cam = c.take<int>(rows_cap / 128);
  t.flist = c.take<int>((size_t)F);
  t.mu = c.take<float>((size_t)rows_cap * d);
  t.mu_cam = c.take<float>((size_t)ncam * d);
  t.G = c.take<float>((size_t)ncam * d * d);
  t.X = c.take<float>((size_t)rows_cap * d);
  t.R = c.take<float>((size_t)rows_cap * d);
  t.P = c.take<float>((size_t)rows_cap * d);
  t.Q = c.take<float>((size_t)rows_cap * d);
  t.rr = c.take<double>(rows_cap);
  if (w) *w = t;
  return c.off;
}

cudaError_t launch_gcrv(const float* frames, int64_t F, int d, const int64_t* off, const int32_t* cam, int C,
                        int ncam, float lambda, float* W, const GcrvWs& w, cudaStream_t st) {
  Layout L{w.cam_cnt, w.cam_nf, w.blk0, w.perm, w.pos, w.fstart, w.foff, w.row_cam};
  frame_inv_norm_kernel<<<(unsigned)((F + 7) / 8), 256, 0, st>>>(frames, F, d, w.inv);
  layout_kernel<<<1, 1024, 0, st>>>(off, cam, C, ncam, w.rows_cap, L);
  frame_list_kernel<<<C, 128, 0, st>>>(off, C, w.fstart, w.flist);
  means_kernel<<<w.rows_cap, 256, 0, st>>>(frames, d, off, w.inv, w.perm, w.mu);
  cam_means_kernel<<<dim3((d + 255) / 256, ncam), 256, 0, st>>>(w.mu, d, off, w.perm, L, w.mu_cam);
  const int td = (d + BM - 1) / BM;
  gram_kernel<<<dim3(td, td, ncam), 256, 0, st>>>(frames, d, w.inv, w.flist, L, lambda, w.G);
  const int rows = w.rows_cap;
  cg_init_kernel<<<(rows + 7) / 8, 256, 0, st>>>(w.mu, w.mu_cam, d, w.perm, w.row_cam, rows, w.X, w.R, w.P, w.rr);
  const int iters = gcrv_iterations(lambda);
  const int vpl = (d + 127) / 128;
  for (int it = 0; it < iters; ++it) {
    cg_apply_kernel<<<dim3(td, rows / 128), 256, 0, st>>>(w.P, w.G, d, w.row_cam, w.Q);
    if (vpl <= 2) cg_update_kernel<2><<<(rows + 7) / 8, 256, 0, st>>>(w.X, w.R, w.P, w.Q, w.rr, w.perm, rows, d);
    else if (vpl <= 4) cg_update_kernel<4><<<(rows + 7) / 8, 256, 0, st>>>(w.X, w.R, w.P, w.Q, w.rr, w.perm, rows, d);
    else if (vpl <= 8) cg_update_kernel<8><<<(rows + 7) / 8, 256, 0, st>>>(w.X, w.R, w.P, w.Q, w.rr, w.perm, rows, d);
    else if (vpl <= 16) cg_update_kernel<16><<<(rows + 7) / 8, 256, 0, st>>>(w.X, w.R, w.P, w.Q, w.rr, w.perm, rows, d);
    else cg_update_kernel<32><<<(rows + 7) / 8, 256, 0, st>>>(w.X, w.R, w.P, w.Q, w.rr, w.perm, rows, d);
  }
  gcrv_out_kernel<<<C, 256, 0, st>>>(w.X, w.mu, d, C, cam, L, W);
  return cudaGetLastError();
}

}  // namespace gcr
