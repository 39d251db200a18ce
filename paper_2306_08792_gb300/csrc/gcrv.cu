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
//   4. per-camera Gram G_s on the tcgen05 tensor cores: the camera's normalised frames are
//      written transposed (features x frames, camera blocks padded to 64 frames) as BF16
//      hi + lo, and G_s = hi.hi^T + hi.lo^T + lo.hi^T is accumulated in FP32 (error about
//      2^-16 relative, against 2^-11 for TF32 operands), plus lambda n_s on the diagonal; only
//      the tiles on or above the diagonal are computed, the lower triangle is mirrored;
//   5. conjugate gradients for all right-hand sides at once: each iteration is one
//      (rows of P) x G_s product per camera (tensor cores, TF32 hi + lo operands) plus one
//      row-wise update. Since every frame has
//      unit norm, the eigenvalues of G_s lie in [0, n_s], so cond(G_s + lambda n_s I) <=
//      1 + 1/lambda and the iteration count needed for a relative error of 1e-7 follows
//      from the standard CG bound 2 ((sqrt(k)-1)/(sqrt(k)+1))^m.
#include <cmath>

#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

constexpr int kMaxCams = 64;

__global__ void frame_inv_norm_kernel(const float* __restrict__ F, int64_t nf, int d, float* __restrict__ inv) {
  const int lane = threadIdx.x & 31;
  const int64_t f = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (f >= nf) return;
  const float4* x = reinterpret_cast<const float4*>(F + f * d);
  FF acc;  // float-float: FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU
  for (int v = lane; v < (d >> 2); v += 32) {
    const float4 a = x[v];
    acc.add_sq(a.x); acc.add_sq(a.y); acc.add_sq(a.z); acc.add_sq(a.w);
  }
  const double ss = warp_sum_d(acc.value());
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
  __shared__ int wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid < kMaxCams) { cnt[tid] = 0; nfr[tid] = 0; run[tid] = 0; }
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

// Column blocks (64 frames each) of every camera in the transposed frame matrix Z:
// camera s owns blocks [kstart[s], kstart[s] + knum[s]), knum[s] = ceil(n_s / 64).
__global__ void zt_blocks_kernel(const int64_t* __restrict__ cam_nf, int ncam, int64_t* __restrict__ kstart,
                                 int64_t* __restrict__ knum) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t b = 0;
  for (int s = 0; s < ncam; ++s) {
    kstart[s] = b;
    knum[s] = (cam_nf[s] + 63) / 64;
    b += knum[s];
  }
}

// Z^T in BF16 hi + lo for the tensor-core Gram: column q of camera s's block range holds the
// camera's q-th frame (frame-list order), normalised; hi = bf16(x), lo = bf16(x - hi), so that
// hi.hi + hi.lo + lo.hi reproduces x.x' to about 2^-16 relative. Columns past n_s are zero. One
// block per 64 columns x 64 features, transposed through shared memory.
__global__ void __launch_bounds__(256) zt_split_kernel(const float* __restrict__ F, int d, const float* __restrict__ inv,
                                                       const int* __restrict__ flist, const int64_t* __restrict__ foff,
                                                       const int64_t* __restrict__ cam_nf,
                                                       const int64_t* __restrict__ kstart,
                                                       const int64_t* __restrict__ knum, int ncam, int64_t cols,
                                                       __nv_bfloat16* __restrict__ zt_hi,
                                                       __nv_bfloat16* __restrict__ zt_lo) {
  __shared__ float tile[64][65];
  const int64_t cb = blockIdx.x;  // column block
  const int a0 = blockIdx.y * 64;
  int s = -1;
  for (int t = 0; t < ncam; ++t)
    if (cb >= kstart[t] && cb < kstart[t] + knum[t]) s = t;
  if (s < 0) return;  // past the last camera's blocks
  const int64_t q0 = (cb - kstart[s]) * 64, ns = cam_nf[s];
  // load 64 frames x 64 features (4 floats per thread per step)
  for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {
    const int fr = e / 16, c4 = (e % 16) * 4;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q0 + fr < ns && a0 + c4 < d) {
      const int f = flist[foff[s] + q0 + fr];
      const float sc = inv[f];
      x = *reinterpret_cast<const float4*>(F + (size_t)f * d + a0 + c4);
      x.x *= sc; x.y *= sc; x.z *= sc; x.w *= sc;
    }
    tile[fr][c4] = x.x; tile[fr][c4 + 1] = x.y; tile[fr][c4 + 2] = x.z; tile[fr][c4 + 3] = x.w;
  }
  __syncthreads();
  // write 64 feature rows x 64 frame columns, two columns per thread per step
  for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
    const int a = e / 32, q = (e % 32) * 2;
    if (a0 + a >= d) continue;
    const float x0 = tile[q][a], x1 = tile[q + 1][a];
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
    const size_t o = (size_t)(a0 + a) * cols + cb * 64 + q;
    *reinterpret_cast<__nv_bfloat162*>(zt_hi + o) = __halves2bfloat162(h0, h1);
    *reinterpret_cast<__nv_bfloat162*>(zt_lo + o) = __halves2bfloat162(l0, l1);
  }
}

// The tensor-core Gram computes the tiles on or above the diagonal; the strictly lower
// triangle is then copied from the upper one (32 x 32 tiles through shared memory), so G_s is
// exactly symmetric. grid = (d/32, d/32, ncam), block (32, 8).
__global__ void gram_mirror_kernel(float* __restrict__ G, int d) {
  __shared__ float t[32][33];
  const int bx = blockIdx.x, by = blockIdx.y;  // lower tile: rows by*32.., cols bx*32..
  if (by < bx) return;
  float* Gs = G + (size_t)blockIdx.z * d * d;
  for (int r = threadIdx.y; r < 32; r += 8) {  // read the upper tile (rows bx*32.., cols by*32..)
    const int a = bx * 32 + r, b = by * 32 + threadIdx.x;
    if (a < d && b < d) t[r][threadIdx.x] = Gs[(size_t)a * d + b];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int a = by * 32 + r, b = bx * 32 + threadIdx.x;
    if (a < d && b < d && a > b) Gs[(size_t)a * d + b] = t[threadIdx.x][r];
  }
}

// mu[row] = mean of the tracklet's normalised frames (Eq. 10); padded rows are zero.
__global__ void means_kernel(const float* __restrict__ F, int d, const int64_t* __restrict__ off,
                             const float* __restrict__ inv, const int* __restrict__ perm, float* __restrict__ mu) {
  const int row = blockIdx.x;
  const int c = perm ? perm[row] : row;  // no permutation: row r is tracklet r
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

// x = hi + lo with hi = tf32(x), lo = tf32(x - hi): hi.hi + hi.lo + lo.hi reproduces products to
// about 2^-21 relative on the tensor cores.
__global__ void split_tf32_kernel(const float* __restrict__ x, int64_t n, float* __restrict__ hi,
                                  float* __restrict__ lo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[i];
    const float h = round_tf32(v);
    hi[i] = h;
    lo[i] = round_tf32(v - h);
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
  FF pqa;  // float-float: FP64 arithmetic is slow on this GPU
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int a = v * 128 + lane * 4;
    if (a < d) {
      p[v] = *reinterpret_cast<const float4*>(P + (size_t)r * d + a);
      q[v] = *reinterpret_cast<const float4*>(Q + (size_t)r * d + a);
      pqa.add_prod(p[v].x, q[v].x); pqa.add_prod(p[v].y, q[v].y);
      pqa.add_prod(p[v].z, q[v].z); pqa.add_prod(p[v].w, q[v].w);
    }
  }
  const double pq = warp_sum_d(pqa.value());
  if (!(pq > 0.0)) return;
  const float alpha = (float)(rr0 / pq);
  FF rra;
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
      rra.add_sq(rt.x); rra.add_sq(rt.y); rra.add_sq(rt.z); rra.add_sq(rt.w);
    }
  }
  const double rr1 = warp_sum_d(rra.value());
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
  t.g_hi = c.take<float>((size_t)ncam * d * d);
  t.g_lo = c.take<float>((size_t)ncam * d * d);
  t.p_hi = c.take<float>((size_t)rows_cap * d);
  t.p_lo = c.take<float>((size_t)rows_cap * d);
  t.zt_cols = (F + 63) / 64 * 64 + 64 * (int64_t)ncam;  // camera blocks padded to 64 frames
  t.zt_hi = c.take<__nv_bfloat16>((size_t)d * t.zt_cols);
  t.zt_lo = c.take<__nv_bfloat16>((size_t)d * t.zt_cols);
  t.kstart = c.take<int64_t>(kMaxCams);
  t.knum = c.take<int64_t>(kMaxCams);
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
  // G_s on the tensor cores: compensated BF16 operands of the transposed normalised frames
  zt_blocks_kernel<<<1, 32, 0, st>>>(w.cam_nf, ncam, w.kstart, w.knum);
  zt_split_kernel<<<dim3((unsigned)(w.zt_cols / 64), (unsigned)((d + 63) / 64)), 256, 0, st>>>(
      frames, d, w.inv, w.flist, w.foff, w.cam_nf, w.kstart, w.knum, ncam, w.zt_cols, w.zt_hi, w.zt_lo);
  cudaError_t e = launch_umma_gram(w.zt_hi, w.zt_lo, d, w.zt_cols, w.kstart, w.knum, w.cam_nf, ncam, lambda, w.G,
                                   st);
  if (e != cudaSuccess) return e;
  gram_mirror_kernel<<<dim3((d + 31) / 32, (d + 31) / 32, ncam), dim3(32, 8), 0, st>>>(w.G, d);
  const int rows = w.rows_cap;
  cg_init_kernel<<<(rows + 7) / 8, 256, 0, st>>>(w.mu, w.mu_cam, d, w.perm, w.row_cam, rows, w.X, w.R, w.P, w.rr);
  const int iters = gcrv_iterations(lambda);
  const int vpl = (d + 127) / 128;
  split_tf32_kernel<<<152 * 8, 256, 0, st>>>(w.G, (int64_t)ncam * d * d, w.g_hi, w.g_lo);
  for (int it = 0; it < iters; ++it) {
    // Q = P (G_s + lambda n_s I) per camera block, on the tensor cores (TF32 hi + lo operands)
    split_tf32_kernel<<<152 * 8, 256, 0, st>>>(w.P, (int64_t)rows * d, w.p_hi, w.p_lo);
    e = launch_umma_mul(w.p_hi, w.p_lo, rows, w.g_hi, w.g_lo, ncam, d, w.row_cam, w.Q, st);
    if (e != cudaSuccess) return e;
    if (vpl <= 2) cg_update_kernel<2><<<(rows + 7) / 8, 256, 0, st>>>(w.X, w.R, w.P, w.Q, w.rr, w.perm, rows, d);
    else if (vpl <= 4) cg_update_kernel<4><<<(rows + 7) / 8, 256, 0, st>>>(w.X, w.R, w.P, w.Q, w.rr, w.perm, rows, d);
    else if (vpl <= 8) cg_update_kernel<8><<<(rows + 7) / 8, 256, 0, st>>>(w.X, w.R, w.P, w.Q, w.rr, w.perm, rows, d);
    else if (vpl <= 16) cg_update_kernel<16><<<(rows + 7) / 8, 256, 0, st>>>(w.X, w.R, w.P, w.Q, w.rr, w.perm, rows, d);
    else cg_update_kernel<32><<<(rows + 7) / 8, 256, 0, st>>>(w.X, w.R, w.P, w.Q, w.rr, w.perm, rows, d);
  }
  gcrv_out_kernel<<<C, 256, 0, st>>>(w.X, w.mu, d, C, cam, L, W);
  return cudaGetLastError();
}

cudaError_t launch_gcrv_means(const float* frames, int64_t F, int d, const int64_t* off, int C, float* inv, float* W,
                              cudaStream_t st) {
  frame_inv_norm_kernel<<<(unsigned)((F + 7) / 8), 256, 0, st>>>(frames, F, d, inv);
  means_kernel<<<C, 256, 0, st>>>(frames, d, off, inv, nullptr, W);
  return cudaGetLastError();
}

}  // namespace gcr
