// Certified refinement of the kNN candidate pools (exact N_i of Eq. 4 and N_i^cr of Eq. 8).
//
// The pool of row i holds its KP best GEMM scores s^_ij (descending); every score left
// out is <= the last pool entry tau. With a rigorous bound |s^_ij - s_ij| <= delta_i for
// the GEMM (FP32: gamma_d ||x_i|| max||x_j||; BF16: ||bf16(x_i)|| max||e_j|| +
// ||e_i|| max||x_j|| + gamma_acc ||bf16(x_i)|| max||bf16(x_j)||, e = bf16(x) - x) the
// refinement:
//   1. re-scores in FP32 every pool entry that could still be among the k nearest
//      (s^ >= s^_(k) - 2 delta - spread of ||x_j||^2 / 2); one warp per (row, graph), each
//      lane a d/32 slice then a butterfly, so |s~ - s| <= gamma_{d/32+6} ||x_i|| ||x_j||;
//   2. ranks by sigma = s~ - ||x_j||^2 / 2, which orders like -||x_i - x_j||^2;
//   3. certifies that no sample outside the pool can enter: sigma_(k) - eps > tau + delta -
//      min||x_j||^2 / 2; rows that fail are queued for a threshold rescan (band);
//   4. settles the k-th / (k+1)-th boundary in FP64 where FP32 cannot separate candidates;
//      exact FP64 ties go to the smaller index.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

constexpr double kU32 = 5.9604644775390625e-08;  // 2^-24
constexpr double kU32rz = 1.1920928955078125e-07; // 2^-23 (truncating accumulation)

__device__ __forceinline__ double gamma_n(double h, double u) { return h * u / (1.0 - h * u); }

// ---- warp list of 32*P entries, entry e = p*32 + lane: key sig (desc), index id, value val
template <int P>
struct WList {
  double sig[P];
  int id[P];
  double val[P];
};

template <int P>
__device__ __forceinline__ double wl_sig(const WList<P>& L, int e) {
  double r = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    double t = __shfl_sync(GCR_FULL, L.sig[p], e & 31);
    if ((e >> 5) == p) r = t;
  }
  return r;
}
template <int P>
__device__ __forceinline__ int wl_id(const WList<P>& L, int e) {
  int r = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    int t = __shfl_sync(GCR_FULL, L.id[p], e & 31);
    if ((e >> 5) == p) r = t;
  }
  return r;
}

// Descending bitonic sort of the whole list by (sig, smaller id first).
template <int P>
__device__ __forceinline__ void wl_sort(WList<P>& L, int lane) {
  constexpr int N = 32 * P;
#pragma unroll
  for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 32) {  // partner lives in the same lane: entry p ^ (stride / 32)
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int q2 = p ^ (stride >> 5);
          if (q2 > p) {
            const int s = p * 32 + lane;
            const bool desc = (s & size) == 0;
            const bool sw = desc ? better_d(L.sig[q2], L.id[q2], L.sig[p], L.id[p])
                                 : better_d(L.sig[p], L.id[p], L.sig[q2], L.id[q2]);
            if (sw) {
              double ts = L.sig[p]; L.sig[p] = L.sig[q2]; L.sig[q2] = ts;
              int ti = L.id[p]; L.id[p] = L.id[q2]; L.id[q2] = ti;
              double tv = L.val[p]; L.val[p] = L.val[q2]; L.val[q2] = tv;
            }
          }
        }
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          double os = __shfl_xor_sync(GCR_FULL, L.sig[p], stride);
          int oi = __shfl_xor_sync(GCR_FULL, L.id[p], stride);
          double ov = __shfl_xor_sync(GCR_FULL, L.val[p], stride);
          const int s = p * 32 + lane;
          const bool desc = (s & size) == 0;
          const bool lower = (s & stride) == 0;
          const bool take = (lower == desc) ? better_d(os, oi, L.sig[p], L.id[p])
                                            : better_d(L.sig[p], L.id[p], os, oi);
          if (take) { L.sig[p] = os; L.id[p] = oi; L.val[p] = ov; }
        }
      }
    }
  }
}

// Merge a sorted-descending chunk of 32 (one per lane) into a sorted list of 32P: keeps the top 32P.
template <int P>
__device__ __forceinline__ void wl_merge(WList<P>& L, double cs, int ci, double cv, int lane) {
  double rs = __shfl_sync(GCR_FULL, cs, 31 - lane);
  int ri = __shfl_sync(GCR_FULL, ci, 31 - lane);
  double rv = __shfl_sync(GCR_FULL, cv, 31 - lane);
  if (better_d(rs, ri, L.sig[P - 1], L.id[P - 1])) { L.sig[P - 1] = rs; L.id[P - 1] = ri; L.val[P - 1] = rv; }
#pragma unroll
  for (int stride = 16 * P; stride >= 32; stride >>= 1) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int q2 = p ^ (stride >> 5);
      if (q2 > p && better_d(L.sig[q2], L.id[q2], L.sig[p], L.id[p])) {
        double ts = L.sig[p]; L.sig[p] = L.sig[q2]; L.sig[q2] = ts;
        int ti = L.id[p]; L.id[p] = L.id[q2]; L.id[q2] = ti;
        double tv = L.val[p]; L.val[p] = L.val[q2]; L.val[q2] = tv;
      }
    }
  }
#pragma unroll
  for (int p = 0; p < P; ++p) {
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
      double os = __shfl_xor_sync(GCR_FULL, L.sig[p], stride);
      int oi = __shfl_xor_sync(GCR_FULL, L.id[p], stride);
      double ov = __shfl_xor_sync(GCR_FULL, L.val[p], stride);
      const bool lower = (lane & stride) == 0;
      const bool take = lower ? better_d(os, oi, L.sig[p], L.id[p]) : better_d(L.sig[p], L.id[p], os, oi);
      if (take) { L.sig[p] = os; L.id[p] = oi; L.val[p] = ov; }
    }
  }
}

__device__ __forceinline__ void sort32_d(double& s, int& i, double& v, int lane) {
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      double os = __shfl_xor_sync(GCR_FULL, s, stride);
      int oi = __shfl_xor_sync(GCR_FULL, i, stride);
      double ov = __shfl_xor_sync(GCR_FULL, v, stride);
      const bool desc = (lane & size) == 0 || size == 32;
      const bool lower = (lane & stride) == 0;
      const bool take = (lower == desc) ? better_d(os, oi, s, i) : better_d(s, i, os, oi);
      if (take) { s = os; i = oi; v = ov; }
    }
  }
}

// The row's own features x_i are not held in registers (at d = 2048 that would be 64 per lane
// and cap the resident warps of these latency-bound kernels): every dot product reads the lane's
// slice (elements v*128 + lane*4 .. +3) again, from L1 after the first time.

// FP32 dots of x_i with up to 4 rows (j < 0: skipped); sequential per-lane chain then butterfly.
// The four rows' next 128-column slices are loaded while the current ones are multiplied, so a
// lane keeps eight 16-byte loads of rows j in flight (the rescoring is bound by the latency of
// these L2 gathers, not by their bandwidth). The rows are read through L2 only, so that they do
// not evict x_i, which every dot product reads from L1.
template <int VPL>
__device__ __forceinline__ void dot4_f32(const float* __restrict__ X, int d, const float* __restrict__ xrow,
                                         const int (&j)[4], int lane, float (&out)[4]) {
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const float* rp[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) rp[t] = X + (size_t)(j[t] >= 0 ? j[t] : 0) * d + lane * 4;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 cur[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) cur[t] = (j[t] >= 0 && lane * 4 < d) ? __ldcg(reinterpret_cast<const float4*>(rp[t])) : zero;
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int off = v * 128 + lane * 4;
    float4 nxt[4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
      nxt[t] = (v + 1 < VPL && j[t] >= 0 && off + 128 < d) ? __ldcg(reinterpret_cast<const float4*>(rp[t] + (v + 1) * 128))
                                                            : zero;
    if (off < d) {
      const float4 xv = *reinterpret_cast<const float4*>(xrow + off);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (j[t] >= 0) {
          acc[t] = fmaf(xv.x, cur[t].x, acc[t]);
          acc[t] = fmaf(xv.y, cur[t].y, acc[t]);
          acc[t] = fmaf(xv.z, cur[t].z, acc[t]);
          acc[t] = fmaf(xv.w, cur[t].w, acc[t]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) cur[t] = nxt[t];
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) out[t] = warp_sum(acc[t]);
}

template <int VPL>
__device__ __forceinline__ double dot_f64(const float* __restrict__ X, int d, const float* __restrict__ xrow,
                                          int j, int lane) {
  double acc = 0.0;
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int off = v * 128 + lane * 4;
    if (off < d) {
      const float4 xv = *reinterpret_cast<const float4*>(xrow + off);
      const float4 y = *reinterpret_cast<const float4*>(X + (size_t)j * d + off);
      acc = fma((double)xv.x, (double)y.x, acc);
      acc = fma((double)xv.y, (double)y.y, acc);
      acc = fma((double)xv.z, (double)y.z, acc);
      acc = fma((double)xv.w, (double)y.w, acc);
    }
  }
  return warp_sum_d(acc);
}

// Re-scores entries [0, r) of L in FP32 (entry e's index is L.id), setting sig and val.
template <int VPL, int P>
__device__ __forceinline__ void rescore(const RefineArgs& a, const float* __restrict__ xi, WList<P>& L, int r, int lane) {
  for (int e0 = 0; e0 < r; e0 += 4) {
    int j[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = e0 + t;
      const int jj = wl_id(L, e < 32 * P ? e : 0);
      j[t] = e < r ? jj : -1;
    }
    float s[4];
    dot4_f32<VPL>(a.XB, a.d, xi, j, lane, s);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = e0 + t;
      if (e < r) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          if (e == p * 32 + lane) {
            L.val[p] = (double)s[t];
            L.sig[p] = (double)s[t] - 0.5 * a.n64B[j[t]];
          }
        }
      }
    }
  }
}

// Settles the k-th boundary of the FP32-ranked list L (sorted, r >= kk finite entries) and
// writes the kk neighbours of (row, kind) with their squared distances; pads to k.
// frow: the row's index in X (its norm n64[frow]); orow: the output row; idmap (may be NULL):
// the output index of a candidate (the ball search lists gathered positions), also the key of
// exact FP64 ties.
template <int VPL, int P>
__device__ void finalize(const RefineArgs& a, const float* __restrict__ xi, WList<P>& L, int r, int kk,
                         double eps, int frow, int orow, int kind, int lane, const int* idmap = nullptr) {
  int32_t* onbr = a.nbr[kind] + (size_t)orow * a.k;
  float* od2 = a.d2[kind] + (size_t)orow * a.k;
  const double n_i = a.n64[frow];
  int acnt = kk, zcnt = kk;
  int rank[P];
#pragma unroll
  for (int p = 0; p < P; ++p) rank[p] = 0;
  if (r > kk) {
    const double sig_next = wl_sig(L, kk);
    const double sig_k = wl_sig(L, kk - 1);
    acnt = 0;
    zcnt = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int e = p * 32 + lane;
      acnt += __popc(__ballot_sync(GCR_FULL, e < kk && L.sig[p] - eps > sig_next + eps));
      zcnt += __popc(__ballot_sync(GCR_FULL, e < r && L.sig[p] + eps >= sig_k - eps));
    }
    if (acnt < kk) {
      // FP64 for the ambiguous entries [acnt, zcnt)
      double sig64[P];
#pragma unroll
      for (int p = 0; p < P; ++p) sig64[p] = -CUDART_INF;
      for (int e = acnt; e < zcnt; ++e) {
        const int j = wl_id(L, e);
        const double dot = dot_f64<VPL>(a.XB, a.d, xi, j, lane);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          if (e == p * 32 + lane) {
            L.val[p] = dot;
            sig64[p] = dot - 0.5 * a.n64B[j];
          }
        }
      }
      // rank of each ambiguous entry among the ambiguous ones (larger sig64 first, then the
      // smaller output index)
      int key[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int me = p * 32 + lane;
        key[p] = (idmap && me >= acnt && me < zcnt) ? idmap[L.id[p]] : L.id[p];
      }
      for (int e = acnt; e < zcnt; ++e) {
        double os = -CUDART_INF;
        int oi = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const double t = __shfl_sync(GCR_FULL, sig64[p], e & 31);
          const int ti = __shfl_sync(GCR_FULL, key[p], e & 31);
          if ((e >> 5) == p) { os = t; oi = ti; }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int me = p * 32 + lane;
          if (me >= acnt && me < zcnt && me != e && better_d(os, oi, sig64[p], key[p])) ++rank[p];
        }
      }
      if (lane == 0 && a.stats) {
        atomicAdd(&a.stats[GCR_STAT_FP64_ROWS], 1ull);
        atomicAdd(&a.stats[GCR_STAT_FP64_DOTS], (unsigned long long)(zcnt - acnt));
      }
    }
  }
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int e = p * 32 + lane;
    int slot = -1;
    if (e < acnt) slot = e;
    else if (e >= acnt && e < zcnt && acnt < kk && rank[p] < kk - acnt) slot = acnt + rank[p];
    if (slot >= 0) {
      const int j = L.id[p];
      double dd = n_i + a.n64B[j] - 2.0 * L.val[p];
      onbr[slot] = idmap ? idmap[j] : j;
      od2[slot] = (float)(dd > 0.0 ? dd : 0.0);
    }
  }
  for (int s = kk + lane; s < a.k; s += 32) {
    onbr[s] = -1;
    od2[s] = CUDART_INF_F;
  }
}

template <int P>
__device__ __forceinline__ void bounds(const RefineArgs& a, int row, int vpl, double& delta, double& eps,
                                       RowScalars& sc) {
  sc = *a.sc;
  sc.bmax = sqrt(sc.nmax) * (1.0 + 1e-12);  // max ||x_j||, rounded up
  const double b_i = sqrt(a.n64[row]);
  if (a.precision == GCR_PREC_FP32) {
    delta = gamma_n((double)a.d, kU32) * b_i * sc.bmax;
  } else {
    const double ai = a.anrm[row], ei = a.enrm[row];
    delta = ai * sc.emax + ei * sc.bmax + gamma_n((double)a.d + 32.0, kU32rz) * ai * sc.amax;
  }
  delta *= 1.0 + 1e-6;
  eps = gamma_n((double)(4 * vpl + 6), kU32) * b_i * sc.bmax * (1.0 + 1e-6);
}

// One warp per (row, kind).
template <int VPL, int P>
__global__ void __launch_bounds__(256, 4) refine_pool_kernel(RefineArgs a) {
  constexpr int KP = 32 * P;
  const int lane = threadIdx.x & 31;
  const long wid = (long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (wid >= (long)a.n * a.kinds) return;
  const int kind = (int)(wid / a.n);
  const int row = a.order ? a.order[wid % a.n] : (int)(wid % a.n);
  const float* pv = a.pool_v + ((size_t)kind * a.n + row) * KP;
  const int* pi = a.pool_i + ((size_t)kind * a.n + row) * KP;
  WList<P> L;
  float pval[P];
  int mvalid = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    pval[p] = pv[p * 32 + lane];
    L.id[p] = pi[p * 32 + lane];
    L.sig[p] = -CUDART_INF;
    L.val[p] = 0.0;
    mvalid += __popc(__ballot_sync(GCR_FULL, L.id[p] >= 0));
  }
  if (lane == 0 && a.stats) atomicAdd(&a.stats[GCR_STAT_ROWS], 1ull);
  if (mvalid == 0) {
    for (int s = lane; s < a.k; s += 32) {
      a.nbr[kind][(size_t)row * a.k + s] = -1;
      a.d2[kind][(size_t)row * a.k + s] = CUDART_INF_F;
    }
    if (lane == 0 && a.stats && a.k > 0) atomicAdd(&a.stats[GCR_STAT_CLAMPED], 1ull);
    return;
  }
  const int kk = min(a.k, mvalid);
  if (kk < a.k && lane == 0 && a.stats) atomicAdd(&a.stats[GCR_STAT_CLAMPED], 1ull);
  if (kk == 0) return;
  auto pool_at = [&](int e) {
    float r = 0.f;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      float t = __shfl_sync(GCR_FULL, pval[p], e & 31);
      if ((e >> 5) == p) r = t;
    }
    return r;
  };
  const float s_k = pool_at(kk - 1);
  // bound on every approximate score left out of the pool: its last entry when full, else the
  // admission floor it was searched with (-inf: nothing was left out)
  const float fl = a.floor ? a.floor[row] : -CUDART_INF_F;
  const bool full = mvalid == KP;
  const float tau = full ? pool_at(KP - 1) : fl;
  double delta, eps;
  RowScalars sc;
  bounds<P>(a, row, VPL, delta, eps, sc);
  const double thr = (double)s_k - 2.0 * delta - 0.5 * (sc.nmax - sc.nmin);
  int r = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) r += __popc(__ballot_sync(GCR_FULL, L.id[p] >= 0 && (double)pval[p] >= thr));
  const float* xi = a.X + (size_t)row * a.d;
  rescore<VPL, P>(a, xi, L, r, lane);
  if (lane == 0 && a.stats) atomicAdd(&a.stats[GCR_STAT_RESCORED], (unsigned long long)r);
  wl_sort<P>(L, lane);
  const double sig_k = wl_sig(L, kk - 1);
  // at least kk candidates have exact sigma >= sig_k - eps: the exact k-th squared distance is at
  // most n_i - 2 (sig_k - eps) (the local scale the ball search groups rows by)
  const float dk = __double2float_ru(fmax(0.0, a.n64[row] - 2.0 * (sig_k - eps)) * (1.0 + 1e-9));
  if (a.dk_all && lane == 0) a.dk_all[(size_t)kind * a.n + row] = dk;
  if (full || fl > -CUDART_INF_F) {
    const bool cert = (sig_k - eps) > ((double)tau + delta - 0.5 * sc.nmin);
    // Saturated pool: the density of the pool's lower half, extrapolated over the band's
    // window below tau (about 2*delta wide), predicts more than 512 band entries, so the
    // rescan would overflow; it is skipped. Either way the pool's exact top k is within
    // 2*delta of the exact k-th score: every column outside the pool has s <= tau + delta,
    // every pool entry s >= tau - delta.
    const float mid = pool_at(KP / 2);
    const double dens = (KP / 2) / fmax((double)mid - (double)tau, 1e-30);
    const double below = fmax(0.0, 2.0 * delta + 0.5 * (sc.nmax - sc.nmin) - ((double)s_k - (double)tau));
    const bool dense = full && KP + dens * below > 512.0;
    const bool saturated = a.skip_saturated && dense;
    if (!cert && lane == 0) {
      if (a.stats) atomicAdd(&a.stats[GCR_STAT_UNCERTIFIED], 1ull);
      if (saturated) {
        if (a.stats) atomicAdd(&a.stats[GCR_STAT_SATURATED], 1ull);
      } else {
        const int u = atomicAdd(a.unc_count, 1);
        a.unc_row[u] = row;
        a.unc_kind[u] = kind;
        a.unc_thr[u] = __double2float_rd(sig_k - eps + 0.5 * sc.nmin - delta);
        // negative (never -0): the pair's band is predicted to overflow
        if (a.unc_dk) a.unc_dk[u] = dense ? -fmaxf(dk, 1e-30f) : dk;
      }
    }
  }
  finalize<VPL, P>(a, xi, L, r, kk, eps, row, row, kind, lane);
}

// The kk-th largest of the cnt (<= 512) band scores bv[0..cnt): an MSB-first radix select on
// their order-preserving 32-bit images, one bit per step (the same value on every lane).
__device__ __forceinline__ float band_kth(const float* __restrict__ bv, int cnt, int kk, int lane) {
  uint32_t key[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int e = i * 32 + lane;
    key[i] = e < cnt ? float_to_ordered(bv[e]) : 0u;
  }
  uint32_t prefix = 0, mask = 0;
  int need = kk;
  for (int b = 31; b >= 0; --b) {
    const uint32_t bit = 1u << b, cand = prefix | bit;
    int c = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) c += (i * 32 + lane < cnt && (key[i] & (mask | bit)) == cand) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(GCR_FULL, c, o);
    if (c >= need) prefix = cand;
    else need -= c;
    mask |= bit;
  }
  return ordered_to_float(prefix);
}

// One warp per uncertified (row, kind). The band holds every column whose approximate score
// reaches the row's threshold; of those, only the entries within 2 delta (plus the spread of
// ||x_j||^2 / 2) of the kk-th best approximate score can be among the kk nearest (the same
// rule as the pool refinement), and only they are re-scored. Capped at 85 registers (three
// blocks per SM): the band's long candidate loops gain more from resident warps than they lose
// to the few spills (measured 0.98 -> 0.80 ms per step on the cross-camera workload).
template <int VPL, int P>
__global__ void __launch_bounds__(256, 3) refine_band_kernel(RefineArgs a) {
  __shared__ int sel_ids[8][64];
  const int lane = threadIdx.x & 31;
  int* sb = sel_ids[threadIdx.x >> 5];
  const int U = *a.unc_count;
  const int nw = gridDim.x * 8;
  for (int u = blockIdx.x * 8 + (threadIdx.x >> 5); u < U; u += nw) {
    const int row = a.unc_row[u], kind = a.unc_kind[u];
    const int cnt = u < a.band_rows ? a.band_cnt[u] : a.bcap + 1;
    if (cnt > a.bcap || cnt > 512) {
      if (lane == 0 && a.stats) atomicAdd(&a.stats[GCR_STAT_BAND_FAILED], 1ull);
      continue;
    }
    double delta, eps;
    RowScalars sc;
    bounds<P>(a, row, VPL, delta, eps, sc);
    const float* xi = a.X + (size_t)row * a.d;
    WList<P> L;
#pragma unroll
    for (int p = 0; p < P; ++p) { L.sig[p] = -CUDART_INF; L.id[p] = 0x7fffffff; L.val[p] = 0.0; }
    const int* bi = a.band_i + (size_t)u * a.bcap;
    const float* bv = a.band_v + (size_t)u * a.bcap;
    const int kb = min(a.k, cnt);
    const double thr = kb > 0 ? (double)band_kth(bv, cnt, kb, lane) - 2.0 * delta - 0.5 * (sc.nmax - sc.nmin)
                              : -CUDART_INF;
    // selected entries are staged per warp (at most 31 left over + 32 new) and re-scored 32 at
    // a time
    int nsel = 0, total = 0;
    for (int c0 = 0; c0 < cnt || nsel > 0; c0 += 32) {
      if (c0 < cnt) {
        const int e = c0 + lane;
        const bool s = e < cnt && (double)bv[e] >= thr;
        const unsigned m = __ballot_sync(GCR_FULL, s);
        if (s) sb[nsel + __popc(m & ((1u << lane) - 1u))] = bi[e];
        nsel += __popc(m);
        __syncwarp();
      }
      const bool last = c0 + 32 >= cnt;
      while (nsel >= 32 || (last && nsel > 0)) {
        const int take = min(nsel, 32);
        WList<1> C;
        C.id[0] = lane < take ? sb[lane] : -1;
        C.sig[0] = -CUDART_INF;
        C.val[0] = 0.0;
        rescore<VPL, 1>(a, xi, C, take, lane);
        if (C.id[0] < 0) C.id[0] = 0x7fffffff;
        sort32_d(C.sig[0], C.id[0], C.val[0], lane);
        wl_merge<P>(L, C.sig[0], C.id[0], C.val[0], lane);
        total += take;
        const int rem = nsel - take;
        const int v = lane < rem ? sb[take + lane] : 0;
        __syncwarp();
        if (lane < rem) sb[lane] = v;
        __syncwarp();
        nsel = rem;
      }
    }
    if (lane == 0 && a.stats) atomicAdd(&a.stats[GCR_STAT_RESCORED], (unsigned long long)total);
    const int r = min(total, 32 * P);
    const int kk = min(a.k, r);
    finalize<VPL, P>(a, xi, L, r, kk, eps, row, row, kind, lane);
  }
}

// One warp per queued pair (i, graph) of the ball search. The pool of the pair's position p in
// its ball holds the best approximate sigma^ = y_p . y_j - ||y_j||^2 / 2 (y centred on the
// ball), so it ranks by distance and needs no norm-spread slack. With delta the GEMM bound over
// the ball plus the rounding of the bias and of the subtraction, the pair is certified when the
// pool holds every eligible member (not full) or sigma_(k) - eps > tau + delta; every exact
// neighbour lies in the ball, so the pool's refined top k is then N_i. Otherwise, and for pairs
// outside the searched groups, the pair goes on to the band queue with its original threshold.
template <int VPL, int P>
__device__ void refine_ball_one(const RefineArgs& a, const BallArgs& b, int u, int lane);

template <int VPL, int P>
__global__ void __launch_bounds__(256) refine_ball_kernel(RefineArgs a, BallArgs b) {
  const int lane = threadIdx.x & 31;
  const int U = min(*a.unc_count, b.unc_cap);
  for (int u = blockIdx.x * 8 + (threadIdx.x >> 5); u < U; u += gridDim.x * 8) refine_ball_one<VPL, P>(a, b, u, lane);
}

template <int VPL, int P>
__device__ void refine_ball_one(const RefineArgs& a, const BallArgs& b, int u, int lane) {
  constexpr int KP = 32 * P;
  const int i = a.unc_row[u], kind = a.unc_kind[u];
  const int p = b.pos_of_row[i];
  const int g = p >= 0 ? b.ggrp[p] : -1;
  // pairs handed on to the band rescan are flagged; a stable compaction keeps the pending
  // queue's (cluster-local) order for the rescan, whose candidate gathers then hit in L2
  auto hand_on = [&]() {
    if (lane == 0) a.bq_flag[u] = 1;
  };
  if (g < 0 || b.gfail[g] || !ball_participates(a.unc_dk[u], a.n64[i])) { hand_on(); return; }
  const float* pv = b.gpool_v + ((size_t)kind * b.cap_rows + p) * KP;
  const int* pi = b.gpool_i + ((size_t)kind * b.cap_rows + p) * KP;
  WList<P> L;
  float pval[P];
  int mvalid = 0;
#pragma unroll
  for (int q = 0; q < P; ++q) {
    pval[q] = pv[q * 32 + lane];
    L.id[q] = pi[q * 32 + lane];
    L.sig[q] = -CUDART_INF;
    L.val[q] = 0.0;
    mvalid += __popc(__ballot_sync(GCR_FULL, L.id[q] >= 0));
  }
  const int kk = min(a.k, mvalid);
  if (kk < a.k || kk == 0) { hand_on(); return; }  // the ball lacks k eligible members
  auto pool_at = [&](int e) {
    float r = 0.f;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      float t = __shfl_sync(GCR_FULL, pval[q], e & 31);
      if ((e >> 5) == q) r = t;
    }
    return r;
  };
  const float s_k = pool_at(kk - 1);
  const bool full = mvalid == KP;
  const double tau = full ? (double)pool_at(KP - 1) : -CUDART_INF;
  const RowScalars sc = b.gsc[g];
  const double bmax = sqrt(sc.nmax) * (1.0 + 1e-12);
  const double b_i = sqrt(b.n64y[p]);
  double delta;
  if (a.precision == GCR_PREC_FP32) {
    delta = gamma_n((double)a.d, kU32) * b_i * bmax;
  } else {
    const double ai = b.anrm_y[p], ei = b.enrm_y[p];
    delta = ai * sc.emax + ei * bmax + gamma_n((double)a.d + 32.0, kU32rz) * ai * sc.amax;
  }
  // the bias ||y_j||^2 / 2 is rounded to FP32, and so is the difference stored in the pool
  const double amax = a.precision == GCR_PREC_FP32 ? bmax : sc.amax;
  const double ai_ = a.precision == GCR_PREC_FP32 ? b_i : (double)b.anrm_y[p];
  delta += 2.0 * kU32 * (ai_ * amax * 1.01 + sc.nmax);
  delta *= 1.0 + 1e-6;
  const int vpl = VPL;
  const double eps = gamma_n((double)(4 * vpl + 6), kU32) * b_i * bmax * (1.0 + 1e-6);
  const double thr = (double)s_k - 2.0 * delta;
  int r = 0;
#pragma unroll
  for (int q = 0; q < P; ++q) r += __popc(__ballot_sync(GCR_FULL, L.id[q] >= 0 && (double)pval[q] >= thr));
  RefineArgs c = a;  // the ball's coordinates: centred rows and their norms, indexed by position
  c.X = b.Y;
  c.XB = b.Y;
  c.n64 = b.n64y;
  c.n64B = b.n64y;
  const float* xi = b.Y + (size_t)p * a.d;
  rescore<VPL, P>(c, xi, L, r, lane);
  if (lane == 0 && a.stats) atomicAdd(&a.stats[GCR_STAT_RESCORED], (unsigned long long)r);
  wl_sort<P>(L, lane);
  const double sig_k = wl_sig(L, kk - 1);
  if (full && !(sig_k - eps > tau + delta)) { hand_on(); return; }
  if (lane == 0 && a.stats) atomicAdd(&a.stats[GCR_STAT_BALL], 1ull);
  finalize<VPL, P>(c, xi, L, r, kk, eps, p, i, kind, lane, b.gmap);
}

// Cluster-local processing order. key(i) = the smallest index among i and its first k pool
// candidates: rows of one tight cluster share it, so a counting sort by key puts them next to
// each other and their (largely common) candidate rows are fetched from memory once.
__global__ void order_key_kernel(const int* __restrict__ pool_i, int n, int kp, int k, int* __restrict__ key,
                                 int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int m = i;
  for (int s = 0; s < k; ++s) {
    const int j = pool_i[(size_t)i * kp + s];
    if (j >= 0 && j < m) m = j;
  }
  key[i] = m;
  atomicAdd(&cnt[m], 1);
}

__global__ void order_scatter_kernel(const int* __restrict__ key, const int* __restrict__ off, int n,
                                     int* __restrict__ fill, int* __restrict__ order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = key[i];
  order[off[m] + atomicAdd(&fill[m], 1)] = i;
}

// Row gather in 16-byte units: w16 units per row.
__global__ void gather_rows_kernel(const uint4* __restrict__ src, long w16, const int* __restrict__ count,
                                   const int* __restrict__ rows, int max_rows, uint4* __restrict__ out) {
  const int U = min(*count, max_rows);
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < (long)U * w16; t += (long)gridDim.x * blockDim.x) {
    const long u = t / w16, c = t % w16;
    out[u * w16 + c] = src[(size_t)rows[u] * w16 + c];
  }
}

template <int P>
cudaError_t launch_pool_vpl(const RefineArgs& a, cudaStream_t st) {
  const long warps = (long)a.n * a.kinds;
  dim3 grid((unsigned)((warps + 7) / 8));
  const int vpl = (a.d + 127) / 128;
  if (vpl <= 1) refine_pool_kernel<1, P><<<grid, 256, 0, st>>>(a);
  else if (vpl <= 2) refine_pool_kernel<2, P><<<grid, 256, 0, st>>>(a);
  else if (vpl <= 4) refine_pool_kernel<4, P><<<grid, 256, 0, st>>>(a);
  else if (vpl <= 8) refine_pool_kernel<8, P><<<grid, 256, 0, st>>>(a);
  else if (vpl <= 16) refine_pool_kernel<16, P><<<grid, 256, 0, st>>>(a);
  else if (vpl <= 32) refine_pool_kernel<32, P><<<grid, 256, 0, st>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------- split-pool seeds
// Serving splits the gallery sweep of a query batch over many CTAs, and each split's pool starts
// empty: most of the search's time goes to filling those pools. A seed s_q lets every split
// admit only scores above it. It comes from distinct gallery rows j scored here in FP32 (the
// rows of the query's previous pool, their gallery kNN lists and, where there is no previous
// pool or it cannot supply k rows, an evenly spaced sample of the gallery, whose best scores
// bound the sweep's quantile at about (k - graph candidates) / sample from below): with valid
// such rows, V =
// min(valid, kp) and S the V-th best of their scores, each within eps of the exact dot product,
// and delta the certified bound of the GEMM's approximate scores (the same delta the refinement
// uses), V rows have an approximate score >= S - eps - delta, so the search keeps at least V
// entries above s_q = (S - eps - delta - (spread of the gallery's squared norms) / 2, rounded
// down, one ulp lower). A pool may then hold fewer than kp entries; the refinement takes s_q as
// the bound on every score left out of it and certifies (or rescans) the row as for a full
// pool. With fewer than k candidates the seed is -inf and the row is searched unseeded.
constexpr int kSeedCap = kSeedCandidates;  // candidate slots per query

// Ascending bitonic sort of n (a power of two, <= kSeedCap) values in shared memory; the block's
// threads share the compare-exchanges. KEY_DESC sorts descending instead.
template <typename T, bool DESC>
__device__ void block_bitonic(T* v, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int e = threadIdx.x; e < (n >> 1); e += blockDim.x) {
        const int lo = 2 * e - (e & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0) != DESC;
        const T a = v[lo], b = v[hi];
        if ((a > b) == up) { v[lo] = b; v[hi] = a; }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(1024) serve_seed_kernel(SeedArgs a) {
  __shared__ int cand[kSeedCap];
  __shared__ float score[kSeedCap];
  __shared__ int s_valid;
  const int q = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int per = 1 + (a.hop ? a.hop_k : 0);
  const int total1 = a.prev_kp * per;
  const int total = total1 + a.sample;
  int N = 32;
  while (N < total) N <<= 1;
  // candidates: the previous pool's rows, each followed by its hop list, then the evenly spaced
  // sample rows floor(i * ng / sample) (absent entries: INT_MAX)
  for (int e = t; e < N; e += blockDim.x) {
    int j = -1;
    if (e < total1) {
      const int p = e / per, h = e % per;
      const int j0 = a.pool_i[(size_t)q * a.prev_kp + p];
      j = h == 0 ? j0 : (j0 >= 0 && j0 < a.ng ? a.hop[(size_t)j0 * a.hop_k + h - 1] : -1);
    } else if (e < total) {
      j = (int)((long)(e - total1) * a.ng / a.sample);
    }
    cand[e] = (j >= 0 && j < a.ng) ? j : INT_MAX;
  }
  if (t == 0) s_valid = 0;
  __syncthreads();
  block_bitonic<int, false>(cand, N);
  // FP32 score of each distinct candidate (duplicates and absent slots: -inf); each warp takes
  // four candidates at a time (their row loads in flight together), each lane a sequential chain
  // over its slice, then the butterfly
  const int vpl = (a.d + 127) / 128;
  const float* x = a.xq + (size_t)q * a.d;
  int nv = 0;
  for (int e0 = warp * 4; e0 < N; e0 += (blockDim.x >> 5) * 4) {
    int j[4];
    bool ok[4];
    float acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int e = e0 + c;
      j[c] = cand[e];
      ok[c] = j[c] != INT_MAX && (e == 0 || cand[e - 1] != j[c]);
      acc[c] = 0.f;
    }
    for (int v = 0; v < vpl; ++v) {
      const int off = v * 128 + lane * 4;
      if (off < a.d) {
        const float4 xv = *reinterpret_cast<const float4*>(x + off);
        float4 gv[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          gv[c] = ok[c] ? *reinterpret_cast<const float4*>(a.G + (size_t)j[c] * a.d + off) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[c] = fmaf(xv.x, gv[c].x, acc[c]);
          acc[c] = fmaf(xv.y, gv[c].y, acc[c]);
          acc[c] = fmaf(xv.z, gv[c].z, acc[c]);
          acc[c] = fmaf(xv.w, gv[c].w, acc[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[c] = warp_sum(acc[c]);
      nv += ok[c] ? 1 : 0;
      if (lane == 0) score[e0 + c] = ok[c] ? acc[c] : -CUDART_INF_F;
    }
  }
  if (lane == 0 && nv) atomicAdd(&s_valid, nv);
  __syncthreads();
  const int valid = s_valid;
  block_bitonic<float, true>(score, N);
  if (t != 0) return;
  if (valid < a.k || a.k < 1) {
    a.seed[q] = -CUDART_INF_F;
    return;
  }
  RowScalars sc = *a.gsc;
  const double bmax = sqrt(sc.nmax) * (1.0 + 1e-12);
  const double b_i = sqrt(a.n64q[q]);
  double delta;
  if (a.precision == GCR_PREC_FP32) {
    delta = gamma_n((double)a.d, kU32) * b_i * bmax;
  } else {
    const double ai = a.anrm[q], ei = a.enrm[q];
    delta = ai * sc.emax + ei * bmax + gamma_n((double)a.d + 32.0, kU32rz) * ai * sc.amax;
  }
  delta *= 1.0 + 1e-6;
  const double eps = gamma_n((double)(4 * vpl + 6), kU32) * b_i * bmax * (1.0 + 1e-6);
  // below the approximate score of each of the best V candidates (their exact scores are within
  // eps of these, their approximate ones within delta of the exact), with the spread of the
  // gallery's squared norms as slack for ranking by distance rather than by score
  const int V = valid < a.kp ? valid : a.kp;
  const double th = (double)score[V - 1] - eps - delta - 0.5 * (sc.nmax - sc.nmin);
  a.seed[q] = nextafterf(__double2float_rd(th), -CUDART_INF_F);
}

cudaError_t launch_serve_seed(const SeedArgs& a, cudaStream_t st) {
  const long total = (long)a.prev_kp * (1 + (a.hop ? a.hop_k : 0)) + a.sample;
  if (total > kSeedCap || total < 1 || a.prev_kp < 0 || (a.prev_kp > 0 && !a.pool_i) || a.kp < 1 || a.k < 1 ||
      a.k > a.kp || a.b < 1 || a.sample < 0 || a.sample > a.ng)
    return cudaErrorInvalidValue;
  serve_seed_kernel<<<a.b, 1024, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_refine_pool(const RefineArgs& a, cudaStream_t st) {
  if (a.kp == 32) return launch_pool_vpl<1>(a, st);
  if (a.kp == 64) return launch_pool_vpl<2>(a, st);
  if (a.kp == 128) return launch_pool_vpl<4>(a, st);
  return cudaErrorInvalidValue;
}

template <int P>
cudaError_t launch_band_p(const RefineArgs& a, cudaStream_t st) {
  dim3 grid(152 * 4);
  const int vpl = (a.d + 127) / 128;
  if (vpl <= 1) refine_band_kernel<1, P><<<grid, 256, 0, st>>>(a);
  else if (vpl <= 2) refine_band_kernel<2, P><<<grid, 256, 0, st>>>(a);
  else if (vpl <= 4) refine_band_kernel<4, P><<<grid, 256, 0, st>>>(a);
  else if (vpl <= 8) refine_band_kernel<8, P><<<grid, 256, 0, st>>>(a);
  else if (vpl <= 16) refine_band_kernel<16, P><<<grid, 256, 0, st>>>(a);
  else if (vpl <= 32) refine_band_kernel<32, P><<<grid, 256, 0, st>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_ball_vpl(const RefineArgs& a, const BallArgs& b, cudaStream_t st) {
  // one block per SM (the kernel's registers allow no more); warps stride over the pending pairs
  dim3 grid((unsigned)std::min((b.unc_cap + 7) / 8, 152));
  const int vpl = (a.d + 127) / 128;
  if (vpl <= 1) refine_ball_kernel<1, P><<<grid, 256, 0, st>>>(a, b);
  else if (vpl <= 2) refine_ball_kernel<2, P><<<grid, 256, 0, st>>>(a, b);
  else if (vpl <= 4) refine_ball_kernel<4, P><<<grid, 256, 0, st>>>(a, b);
  else if (vpl <= 8) refine_ball_kernel<8, P><<<grid, 256, 0, st>>>(a, b);
  else if (vpl <= 16) refine_ball_kernel<16, P><<<grid, 256, 0, st>>>(a, b);
  else if (vpl <= 32) refine_ball_kernel<32, P><<<grid, 256, 0, st>>>(a, b);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

__global__ void hand_on_kernel(RefineArgs a, int cap) {
  const int U = min(*a.unc_count, cap);
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x) {
    if (!a.bq_flag[u]) continue;
    const int v = a.bq_pos[u];
    a.bq_row[v] = a.unc_row[u];
    a.bq_kind[v] = a.unc_kind[u];
    a.bq_thr[v] = a.unc_thr[u];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.bq_count = a.bq_pos[cap];
}

cudaError_t launch_refine_ball(const RefineArgs& a, const BallArgs& b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.bq_flag, 0, sizeof(int) * b.unc_cap, st);
  if (e != cudaSuccess) return e;
  if (a.kp == 32) e = launch_ball_vpl<1>(a, b, st);
  else if (a.kp == 64) e = launch_ball_vpl<2>(a, b, st);
  else if (a.kp == 128) e = launch_ball_vpl<4>(a, b, st);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  e = launch_scan(a.bq_flag, a.bq_pos, b.unc_cap, st);
  if (e != cudaSuccess) return e;
  hand_on_kernel<<<std::min((b.unc_cap + 255) / 256, 152 * 4), 256, 0, st>>>(a, b.unc_cap);
  return cudaGetLastError();
}

cudaError_t launch_refine_band(const RefineArgs& a, cudaStream_t st) {
  return a.k >= 64 ? launch_band_p<4>(a, st) : launch_band_p<2>(a, st);
}

cudaError_t launch_row_order(const int* pool_i, int n, int kp, int k, int* key, int* cnt, int* off, int* fill,
                             int* order, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(fill, 0, sizeof(int) * n, st);
  if (e != cudaSuccess) return e;
  order_key_kernel<<<(n + 255) / 256, 256, 0, st>>>(pool_i, n, kp, k, key, cnt);
  e = launch_scan(cnt, off, n, st);
  if (e != cudaSuccess) return e;
  order_scatter_kernel<<<(n + 255) / 256, 256, 0, st>>>(key, off, n, fill, order);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const void* src, size_t row_bytes, const int* count, const int* rows,
                               int max_rows, void* out, cudaStream_t st) {
  if (row_bytes % 16) return cudaErrorInvalidValue;
  gather_rows_kernel<<<152 * 4, 256, 0, st>>>(static_cast<const uint4*>(src), (long)(row_bytes / 16), count, rows,
                                              max_rows, static_cast<uint4*>(out));
  return cudaGetLastError();
}

}  // namespace gcr
