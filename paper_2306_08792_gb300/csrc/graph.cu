// Affinity weights, degrees and the propagation operator (Eq. 4-9).
//
// From the kNN lists (ELL: row i lists N_i) this builds, per graph (global, cross-camera):
//   w_ij = exp(-||x_i - x_j||^2 / gamma) for j in N_i        (Eq. 4 / Eq. 8; A~_ii = 1)
//   D_r(i) = 1 + sum_{j in N_i} w_ij,  D_c(j) = 1 + sum_{i: j in N_i} w_ij       (Eq. 5)
// and then one CSR matrix M_mix that a propagation layer applies:
//   symmetric (Eq. 7, Eq. 2): M = D^{-1/2} (A~ + A~^T)/2 D^{-1/2}, D = (D_r + D_c)/2
//   asymmetric (Eq. 6):       M = D_r^{-1/2} A~ D_c^{-1/2}
//   M_mix = alpha M + (1 - alpha) M^cr (Eq. 9); alpha = 1 without the cross-camera graph.
// The transpose A~^T is built by a counting sort whose segments are then sorted by source
// row, so every sum (degrees, operator rows) runs in a fixed order: results are
// bit-reproducible run to run. Operator rows are sorted by column with duplicate columns
// (mutual neighbours, overlapping graphs) merged into one entry.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

__global__ void weights_kernel(int n, int k, float gamma, const int32_t* __restrict__ nbr,
                               const float* __restrict__ d2, float* __restrict__ w,
                               float* __restrict__ deg_r, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 1.0f;  // A~_ii = 1
  for (int s = 0; s < k; ++s) {
    const int j = nbr[(size_t)i * k + s];
    float wij = 0.f;
    if (j >= 0) {
      wij = expf(-d2[(size_t)i * k + s] / gamma);
      atomicAdd(&cnt[j], 1);
    }
    w[(size_t)i * k + s] = wij;
    acc += wij;
  }
  deg_r[i] = acc;
}

// Exclusive scan of in[0, n) into out[0, n] (out[n] = total), one block of 1024 threads,
// tiles of 8,192 elements with a running carry: each tile is read with coalesced loads (all 8
// per thread in flight) into shared memory, each thread then takes 8 consecutive elements from
// there (padded against bank conflicts), scans them, and the block combines the threads' sums.
constexpr int kScanPer = 8;
constexpr int kScanTile = 1024 * kScanPer;
__device__ __forceinline__ int scan_pad(int i) { return i + (i >> 5); }
__global__ void __launch_bounds__(1024) scan_kernel(const int* __restrict__ in, int* __restrict__ out, int n) {
  __shared__ int tile[kScanTile + kScanTile / 32];
  __shared__ int wsum[32];
  __shared__ int carry_s;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) carry_s = 0;
  for (int base = 0; base < n; base += kScanTile) {
    int ld[kScanPer];
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
      const int idx = base + e * 1024 + tid;
      ld[e] = idx < n ? in[idx] : 0;
    }
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) tile[scan_pad(e * 1024 + tid)] = ld[e];
    __syncthreads();
    int v[kScanPer];
    int loc = 0;
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
      v[e] = tile[scan_pad(tid * kScanPer + e)];
      loc += v[e];
    }
    int incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(GCR_FULL, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      int s = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(GCR_FULL, s, o);
        if (lane >= o) s += t;
      }
      wsum[lane] = s;
    }
    __syncthreads();
    int run = carry_s + (w > 0 ? wsum[w - 1] : 0) + incl - loc;
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
      tile[scan_pad(tid * kScanPer + e)] = run;
      run += v[e];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
      const int idx = base + e * 1024 + tid;
      if (idx < n) out[idx] = tile[scan_pad(e * 1024 + tid)];
    }
    if (tid == 1023) carry_s = run;
    __syncthreads();
  }
  if (tid == 0) out[n] = carry_s;
}

__global__ void scatter_kernel(int n, int k, const int32_t* __restrict__ nbr, const float* __restrict__ w,
                               const int* __restrict__ tptr, int* __restrict__ fill,
                               int* __restrict__ src_tmp, float* __restrict__ w_tmp) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)n * k) return;
  const int i = (int)(t / k);
  const int j = nbr[t];
  if (j < 0) return;
  const int pos = tptr[j] + atomicAdd(&fill[j], 1);
  src_tmp[pos] = i;
  w_tmp[pos] = w[t];
}

// Sorting 64-bit keys held P per lane (element e = p*32 + lane), ascending, payload float.
template <int P>
__device__ __forceinline__ void warp_sort_keys(unsigned long long (&key)[P], float (&pay)[P], int lane) {
  constexpr int N = 32 * P;
#pragma unroll
  for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 32) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int q = p ^ (stride >> 5);
          if (q > p) {
            const int s = p * 32 + lane;
            const bool asc = (s & size) == 0;
            const bool sw = asc ? key[q] < key[p] : key[q] > key[p];
            if (sw) {
              unsigned long long tk = key[p]; key[p] = key[q]; key[q] = tk;
              float tp = pay[p]; pay[p] = pay[q]; pay[q] = tp;
            }
          }
        }
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const unsigned long long ok = __shfl_xor_sync(GCR_FULL, key[p], stride);
          const float op = __shfl_xor_sync(GCR_FULL, pay[p], stride);
          const int s = p * 32 + lane;
          const bool asc = (s & size) == 0;
          const bool lower = (s & stride) == 0;
          const bool take = (lower == asc) ? ok < key[p] : ok > key[p];
          if (take) { key[p] = ok; pay[p] = op; }
        }
      }
    }
  }
}

// Sort one transposed segment by source row (register bitonic for <= 32*P entries).
template <int P>
__device__ void tseg_sort_regs(int beg, int len, const int* __restrict__ src_tmp, const float* __restrict__ w_tmp,
                               int* __restrict__ src, float* __restrict__ tw, int lane) {
  unsigned long long key[P];
  float pay[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int e = p * 32 + lane;
    key[p] = e < len ? (unsigned long long)(unsigned)src_tmp[beg + e] : ~0ull;
    pay[p] = e < len ? w_tmp[beg + e] : 0.f;
  }
  warp_sort_keys<P>(key, pay, lane);
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int e = p * 32 + lane;
    if (e < len) { src[beg + e] = (int)key[p]; tw[beg + e] = pay[p]; }
  }
}

constexpr int kLongSeg = 256;  // longer transposed segments (in-degree hubs) go to tsort_long_kernel

// One warp per transposed row j: sort its entries by source, then D_c(j) = 1 + sum.
__global__ void tsort_kernel(int n, const int* __restrict__ tptr, const int* __restrict__ src_tmp,
                             const float* __restrict__ w_tmp, int* __restrict__ src, float* __restrict__ tw,
                             float* __restrict__ deg_c) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  const int beg = tptr[j], len = tptr[j + 1] - beg;
  if (len <= 32) tseg_sort_regs<1>(beg, len, src_tmp, w_tmp, src, tw, lane);
  else if (len <= 64) tseg_sort_regs<2>(beg, len, src_tmp, w_tmp, src, tw, lane);
  else if (len <= 128) tseg_sort_regs<4>(beg, len, src_tmp, w_tmp, src, tw, lane);
  else if (len <= kLongSeg) tseg_sort_regs<8>(beg, len, src_tmp, w_tmp, src, tw, lane);
  else return;  // a hub's long segment: tsort_long_kernel sorts it and sets its D_c
  __syncwarp();
  if (lane == 0) {
    float acc = 1.0f;  // A~_jj = 1
    for (int e = 0; e < len; ++e) acc += tw[beg + e];
    deg_c[j] = acc;
  }
}

// Transposed rows longer than kLongSeg, listed in arbitrary order (each is processed on its own).
__global__ void long_list_kernel(int n, const int* __restrict__ tptr, int* __restrict__ list, int* __restrict__ count) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  if (tptr[j + 1] - tptr[j] > kLongSeg) list[atomicAdd(count, 1)] = j;
}

// One CTA per long transposed segment (a persistent loop over the list): a stable LSD radix
// sort of the segment by source row (8-bit digits, nbits = bits of the largest row index),
// chunk by chunk through global memory in segment order, so the work is linear in the
// segment's length (an in-degree hub can hold tens of thousands of entries). Within a chunk
// each warp ranks its keys slot by slot (lanes with equal digits found by ballots); a running
// per-digit offset carries the order from chunk to chunk. The weights follow their keys. Then D_c(j) = 1 + sum
// of the weights, reduced in a fixed order.
template <int IPT>
__global__ void __launch_bounds__(256) tsort_long_kernel(const int* __restrict__ tptr, int* src_tmp, float* w_tmp,
                                                         int* src, float* tw, float* __restrict__ deg_c,
                                                         const int* __restrict__ list, const int* __restrict__ count,
                                                         int nbits) {
  constexpr int NT = 256, NW = NT / 32, CH = NT * IPT;
  __shared__ uint32_t dbase[256];       // running offset of each digit in the segment
  __shared__ uint32_t wcnt[NW][257];    // per-warp digit counts of a chunk (column 256: past the end)
  __shared__ float red[NW];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int total = *count;
  for (int li = blockIdx.x; li < total; li += gridDim.x) {
    const int j = list[li];
    const int beg = tptr[j], L = tptr[j + 1] - beg;
    int* ka = src_tmp + beg;
    float* va = w_tmp + beg;
    int* kb = src + beg;
    float* vb = tw + beg;
    for (int shift = 0; shift < nbits; shift += 8) {
      for (int v = t; v < 256; v += NT) dbase[v] = 0;
      __syncthreads();
      for (int e = t; e < L; e += NT) atomicAdd(&dbase[((uint32_t)ka[e] >> shift) & 255u], 1u);
      __syncthreads();
      if (w == 0) {  // exclusive scan of the 256 digit counts
        uint32_t c[8], sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) { c[q] = dbase[lane * 8 + q]; sum += c[q]; }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(GCR_FULL, inc, o);
          if (lane >= o) inc += y;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int q = 0; q < 8; ++q) { dbase[lane * 8 + q] = run; run += c[q]; }
      }
      __syncthreads();
      for (int c0 = 0; c0 < L; c0 += CH) {
        for (int v = t; v < NW * 257; v += NT) (&wcnt[0][0])[v] = 0;
        __syncthreads();
        uint32_t key[IPT], off[IPT], dg[IPT];
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
          const int e = c0 + w * 32 * IPT + i * 32 + lane;
          key[i] = e < L ? (uint32_t)ka[e] : 0u;
          dg[i] = e < L ? ((key[i] >> shift) & 255u) : 256u;
          const unsigned peers = warp_peers(dg[i], 9);  // digits 0..256 (256: past the end)
          const uint32_t base = wcnt[w][dg[i]];
          __syncwarp();
          if ((peers & lt) == 0) wcnt[w][dg[i]] = base + (uint32_t)__popc(peers);  // the lowest peer updates
          __syncwarp();
          off[i] = base + (uint32_t)__popc(peers & lt);
        }
        __syncthreads();
        {  // digit t: offsets of each warp's keys in (digit, warp) order, then the running base
          uint32_t run = dbase[t];
#pragma unroll
          for (int ww = 0; ww < NW; ++ww) {
            const uint32_t cc = wcnt[ww][t];
            wcnt[ww][t] = run;
            run += cc;
          }
          dbase[t] = run;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
          const int e = c0 + w * 32 * IPT + i * 32 + lane;
          if (e < L) {
            const uint32_t dst = wcnt[w][dg[i]] + off[i];
            kb[dst] = (int)key[i];
            vb[dst] = va[e];
          }
        }
        __syncthreads();
      }
      int* tk = ka; ka = kb; kb = tk;
      float* tv = va; va = vb; vb = tv;
    }
    if (ka != src + beg) {  // an even number of passes leaves the result in the scratch
      for (int e = t; e < L; e += NT) { src[beg + e] = ka[e]; tw[beg + e] = va[e]; }
      __syncthreads();
    }
    float sum = 0.f;
    for (int e = t; e < L; e += NT) sum += tw[beg + e];
    sum = warp_sum(sum);
    if (lane == 0) red[w] = sum;
    __syncthreads();
    if (t == 0) {
      float acc = 1.0f;  // A~_jj = 1
      for (int ww = 0; ww < NW; ++ww) acc += red[ww];
      deg_c[j] = acc;
    }
    __syncthreads();
  }
}

struct OpArgs {
  int n, k, kinds, symmetric;
  float coef[2];          // alpha, 1 - alpha
  const int32_t* nbr[2];
  const float* w[2];
  const float* deg_r[2];
  const float* deg_c[2];
  const int* tptr[2];
  const int* tsrc[2];
  const float* tw[2];
  const double* inv_r[2];  // per graph: 1/sqrt(D_i) (Eq. 7, D the mean of row and column
  const double* inv_c[2];  // degrees) in both, or 1/sqrt(D_r,i) and 1/sqrt(D_c,i) (Eq. 6)
  const int* rowptr;
  int* len;
  int* col;
  float* val;
  int* raw_col;
  float* raw_val;
};

// Inverse square roots of the degrees, once per row and graph (FP64): every operator entry
// is then a product, without a square root or division per entry.
__global__ void inv_sqrt_degree_kernel(int n, int symmetric, const float* __restrict__ deg_r,
                                       const float* __restrict__ deg_c, double* __restrict__ inv_r,
                                       double* __restrict__ inv_c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (symmetric) {
    const double r = 1.0 / sqrt(0.5 * ((double)deg_r[i] + (double)deg_c[i]));
    inv_r[i] = r;
    inv_c[i] = r;
  } else {
    inv_r[i] = 1.0 / sqrt((double)deg_r[i]);
    inv_c[i] = 1.0 / sqrt((double)deg_c[i]);
  }
}

__global__ void op_count_kernel(OpArgs a, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  int c = 1;
  for (int g = 0; g < a.kinds; ++g) {
    c += a.k;
    if (a.symmetric) c += a.tptr[g][i + 1] - a.tptr[g][i];
  }
  cnt[i] = c;
}

// Raw entries of operator row i in a fixed generation order: self, then per graph its
// N_i entries (rank order) and, when symmetric, its transposed entries (by source).
__device__ __forceinline__ void gen_entry(const OpArgs& a, int i, int e, int& col, double& v) {
  // e == 0: self loop
  // self loop: A~_ii = 1, scaled by 1/D_i (Eq. 7) or 1/sqrt(D_r,i D_c,i) (Eq. 6)
  if (e == 0) {
    double s = 0.0;
    for (int g = 0; g < a.kinds; ++g) s += a.coef[g] * (a.inv_r[g][i] * a.inv_c[g][i]);
    col = i;
    v = s;
    return;
  }
  const double half = a.symmetric ? 0.5 : 1.0;  // (A~ + A~^T) / 2 in Eq. 7
  int r = e - 1;
  for (int g = 0; g < a.kinds; ++g) {
    if (r < a.k) {
      const int j = a.nbr[g][(size_t)i * a.k + r];
      const double wij = a.w[g][(size_t)i * a.k + r];
      if (j < 0) { col = -1; v = 0.0; return; }
      col = j;
      v = a.coef[g] * half * wij * (a.inv_r[g][i] * a.inv_c[g][j]);
      return;
    }
    r -= a.k;
    if (a.symmetric) {
      const int tb = a.tptr[g][i], tl = a.tptr[g][i + 1] - tb;
      if (r < tl) {
        const int s = a.tsrc[g][tb + r];
        const double wsi = a.tw[g][tb + r];
        col = s;
        v = a.coef[g] * 0.5 * wsi * (a.inv_r[g][i] * a.inv_c[g][s]);
        return;
      }
      r -= tl;
    }
  }
  col = -1;
  v = 0.0;
}

template <int P>
__device__ void op_row_regs(const OpArgs& a, int i, int beg, int L, int lane) {
  unsigned long long key[P];
  float pay[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int e = p * 32 + lane;
    int c = -1;
    double v = 0.0;
    if (e < L) gen_entry(a, i, e, c, v);
    // key: column, then generation position (invalid entries sort last)
    key[p] = c >= 0 ? (((unsigned long long)(unsigned)c << 32) | (unsigned)e) : ~0ull;
    pay[p] = (float)v;
  }
  warp_sort_keys<P>(key, pay, lane);
  // stage sorted entries in the raw buffer, then merge runs of equal columns
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int e = p * 32 + lane;
    if (e < L) {
      a.raw_col[beg + e] = key[p] == ~0ull ? -1 : (int)(key[p] >> 32);
      a.raw_val[beg + e] = pay[p];
    }
  }
  __syncwarp();
  int written = 0;
  for (int e0 = 0; e0 < L; e0 += 32) {
    const int e = e0 + lane;
    int c = e < L ? a.raw_col[beg + e] : -1;
    const bool head = c >= 0 && (e == 0 || a.raw_col[beg + e - 1] != c);
    float v = 0.f;
    if (head) {
      v = a.raw_val[beg + e];
      for (int f = e + 1; f < L && a.raw_col[beg + f] == c; ++f) v += a.raw_val[beg + f];
    }
    const unsigned hm = __ballot_sync(GCR_FULL, head);
    if (head) {
      const int pos = written + __popc(hm & ((1u << lane) - 1));
      a.col[beg + pos] = c;
      a.val[beg + pos] = v;
    }
    written += __popc(hm);
  }
  if (lane == 0) a.len[i] = written;
}

// One warp per operator row.
__global__ void op_fill_kernel(OpArgs a) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= a.n) return;
  const int beg = a.rowptr[i], L = a.rowptr[i + 1] - beg;
  if (L <= 32) op_row_regs<1>(a, i, beg, L, lane);
  else if (L <= 64) op_row_regs<2>(a, i, beg, L, lane);
  else if (L <= 128) op_row_regs<4>(a, i, beg, L, lane);
  else if (L <= 256) op_row_regs<8>(a, i, beg, L, lane);
  else {
    // very long row (hub): keep the entries unmerged, in generation order
    int written = 0;
    for (int e0 = 0; e0 < L; e0 += 32) {
      const int e = e0 + lane;
      int c = -1;
      double v = 0.0;
      if (e < L) gen_entry(a, i, e, c, v);
      const unsigned hm = __ballot_sync(GCR_FULL, c >= 0);
      if (c >= 0) {
        const int pos = written + __popc(hm & ((1u << lane) - 1));
        a.col[beg + pos] = c;
        a.val[beg + pos] = (float)v;
      }
      written += __popc(hm);
    }
    if (lane == 0) a.len[i] = written;
  }
}

}  // namespace

cudaError_t launch_scan(const int* in, int* out, int n, cudaStream_t st) {
  scan_kernel<<<1, 1024, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

namespace {

// The transposes of the two graphs are independent until the operator is assembled: the
// cross-camera graph's is built on a second stream (forked from and joined back into the
// caller's stream by events, so the pattern also holds under stream capture). One side stream
// per device; the mutex keeps a call's fork, side work and join together, since an event wait
// binds to the event's last record at the time it is enqueued.
constexpr int kMaxGraphDevices = 64;
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
SideStream g_side[kMaxGraphDevices];
std::mutex g_side_mu;

cudaError_t transpose_graph(const GraphArgs& g, int q, int* raw_col, float* raw_val, int* scan_tmp, int* long_list,
                            int* long_count, cudaStream_t st) {
  const int n = g.n, k = g.k;
  cudaError_t e = cudaMemsetAsync(g.cnt[q], 0, sizeof(int) * (n + 1), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(g.fill[q], 0, sizeof(int) * n, st);
  if (e != cudaSuccess) return e;
  weights_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, k, g.gamma, g.nbr[q], g.d2[q], g.w[q], g.deg_r[q], g.cnt[q]);
  // exclusive scan of the in-degree counts: transposed row pointers (into scan_tmp, copied back)
  scan_kernel<<<1, 1024, 0, st>>>(g.cnt[q], scan_tmp, n);
  e = cudaMemcpyAsync(g.cnt[q], scan_tmp, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  if ((long)n * k > 0) {
    // unsorted transpose into raw buffers, then sorted into t_src / t_w
    scatter_kernel<<<(unsigned)(((long)n * k + 255) / 256), 256, 0, st>>>(n, k, g.nbr[q], g.w[q], g.cnt[q],
                                                                         g.fill[q], raw_col, raw_val);
  }
  tsort_kernel<<<(n + 7) / 8, 256, 0, st>>>(n, g.cnt[q], raw_col, raw_val, g.t_src[q], g.t_w[q], g.deg_c[q]);
  e = cudaMemsetAsync(long_count, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  long_list_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, g.cnt[q], long_list, long_count);
  int nbits = 0;
  while (nbits < 31 && ((long)1 << nbits) < (long)n) ++nbits;
  tsort_long_kernel<8><<<2 * 152, 256, 0, st>>>(g.cnt[q], raw_col, raw_val, g.t_src[q], g.t_w[q], g.deg_c[q],
                                                long_list, long_count, nbits);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_build_operator(const GraphArgs& g, cudaStream_t st) {
  const int n = g.n, k = g.k;
  cudaError_t e;
  if (g.kinds == 1) {
    e = transpose_graph(g, 0, g.op_col, g.op_val, g.scan_tmp, g.long_list, g.long_count, st);
    if (e != cudaSuccess) return e;
  } else {
    // graph 0 on the caller's stream with the operator's buffers as scratch; graph 1 on the side
    // stream with the raw buffers (unused until the operator is filled) and its own scan
    // temporary and hub list
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxGraphDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_side_mu);
    SideStream& ss = g_side[dev];
    if (!ss.s) {
      e = cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    e = cudaEventRecord(ss.fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss.s, ss.fork, 0);
    if (e != cudaSuccess) return e;
    e = transpose_graph(g, 1, g.raw_col, g.raw_val, g.scan_tmp2, g.long_list2, g.long_count + 1, ss.s);
    if (e != cudaSuccess) return e;
    e = transpose_graph(g, 0, g.op_col, g.op_val, g.scan_tmp, g.long_list, g.long_count, st);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ss.join, ss.s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ss.join, 0);
    if (e != cudaSuccess) return e;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  OpArgs a;
  a.n = n; a.k = k; a.kinds = g.kinds; a.symmetric = g.symmetric;
  a.coef[0] = g.kinds == 2 ? g.alpha : 1.0f;
  a.coef[1] = 1.0f - g.alpha;
  for (int q = 0; q < 2; ++q) {
    const int qq = q < g.kinds ? q : 0;
    a.nbr[q] = g.nbr[qq]; a.w[q] = g.w[qq]; a.deg_r[q] = g.deg_r[qq]; a.deg_c[q] = g.deg_c[qq];
    a.tptr[q] = g.cnt[qq]; a.tsrc[q] = g.t_src[qq]; a.tw[q] = g.t_w[qq];
    a.inv_r[q] = g.inv + (size_t)(2 * qq) * n;
    a.inv_c[q] = g.inv + (size_t)(2 * qq + 1) * n;
  }
  for (int q = 0; q < g.kinds; ++q)
    inv_sqrt_degree_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, g.symmetric, g.deg_r[q], g.deg_c[q],
                                                            g.inv + (size_t)(2 * q) * n,
                                                            g.inv + (size_t)(2 * q + 1) * n);
  a.rowptr = g.op_rowptr; a.len = g.op_len; a.col = g.op_col; a.val = g.op_val;
  a.raw_col = g.raw_col; a.raw_val = g.raw_val;
  op_count_kernel<<<(n + 255) / 256, 256, 0, st>>>(a, g.op_cnt);
  scan_kernel<<<1, 1024, 0, st>>>(g.op_cnt, g.op_rowptr, n);
  op_fill_kernel<<<(n + 7) / 8, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace gcr
