// Segmented sort of the re-ranked distances (one segment per query).
//
// Each query's gallery distances are ranked ascending with ties broken by the smaller gallery
// index, and the first K (index, distance) pairs are written out. One CTA per query sorts the
// whole segment (up to 16384 keys):
//  * segments of 2048 keys and more: a stable LSD radix sort of the order-preserving 32-bit
//    images of the distances taken relative to the segment's smallest, in 8-bit digit passes
//    over the bits that range needs, or three 9-bit passes when it needs 25 to 27 bits (the
//    usual case for one query's distances). Keys start in gallery-index order and every pass is
//    stable, so equal distances stay in index order. Each thread keeps 16 keys in registers in
//    a warp-striped layout (key e = (warp*16 + slot)*32 + lane); per pass a warp ranks its keys
//    slot by slot (peers with the same digit found by ballots, ranked by lane), per-warp
//    digit counts go to shared memory, one block-wide scan in (digit, warp) order gives every
//    key its destination, and keys and gallery indices are scattered to shared memory (the
//    indices stay there, double-buffered; the keys are reloaded into registers).
//  * shorter segments: a bitonic network on 64-bit keys (distance image, index) whose data stay
//    in registers: each thread holds E consecutive keys, so strides below E are exchanged
//    inside a thread, strides below 32E through warp shuffles, and only the strides of 32E and
//    more go through shared memory.
#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

constexpr int kMaxSeg = 16384;

__device__ __forceinline__ void cmp_swap(unsigned long long& lo, unsigned long long& hi, bool asc) {
  const bool sw = asc ? (lo > hi) : (lo < hi);
  if (sw) {
    const unsigned long long t = lo;
    lo = hi;
    hi = t;
  }
}

// In-thread stage with a compile-time stride (keeps the key array in registers).
template <int E, int S>
__device__ __forceinline__ void reg_stage(unsigned long long (&key)[E], int base, int size) {
  if constexpr (S < E) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int j = i ^ S;
      if (j > i) cmp_swap(key[i], key[j], ((base + i) & size) == 0);
    }
  }
}

// Shared-memory position of key e: one padding word every 32 keys, so that the blocked
// (E consecutive keys per thread) and the strided access patterns both avoid bank conflicts.
__device__ __forceinline__ int pad(int e) { return e + (e >> 5); }

template <int E>
__global__ void __launch_bounds__(1024) rank_rows_kernel(const float* __restrict__ D, int ng, int N, int K,
                                                          int32_t* __restrict__ idx_out, float* __restrict__ dist_out) {
  extern __shared__ unsigned long long sk[];
  const int q = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, T = blockDim.x;
  const int base = t * E;
  const float* row = D + (size_t)q * ng;
  // coalesced load into shared memory, then E consecutive keys per thread into registers
  for (int e = t; e < N; e += T)
    sk[pad(e)] = e < ng ? (((unsigned long long)float_to_ordered(row[e]) << 32) | (unsigned)e) : ~0ull;
  __syncthreads();
  unsigned long long key[E];
#pragma unroll
  for (int i = 0; i < E; ++i) key[i] = sk[pad(base + i)];
  __syncthreads();
  const int wide = 32 * E;  // strides at or above this cross warps
  bool in_smem = false;
  for (int size = 2; size <= N; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= wide) {
        if (!in_smem) {
#pragma unroll
          for (int i = 0; i < E; ++i) sk[pad(base + i)] = key[i];
          __syncthreads();
          in_smem = true;
        }
        for (int p = t; p < (N >> 1); p += T) {
          const int lo = 2 * p - (p & (stride - 1));
          const int hi = lo + stride;
          unsigned long long a = sk[pad(lo)], b = sk[pad(hi)];
          cmp_swap(a, b, (lo & size) == 0);
          sk[pad(lo)] = a;
          sk[pad(hi)] = b;
        }
        __syncthreads();
      } else {
        if (in_smem) {
#pragma unroll
          for (int i = 0; i < E; ++i) key[i] = sk[pad(base + i)];
          __syncthreads();
          in_smem = false;
        }
        if (stride >= E) {
          const int ld = stride / E;  // partner lane distance
          const bool lower = (lane & ld) == 0;
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const unsigned long long o = __shfl_xor_sync(GCR_FULL, key[i], ld);
            const bool asc = ((base + i) & size) == 0;
            const bool keep_small = lower == asc;
            key[i] = keep_small ? (o < key[i] ? o : key[i]) : (o > key[i] ? o : key[i]);
          }
        } else if (stride == 1) {
          reg_stage<E, 1>(key, base, size);
        } else if (stride == 2) {
          reg_stage<E, 2>(key, base, size);
        } else if (stride == 4) {
          reg_stage<E, 4>(key, base, size);
        } else {
          reg_stage<E, 8>(key, base, size);
        }
      }
    }
  }
  if (!in_smem) {
#pragma unroll
    for (int i = 0; i < E; ++i) sk[pad(base + i)] = key[i];
    __syncthreads();
  }
  // coalesced output of the first K ranks
  for (int r = t; r < K; r += T) {
    const unsigned long long k = sk[pad(r)];
    idx_out[(size_t)q * K + r] = (int32_t)(k & 0xffffffffu);
    dist_out[(size_t)q * K + r] = ordered_to_float((uint32_t)(k >> 32));
  }
}


// ---------------------------------------------------------------------------- radix sort
constexpr int kHistStride = 513;  // per-warp digit counts (up to 9-bit digits), padded against bank conflicts

// NT threads (NW = NT/32 warps, a multiple of 8), IPT keys per thread (even), segment <= NT*IPT.
// Keys live in registers; the gallery indices live in shared memory (two buffers, swapped per
// pass); the per-key offsets among the warp's keys of the same digit are packed two per register.
template <int NT, int IPT>
__global__ void __launch_bounds__(NT, 1)
rank_rows_radix_kernel(const float* __restrict__ D, int ng, int K, int32_t* __restrict__ idx_out,
                       float* __restrict__ dist_out) {
  constexpr int NW = NT / 32;
  constexpr int N = NT * IPT;
  static_assert(NW % 8 == 0 && IPT % 2 == 0, "warps: a multiple of 8; keys per thread: even");
  static_assert(N <= 65536, "gallery indices are held in 16 bits");
  extern __shared__ unsigned char smem_raw[];
  uint32_t* sk = reinterpret_cast<uint32_t*>(smem_raw);           // [N] keys
  uint16_t* si0 = reinterpret_cast<uint16_t*>(sk + N);            // [N] gallery indices
  uint16_t* si1 = si0 + N;                                        // [N] (second buffer)
  uint32_t* hist = reinterpret_cast<uint32_t*>(si1 + N);          // [NW][kHistStride]
  __shared__ uint32_t red_min[NW], red_max[NW], wsum[NW];

  const int q = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int e0 = w * 32 * IPT + lane;  // position of this thread's slot 0 (slot i: e0 + 32*i)
  const float* row = D + (size_t)q * ng;
  uint32_t key[IPT];
  uint32_t offp[IPT / 2];
  uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const int e = e0 + 32 * i;
    key[i] = e < ng ? float_to_ordered(row[e]) : 0xffffffffu;
    si0[e] = (uint16_t)e;
    if (e < ng) {
      kmin = min(kmin, key[i]);
      kmax = max(kmax, key[i]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(GCR_FULL, kmin, o));
    kmax = max(kmax, __shfl_xor_sync(GCR_FULL, kmax, o));
  }
  if (lane == 0) { red_min[w] = kmin; red_max[w] = kmax; }
  __syncthreads();
  for (int v = 0; v < NW; ++v) { kmin = min(kmin, red_min[v]); kmax = max(kmax, red_max[v]); }
  // Keys relative to the smallest (order-preserving): their range needs nb bits, usually far
  // fewer than 32 (distances of one query span a narrow band), so three 9-bit digit passes
  // often suffice where four 8-bit ones would be needed. Padding keys are all ones and stay
  // after every real key (on ties the stable passes keep their larger positions last).
  const uint32_t range = kmax - kmin;
  const int nb = range == 0 ? 0 : 32 - __clz((int)range);
  int W = 8, passes = (nb + 7) / 8;
  if (NT >= 512 && nb > 24 && nb <= 27) { W = 9; passes = 3; }  // a scan thread per digit at least
  const uint32_t B = 1u << W, mask = B - 1u;
#pragma unroll
  for (int i = 0; i < IPT; ++i)
    if (e0 + 32 * i < ng) key[i] -= kmin;
  const int TPD = NT / (int)B;       // scan threads per digit
  const int WPT = NW / TPD;          // warp counts per scan thread

  uint32_t* hw = hist + w * kHistStride;
  uint16_t* src = si0;
  uint16_t* dstb = si1;
  for (int pass = 0; pass < passes; ++pass) {  // block-uniform
    const int shift = pass * W;
    for (int v = t; v < NW * kHistStride; v += NT) hist[v] = 0;
    __syncthreads();
    // per-warp stable ranking, slot by slot (slot order = key order inside the warp); the lanes
    // holding the same digit from one ballot per digit bit
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const uint32_t dg = (key[i] >> shift) & mask;
      const unsigned peers = warp_peers(dg, W);
      const uint32_t base = hw[dg];
      __syncwarp();
      if ((peers & lt) == 0) hw[dg] = base + (uint32_t)__popc(peers);  // the lowest peer updates
      __syncwarp();
      const uint32_t off = base + (uint32_t)__popc(peers & lt);
      if (i & 1) offp[i >> 1] |= off << 16;
      else offp[i >> 1] = off;
    }
    __syncthreads();
    // exclusive scan of the counts in (digit, warp) order: thread t owns digit t / TPD and the
    // warps WPT * (t % TPD) .. + WPT - 1
    const int sdg = t / TPD, sw0 = (t % TPD) * WPT;
    uint32_t tot = 0;
    for (int j = 0; j < WPT; ++j) tot += hist[(sw0 + j) * kHistStride + sdg];
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(GCR_FULL, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    uint32_t run = inc - tot;
    for (int v = 0; v < w; ++v) run += wsum[v];
    for (int j = 0; j < WPT; ++j) {  // each thread rewrites only its own counts
      const uint32_t cj = hist[(sw0 + j) * kHistStride + sdg];
      hist[(sw0 + j) * kHistStride + sdg] = run;
      run += cj;
    }
    __syncthreads();
    // scatter keys and indices to their destinations, then reload the keys warp-striped
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const uint32_t off = (i & 1) ? (offp[i >> 1] >> 16) : (offp[i >> 1] & 0xffffu);
      const uint32_t dst = hw[(key[i] >> shift) & mask] + off;
      sk[dst] = key[i];
      dstb[dst] = src[e0 + 32 * i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IPT; ++i) key[i] = sk[e0 + 32 * i];
    uint16_t* tmp = src;
    src = dstb;
    dstb = tmp;
    __syncthreads();
  }
  // registers hold ranks e0 + 32*i in order: coalesced output of the first K
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const int e = e0 + 32 * i;
    if (e < K) {
      idx_out[(size_t)q * K + e] = (int32_t)src[e];
      dist_out[(size_t)q * K + e] = ordered_to_float(key[i] + kmin);
    }
  }
}

template <int NT, int IPT>
cudaError_t launch_radix(const float* D, int nq, int ng, int K, int32_t* idx_out, float* dist_out,
                         cudaStream_t st) {
  const size_t smem = (size_t)NT * IPT * (sizeof(uint32_t) + 2 * sizeof(uint16_t)) +
                      (size_t)(NT / 32) * kHistStride * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(rank_rows_radix_kernel<NT, IPT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  rank_rows_radix_kernel<NT, IPT><<<nq, NT, smem, st>>>(D, ng, K, idx_out, dist_out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rank_rows(const float* D, int nq, int ng, int K, int32_t* idx_out, float* dist_out,
                             cudaStream_t st) {
  if (ng > kMaxSeg) return cudaErrorInvalidValue;
  if (ng > 8192) return launch_radix<1024, 16>(D, nq, ng, K, idx_out, dist_out, st);
  if (ng > 4096) return launch_radix<512, 16>(D, nq, ng, K, idx_out, dist_out, st);
  if (ng >= 2048) return launch_radix<256, 16>(D, nq, ng, K, idx_out, dist_out, st);
  int N = 64;
  while (N < ng) N <<= 1;
  const int E = N >= 512 ? 16 : (N >= 128 ? 4 : 2);
  const int threads = N / E;
  const size_t smem = sizeof(unsigned long long) * (N + N / 32);
  cudaError_t e;
  if (E == 16) {
    e = cudaFuncSetAttribute(rank_rows_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    rank_rows_kernel<16><<<nq, threads, smem, st>>>(D, ng, N, K, idx_out, dist_out);
  } else if (E == 4) {
    rank_rows_kernel<4><<<nq, threads, smem, st>>>(D, ng, N, K, idx_out, dist_out);
  } else {
    rank_rows_kernel<2><<<nq, threads, smem, st>>>(D, ng, N, K, idx_out, dist_out);
  }
  (void)e;
  return cudaGetLastError();
}

}  // namespace gcr
