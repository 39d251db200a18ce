// Streaming per-row candidate pool for the kNN search of Eq. 4 / Eq. 8.
//
// The similarity tile S = X_rows . X_cols^T is produced column tile by column tile and
// never stored. Each row has one owning thread (lane r of a warp owns row warp_row0 + r)
// holding three registers:
//   tau   admission threshold: the KP-th best score seen so far (-inf until KP seen),
//   qcnt  survivors queued in shared memory,
//   len   entries in the row's list.
// A column value v enters the row's queue only if v > tau. Once a queue may overflow,
// the warp merges it (all 32 lanes on one row at a time) into the row's sorted list of
// KP (score, index) pairs, kept in global memory (L2-resident). After the last column
// tile the list holds the row's KP best scores, and every score left out is <= its
// last entry. The certified refinement consumes exactly that guarantee.
#pragma once
#include "common.cuh"

namespace gcr {

// Queue layout in shared memory: for CTA-local row r, slot s lives at r*kQCap + (s ^ (r & 31)),
// so that the owner's appends and the warp's reads during a merge are both conflict-free.
struct PoolOwner {
  float tau;
  int qcnt;
  int len;
};

__device__ __forceinline__ void pool_init(PoolOwner& o, bool valid) {
  o.tau = valid ? -CUDART_INF_F : CUDART_INF_F;
  o.qcnt = 0;
  o.len = 0;
}

__device__ __forceinline__ void pool_push(PoolOwner& o, float v, int j, float* qv, int* qi, int sw) {
  if (v > o.tau) {
    int s = o.qcnt ^ sw;
    qv[s] = v;
    qi[s] = j;
    ++o.qcnt;
  }
}

// Warp-cooperative merge of the queue of the row owned by lane `owner` into its list.
// qv_row/qi_row: that row's queue; lv/li: that row's list (KP entries) in global memory.
template <int KP>
__device__ __forceinline__ void pool_merge_row(int owner, int lane, float* lv, int* li,
                                               const float* qv_row, const int* qi_row, int sw,
                                               PoolOwner& me) {
  __syncwarp();  // the owner's queue writes must be visible to the whole warp
  int q = __shfl_sync(GCR_FULL, me.qcnt, owner);
  int L = __shfl_sync(GCR_FULL, me.len, owner);
  float a = -CUDART_INF_F;
  int ai = -1;
  if (lane < q) {
    a = qv_row[lane ^ sw];
    ai = qi_row[lane ^ sw];
  }
  warp_sort32_desc(a, ai, lane);
  float ar = __shfl_sync(GCR_FULL, a, 31 - lane);
  int ari = __shfl_sync(GCR_FULL, ai, 31 - lane);
  float last;
  if constexpr (KP == 32) {
    float b = -CUDART_INF_F;
    int bi = -1;
    if (lane < L) { b = lv[lane]; bi = li[lane]; }
    // top 32 of (list desc) U (queue desc): elementwise max against the reversed queue
    // gives a bitonic sequence holding exactly those 32; one bitonic merge sorts it.
    if (better(ar, ari, b, bi)) { b = ar; bi = ari; }
    warp_merge32_desc(b, bi, lane);
    lv[lane] = b;
    li[lane] = bi;
    last = __shfl_sync(GCR_FULL, b, 31);
  } else {
    static_assert(KP == 64, "pool size must be 32 or 64");
    float b0 = -CUDART_INF_F, b1 = -CUDART_INF_F;
    int bi0 = -1, bi1 = -1;
    if (lane < L) { b0 = lv[lane]; bi0 = li[lane]; }
    if (lane + 32 < L) { b1 = lv[lane + 32]; bi1 = li[lane + 32]; }
    // C[s] = max(B[s], Qpad[63 - s]); Qpad is -inf past 32, so only the upper half changes.
    if (better(ar, ari, b1, bi1)) { b1 = ar; bi1 = ari; }
    // bitonic merge of 64: stride 32 inside the lane, then each half with shuffles
    if (better(b1, bi1, b0, bi0)) {
      float tv = b0; b0 = b1; b1 = tv;
      int ti = bi0; bi0 = bi1; bi1 = ti;
    }
    warp_merge32_desc(b0, bi0, lane);
    warp_merge32_desc(b1, bi1, lane);
    lv[lane] = b0;
    li[lane] = bi0;
    lv[lane + 32] = b1;
    li[lane + 32] = bi1;
    last = __shfl_sync(GCR_FULL, b1, 31);
  }
  int nl = min(KP, L + q);
  if (lane == owner) {
    me.len = nl;
    me.qcnt = 0;
    me.tau = (nl == KP) ? last : -CUDART_INF_F;
  }
  __syncwarp();  // queue slots are reused only after every lane has read them
}

// Merge every row of this warp whose queue holds more than kQCap - room entries.
// row_of_lane0: global row of lane 0; q_base: CTA-local row index of lane 0 in the queue.
template <int KP>
__device__ __forceinline__ void pool_make_room(int room, int lane, PoolOwner& me, int row_of_lane0,
                                               int qrow0, float* qv, int* qi, float* pool_v,
                                               int* pool_i) {
  unsigned m = __ballot_sync(GCR_FULL, me.qcnt > kQCap - room);
  while (m) {
    int o = __ffs(m) - 1;
    m &= m - 1;
    int qr = qrow0 + o;
    size_t grow = (size_t)(row_of_lane0 + o);
    pool_merge_row<KP>(o, lane, pool_v + grow * KP, pool_i + grow * KP, qv + qr * kQCap,
                       qi + qr * kQCap, qr & 31, me);
  }
}

// Final merge of every valid row of the warp (writes the list even if nothing is queued).
template <int KP>
__device__ __forceinline__ void pool_flush(int lane, bool valid, PoolOwner& me, int row_of_lane0,
                                           int qrow0, float* qv, int* qi, float* pool_v,
                                           int* pool_i) {
  unsigned m = __ballot_sync(GCR_FULL, valid);
  while (m) {
    int o = __ffs(m) - 1;
    m &= m - 1;
    int qr = qrow0 + o;
    size_t grow = (size_t)(row_of_lane0 + o);
    pool_merge_row<KP>(o, lane, pool_v + grow * KP, pool_i + grow * KP, qv + qr * kQCap,
                       qi + qr * kQCap, qr & 31, me);
  }
}

}  // namespace gcr
