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

// Queue layout in shared memory: float2 entries (score, index bits); for CTA-local row r,
// slot s lives at r*kQCap + (s ^ (r & 31)), so that the owner's 8-byte appends and the warp's
// reads during a merge are both conflict-free.
struct PoolOwner {
  float tau;
  float floor;  // admission floor (or -inf): scores at or below it are dropped, so tau never
                // drops below it; the caller bounds what was dropped by it
  int qcnt;
  int len;
};

__device__ __forceinline__ void pool_init(PoolOwner& o, bool valid, float floor) {
  o.floor = floor;
  o.tau = valid ? floor : CUDART_INF_F;
  o.qcnt = 0;
  o.len = 0;
}
__device__ __forceinline__ void pool_init(PoolOwner& o, bool valid) { pool_init(o, valid, -CUDART_INF_F); }

// Branch-free append: the candidate is always written into the next free slot and the count
// only advances when it passes (ok and v > tau). The caller guarantees qcnt < kQCap before
// every call (pool_make_room with room = values pushed before the next check).
__device__ __forceinline__ void pool_push(PoolOwner& o, float v, int j, bool ok, float2* q, int sw) {
  q[o.qcnt ^ sw] = make_float2(v, __int_as_float(j));
  o.qcnt += (ok && v > o.tau) ? 1 : 0;
}

// Warp-cooperative merge of the queue of the row owned by lane `owner` into its list.
// qv_row/qi_row: that row's queue; lv/li: that row's list (KP entries) in global memory.
// Kept out of line (the merge is rare and large); takes and returns plain values so that the
// caller's owner state stays in registers. Returns the new list length and its last score.
struct MergeResult {
  int len;
  float last;
};

template <int KP>
__device__ __noinline__ MergeResult pool_merge_row(int owner, int lane, float* lv, int* li,
                                                   const float2* q_row, int sw, int my_qcnt, int my_len) {
  __syncwarp();  // the owner's queue writes must be visible to the whole warp
  int q = __shfl_sync(GCR_FULL, my_qcnt, owner);
  int L = __shfl_sync(GCR_FULL, my_len, owner);
  float a = -CUDART_INF_F;
  int ai = -1;
  if (lane < q) {
    const float2 e = q_row[lane ^ sw];
    a = e.x;
    ai = __float_as_int(e.y);
  }
  // the list loads (L2 latency) are issued before the queue sort so that the two overlap
  static_assert(KP == 32 || KP == 64 || KP == 128, "pool size must be 32, 64 or 128");
  constexpr int P = KP / 32;  // list entries per lane: entry e = p*32 + lane
  float b[P];
  int bi[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int e = p * 32 + lane;
    b[p] = e < L ? lv[e] : -CUDART_INF_F;
    bi[p] = e < L ? li[e] : -1;
  }
  warp_sort32_desc(a, ai, lane);
  float ar = __shfl_sync(GCR_FULL, a, 31 - lane);
  int ari = __shfl_sync(GCR_FULL, ai, 31 - lane);
  // Top KP of (list, descending) U (queue, descending): C[s] = max(B[s], Q[KP-1-s]) with Q
  // padded by -inf past 32 entries is a bitonic sequence holding exactly those KP; only the
  // last 32 entries can change. A bitonic merge then sorts it.
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
  for (int p = 0; p < P; ++p) {
    warp_merge32_desc(b[p], bi[p], lane);
    lv[p * 32 + lane] = b[p];
    li[p * 32 + lane] = bi[p];
  }
  const float last = __shfl_sync(GCR_FULL, b[P - 1], 31);
  __syncwarp();  // queue slots are reused only after every lane has read them
  return MergeResult{min(KP, L + q), last};
}

template <int KP>
__device__ __forceinline__ void pool_merge_apply(int owner, int lane, float* lv, int* li, const float2* q_row,
                                                 int sw, PoolOwner& me) {
  const MergeResult r = pool_merge_row<KP>(owner, lane, lv, li, q_row, sw, me.qcnt, me.len);
  if (lane == owner) {
    me.len = r.len;
    me.qcnt = 0;
    me.tau = (r.len == KP) ? fmaxf(r.last, me.floor) : me.floor;
  }
}

// Merge every row of this warp whose queue could not take `room` more pushes (the branch-free
// push writes one slot past the count, so the count must stay below kQCap - room).
// row_of_lane0: global row of lane 0; qrow0: CTA-local queue row of lane 0.
template <int KP>
__device__ __forceinline__ void pool_make_room(int room, int lane, PoolOwner& me, int row_of_lane0,
                                               int qrow0, float2* q, float* pool_v, int* pool_i) {
  unsigned m = __ballot_sync(GCR_FULL, me.qcnt >= kQCap - room);
  while (m) {
    int o = __ffs(m) - 1;
    m &= m - 1;
    int qr = qrow0 + o;
    size_t grow = (size_t)(row_of_lane0 + o);
    pool_merge_apply<KP>(o, lane, pool_v + grow * KP, pool_i + grow * KP, q + qr * kQCap, qr & 31, me);
  }
}

// Final merge of every valid row of the warp (writes the list even if nothing is queued).
template <int KP>
__device__ __forceinline__ void pool_flush(int lane, bool valid, PoolOwner& me, int row_of_lane0,
                                           int qrow0, float2* q, float* pool_v, int* pool_i) {
  unsigned m = __ballot_sync(GCR_FULL, valid);
  while (m) {
    int o = __ffs(m) - 1;
    m &= m - 1;
    int qr = qrow0 + o;
    size_t grow = (size_t)(row_of_lane0 + o);
    pool_merge_apply<KP>(o, lane, pool_v + grow * KP, pool_i + grow * KP, q + qr * kQCap, qr & 31, me);
  }
}

}  // namespace gcr
