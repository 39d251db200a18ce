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

// ---------------------------------------------------------------- lane-parallel heap pools
// For 32-entry pools on the tensor-core path. Each row's pool is a heap of (score, index) pairs
// in shared memory ordered by better(): the root is the worst entry kept, so once the heap holds
// KP entries the admission threshold is the root's score (the same threshold as a sorted list's
// last entry). Heaps and queues are slot-major, [slot][128 rows] of float2, so the lanes of a
// warp (consecutive rows) always touch different bank pairs whatever slot each one is at. A lane
// appends the scores that pass to its row's queue; when any lane's queue could overflow, every
// lane drains its own queue into its own heap, so one pass serves the warp's 32 rows (the sorted
// lists instead take one warp-wide merge per row, each waiting on a list in L2). At the end a
// heapsort leaves each pool sorted best first, as the sorted lists are.
constexpr int kHeapQ = 8;                  // queue slots per row
constexpr uint32_t kHeapSlot = 128 * 8;    // bytes between consecutive slots of one row

__device__ __forceinline__ bool worse(float a, int ai, float b, int bi) { return a < b || (a == b && ai > bi); }

__device__ __forceinline__ float2 heap_ld(uint32_t addr) {
  float2 r;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(addr) : "memory");
  return r;
}
__device__ __forceinline__ void heap_st(uint32_t addr, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

struct HeapState {
  float tau;
  int len;
};

// Drains qcnt queued entries (queue slot 0 at qaddr) into the heap at haddr holding len entries.
// An entry that no longer beats the root (the threshold rose since it was queued) is dropped.
// Returns the new threshold (tau unchanged when nothing was queued) and length.
template <int KP>
__device__ __noinline__ HeapState heap_drain(uint32_t haddr, uint32_t qaddr, int qcnt, int len, float tau,
                                             float floor) {
  for (int i = 0; i < qcnt; ++i) {
    const float2 e = heap_ld(qaddr + i * kHeapSlot);
    const int ei = __float_as_int(e.y);
    if (len < KP) {  // not full yet: sift up from the first free slot
      int pos = len++;
      while (pos > 0) {
        const int par = (pos - 1) >> 1;
        const float2 p = heap_ld(haddr + par * kHeapSlot);
        if (!worse(e.x, ei, p.x, __float_as_int(p.y))) break;
        heap_st(haddr + pos * kHeapSlot, p);
        pos = par;
      }
      heap_st(haddr + pos * kHeapSlot, e);
    } else {  // full: replace the root if better, then sift down
      const float2 root = heap_ld(haddr);
      if (!worse(root.x, __float_as_int(root.y), e.x, ei)) continue;
      int pos = 0;
      for (;;) {
        int c = 2 * pos + 1;
        if (c >= KP) break;
        float2 cv = heap_ld(haddr + c * kHeapSlot);
        if (c + 1 < KP) {
          const float2 c2 = heap_ld(haddr + (c + 1) * kHeapSlot);
          if (worse(c2.x, __float_as_int(c2.y), cv.x, __float_as_int(cv.y))) {
            cv = c2;
            ++c;
          }
        }
        if (!worse(cv.x, __float_as_int(cv.y), e.x, ei)) break;
        heap_st(haddr + pos * kHeapSlot, cv);
        pos = c;
      }
      heap_st(haddr + pos * kHeapSlot, e);
    }
  }
  if (qcnt > 0) tau = (len == KP) ? fmaxf(heap_ld(haddr).x, floor) : floor;
  return HeapState{tau, len};
}

// Heapsort of the len entries at haddr (best first) and the row's KP-entry list written to lv /
// li, padded with (-inf, -1) past len.
template <int KP>
__device__ __noinline__ void heap_emit(uint32_t haddr, int len, float* lv, int* li) {
  for (int end = len - 1; end > 0; --end) {
    const float2 root = heap_ld(haddr);
    const float2 last = heap_ld(haddr + end * kHeapSlot);
    const int lasti = __float_as_int(last.y);
    heap_st(haddr + end * kHeapSlot, root);
    int pos = 0;
    for (;;) {
      int c = 2 * pos + 1;
      if (c >= end) break;
      float2 cv = heap_ld(haddr + c * kHeapSlot);
      if (c + 1 < end) {
        const float2 c2 = heap_ld(haddr + (c + 1) * kHeapSlot);
        if (worse(c2.x, __float_as_int(c2.y), cv.x, __float_as_int(cv.y))) {
          cv = c2;
          ++c;
        }
      }
      if (!worse(cv.x, __float_as_int(cv.y), last.x, lasti)) break;
      heap_st(haddr + pos * kHeapSlot, cv);
      pos = c;
    }
    heap_st(haddr + pos * kHeapSlot, last);
  }
  for (int e = 0; e < KP; ++e) {
    float v = -CUDART_INF_F;
    int i = -1;
    if (e < len) {
      const float2 x = heap_ld(haddr + e * kHeapSlot);
      v = x.x;
      i = __float_as_int(x.y);
    }
    lv[e] = v;
    li[e] = i;
  }
}

// Paired column splits: the row's sorted list in this CTA's heap slots (own, best first, len
// entries; slot e at own[e * 128]) merged with the other half's list (KP entries, best first,
// padded with (-inf, -1), read through L2) into the KP best, written to (dv, di). The other
// list is first copied to the scratch slots (same layout), so that dv may be the other list
// itself. Each entry goes straight to its rank: its index in its own list plus the number of
// entries of the other list that rank before it (a binary search; better() orders the two
// lists' entries totally, so the ranks of all entries are distinct).
template <int KP>
__device__ __forceinline__ void pair_merge_lists(const float2* own, int len, const float* ov, const int* oi,
                                                 float2* scratch, float* dv, int* di) {
  for (int e = 0; e < KP; ++e) scratch[e * 128] = make_float2(__ldcg(ov + e), __int_as_float(__ldcg(oi + e)));
  for (int i = 0; i < len; ++i) {
    const float2 x = own[i * 128];
    const int xi = __float_as_int(x.y);
    int lo = 0, hi = KP;  // others before x: the first j with other[j] not better than x
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      const float2 y = scratch[mid * 128];
      if (better(y.x, __float_as_int(y.y), x.x, xi)) lo = mid + 1;
      else hi = mid;
    }
    if (i + lo < KP) {
      dv[i + lo] = x.x;
      di[i + lo] = xi;
    }
  }
  for (int j = 0; j < KP; ++j) {
    const float2 y = scratch[j * 128];
    const int yi = __float_as_int(y.y);
    int lo = 0, hi = len;  // own entries before y
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      const float2 x = own[mid * 128];
      if (better(x.x, __float_as_int(x.y), y.x, yi)) lo = mid + 1;
      else hi = mid;
    }
    if (j + lo < KP) {
      dv[j + lo] = y.x;
      di[j + lo] = yi;
    }
  }
}

}  // namespace gcr
