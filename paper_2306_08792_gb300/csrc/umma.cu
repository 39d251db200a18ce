// Similarity GEMM on the 5th-generation tensor cores (tcgen05), sm_103a.
//
// S = A . B^T with A, B row-major (K = d contiguous, "K-major"), either BF16 or FP32 rows
// rounded to TF32: A holds 128 rows of X, B 256 rows. Per CTA:
//   warp 0        TMA producer: 128-byte K blocks (64 BF16 or 32 TF32 elements) of A (128 rows)
//                 and B (256 rows) into a 3-stage shared-memory ring (128-byte swizzle),
//                 mbarrier transaction counts;
//   warp 1        allocates 512 TMEM columns (two 128 x 256 FP32 accumulators) and, from one
//                 thread, issues tcgen05.mma (kind::f16 with K=16, or kind::tf32 with K=8;
//                 M=128, N=256) for each K block,
//                 committing stage releases and "accumulator full" to mbarriers;
//   warps 2..5    epilogue for the global graph, warps 6..9 for the cross-camera graph:
//                 tcgen05.ld.32x32b gives each thread one accumulator row (32 columns per
//                 load); the scores go into the streaming per-row pool (pool.cuh), or are
//                 appended to the band buffer, or written out as distances.
// The accumulator is double-buffered so the MMAs of column tile j+1 overlap the epilogue of
// tile j. Every mbarrier wait is bounded (2 s of %globaltimer); on a timeout the CTA raises a
// shared abort flag that every role polls, waits (bounded) for its in-flight MMAs, frees TMEM
// and returns; the timeout is counted in a device word that gcr_sync reports.
#include <algorithm>
#include <cmath>
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "pool.cuh"

namespace gcr {

__device__ int g_umma_timeouts;  // bounded waits that ran out since the last gcr_sync

namespace {

constexpr int BM = 128;            // rows of A per tile (UMMA M)
constexpr int BN = 256;            // rows of B per tile (UMMA N)
constexpr int BKB = 128;           // K bytes per stage (one swizzle row): 64 BF16 / 32 TF32
constexpr int NST = 3;             // pipeline stages of the modes with pool queues (POOL, GPOOL)
constexpr int NST_MAX = 4;         // the others (no queues in shared memory)
constexpr int A_BYTES = BM * BKB;
constexpr int B_BYTES = BN * BKB;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 512;
constexpr unsigned long long kTimeoutNs = 2000000000ull;

enum Mode { POOL = 0, BAND = 1, DIST = 2, GRAM = 3, MUL = 4, GPOOL = 5 };

// ------------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the CTA is aborting (or this wait ran out and started the abort).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long limit_ns = kTimeoutNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > limit_ns) {
        *abort_flag = 1;
        atomicAdd(&g_umma_timeouts, 1);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major tile of rows of 128 bytes, 128-byte swizzle,
// 8-row core groups 1024 bytes apart (SBO), tile base 1024-byte aligned.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                          // layout: 128-byte swizzle
  return d;
}
// Instruction descriptors: D = F32 (bits 4-5 = 1), A and B formats (bits 7-9, 10-12: BF16 = 1
// under kind::f16, TF32 = 2 under kind::tf32), both K-major, N >> 3 (bits 17-22), M >> 4
// (bits 24-28); N = 256, M = 128.
constexpr uint32_t kIdescShape = ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | kIdescShape;
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | kIdescShape;

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdescBf16), "r"(accum));
}
__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdescTf32), "r"(accum));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 2-CTA clusters sharing B tiles: the commit arrives on the barrier at the same offset in every
// CTA of the mask; the load writes the tile (and completes its bytes on the barrier) at the same
// offsets in every CTA of the mask.
__device__ __forceinline__ void umma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
               ::"r"(smem_u32(bar)), "h"(mask)
               : "memory");
}
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%3, %4}], [%2], %5;"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "h"(mask)
      : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Asynchronous TMEM load of 32 columns (one accumulator row per thread) ...
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// ... and the wait for it; the registers are passed through the wait so that no use of them
// can be scheduled before the load has landed.
__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  tmem_ld32_async(taddr, r);
  tmem_wait32(r);
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------------ kernel
struct UmmaArgs {
  int mode;
  int tf32;       // operands: 0 BF16 (kind::f16), 1 TF32 held as FP32 (kind::tf32)
  int n;          // rows of B (columns of S)
  int d;
  int a_rows;     // rows of A (POOL: rows owning pools; DIST: nq; BAND: band capacity)
  int self_excl;  // skip column j == row i (A and B are the same matrix)
  int tps;        // POOL: column tiles per split (grid.y = splits)
  const int* cam;
  // POOL
  float* pool_v;
  int* pool_i;
  const float* seed;  // per row of A, or NULL: admission floor of the row's split pools
  // BAND
  const int* count;
  int cap;
  const int* band_row;
  const int* band_kind;
  const float* band_thr;
  int bcap;
  int* band_cnt;
  float* band_v;       // may be NULL (indices only)
  int* band_i;
  const int* band_off; // NULL: row u writes at u * bcap; else at band_off[u]
  const int* band_lim; // NULL: bcap entries per row; else band_lim[u]
  // DIST
  const float* nrm_q;
  const float* nrm_g;
  float* D;
  // GRAM: G_s = Z_s Z_s^T + lambda n_s I per camera s = blockIdx.z, Z = the transposed,
  // normalised frames (feature rows, frame columns) split as hi + lo in BF16; K blocks of 64
  // frames [gram_kstart[s], + gram_knum[s]) run three times: hi.hi, hi.lo, lo.hi
  const int64_t* gram_kstart;
  const int64_t* gram_knum;
  const int64_t* gram_nf;  // n_s
  float gram_lambda;
  float* G;                // [ncam][d][d]
  // MUL: Q = P G_s for each 128-row block of P (camera s = mul_rowcam[block], < 0: skipped);
  // TF32 operands split hi + lo (hi.hi + hi.lo + lo.hi); G stacked as ncam * d rows of d
  const int* mul_rowcam;
  int dist_nrb;    // row tiles of the distance matrix
  int dist_tiles;  // all tiles; CTA b takes tiles b, b + grid, ... in column-major tile order,
                   // so the CTAs at work share the (small) query blocks and stream each gallery
                   // column tile once
  // GPOOL: pools of the rows of a gathered matrix against column ranges of the same matrix.
  // Work item w = {first row, rows (<= BM), first column, columns}; CTA b takes the items
  // b, b + grid, ... of the *n_items; a pool entry holds s - col_bias[j]; column j == row is
  // skipped when self_excl; cam (may be NULL) is indexed by gathered position.
  const int4* items;
  const int* n_items;
  const float* col_bias;
  int vote;        // POOL: pick the kernel that skips groups of four scores below every row's
                   // threshold by a vote (GPOOL always does)
  int warm;        // POOL: admission floors from each row's first column tile (warm_floor)
  // POOL with heap pools, paired splits: two CTAs per row block (grid.x = the 2 column splits,
  // grid.y = row blocks, so both halves of a block run at the same time and the row blocks at
  // work stay few enough for their A rows to stay in L2). Each writes its rows' thresholds to
  // tau_x after every tile and raises its own to the other's (a threshold of either half is a
  // score with KP of the row's scores at or above it); the warp that finishes second merges the
  // two lists into the first split's pools.
  int pair;
  float* tau_x;    // [2][pools][a_rows], NaN-initialised (no threshold yet)
  int* pair_cnt;   // [row blocks][pools][4], zero-initialised: finished warps per (block, pool, quad)
  // POOL with heap pools: 2-CTA clusters of consecutive row blocks that take the same column
  // tiles; each CTA loads its A block and one half of the B tile, and the half goes to both
  // CTAs by TMA multicast (tmB2: B in 128-row boxes), so a CTA reads two thirds of the bytes
  // per stage. Each MMA commit frees the stage in both CTAs (empty barriers count 2 arrivals).
  int mc;
};

struct __align__(8) Bars {
  uint64_t full[NST_MAX];
  uint64_t empty[NST_MAX];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
};

// GPOOL walk over a CTA's work items and their column tiles: every role keeps its own cursor
// and advances it once per tile, so all roles see the same sequence.
struct ItemCursor {
  int item, ct, nt;
  int4 w;
  __device__ void load(const UmmaArgs& a, int nitems) {
    w = item < nitems ? a.items[item] : make_int4(0, 0, 0, 0);
    nt = (w.w + BN - 1) / BN;
  }
  __device__ void start(const UmmaArgs& a, int nitems) {
    item = blockIdx.x;
    ct = 0;
    load(a, nitems);
  }
  __device__ void advance(const UmmaArgs& a, int nitems) {
    if (++ct >= nt) {
      item += gridDim.x;
      ct = 0;
      load(a, nitems);
    }
  }
};

// Work list of a CTA: tiles (row block of A, column tile of B) in order.
template <int MODE>
struct Tiles {
  int count;
  int rb, split;  // POOL: row block and column split of this CTA
  __device__ int row0(const UmmaArgs& a, int t) const {
    if (MODE == POOL) return rb * BM;
    if (MODE == GRAM || MODE == MUL) return blockIdx.y * BM;
    if (MODE == BAND) return (blockIdx.y + t * gridDim.y) * BM;  // row tiles strided over grid.y
    return (((int)blockIdx.x + t * (int)gridDim.x) % a.dist_nrb) * BM;
  }
  __device__ int col0(const UmmaArgs& a, int t) const {
    if (MODE == POOL) return (split * a.tps + t) * BN;
    if (MODE == GRAM || MODE == MUL) return blockIdx.x * BN;
    if (MODE == BAND) return blockIdx.x * BN;
    return (((int)blockIdx.x + t * (int)gridDim.x) / a.dist_nrb) * BN;
  }
};

constexpr int kWarmIters = 6;  // bisection steps of warm_floor

// Admission floor of one row from the first column tile of its sweep. A pool starts empty, so
// without a floor every score of that tile would enter the row's queue and the warp would merge
// it about BN / 28 times before the threshold means anything. Bisection over the tile's eligible
// scores (held in TMEM, read once per step) finds a value f with at least KP of them above it:
// the row's KP best scores of the whole sweep all lie above f, so scores at or below f can be
// dropped from the sweep, and the row's list still ends full with every score left out below its
// last entry. The counts use the same values and the same eligibility (column < n, not the row
// itself, another camera for the cross-camera pool) as the appends. -inf when the tile holds
// KP eligible scores or fewer. All lanes run every step (the TMEM loads are warp-wide).
template <int KP, bool CAMCHK>
__device__ __noinline__ float warm_floor(uint32_t taddr, int cb0, int ncol, int n, int self_excl, int my_row,
                                         const int* __restrict__ cam, int my_cam, int lane) {
  uint32_t elig[BN / 32];
  float lo_v = CUDART_INF_F, hi_v = -CUDART_INF_F;
  int ne = 0;
#pragma unroll
  for (int ch = 0; ch < BN / 32; ++ch) {
    elig[ch] = 0u;
    if (ch * 32 < ncol) {
      float v[32];
      tmem_ld32(taddr + ch * 32, v);
      const int cb = cb0 + ch * 32;
      int ccam = 0;
      if (CAMCHK) ccam = (cb + lane < n) ? cam[cb + lane] : -1;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int cj = CAMCHK ? __shfl_sync(GCR_FULL, ccam, c) : 0;
        const bool e = cb + c < n && !(self_excl && cb + c == my_row) && (!CAMCHK || cj != my_cam);
        if (e) {
          lo_v = fminf(lo_v, v[c]);
          hi_v = fmaxf(hi_v, v[c]);
          ++ne;
          elig[ch] |= 1u << c;
        }
      }
    }
  }
  const bool active = ne > KP;
  float f = -CUDART_INF_F;
  float a = active ? lo_v : 0.f, b = active ? hi_v : 0.f;
#pragma unroll 1
  for (int it = 0; it < kWarmIters; ++it) {
    const float mid = 0.5f * a + 0.5f * b;
    int cnt = 0;
#pragma unroll
    for (int ch = 0; ch < BN / 32; ++ch) {
      if (ch * 32 < ncol) {
        float v[32];
        tmem_ld32(taddr + ch * 32, v);
#pragma unroll
        for (int c = 0; c < 32; ++c) cnt += (((elig[ch] >> c) & 1u) && v[c] > mid) ? 1 : 0;
      }
    }
    if (cnt >= KP) {
      f = mid;
      a = mid;
    } else {
      b = mid;
    }
  }
  return active ? f : -CUDART_INF_F;
}

// MODE is a template parameter (not only a field of UmmaArgs) so that each mode's epilogue is
// compiled alone: no per-value mode branches, and the POOL kernels need 88-90 registers instead
// of 116-118 (similarity GEMM on crosscam 2.72 -> 2.65 ms per TF32 launch, 2.75 -> 2.48 BF16).
template <int MODE, int KP, bool CROSS, bool VOTE = false>
__global__ void __launch_bounds__(320, 1)
umma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2, UmmaArgs a) {
  extern __shared__ __align__(1024) unsigned char dyn_raw[];
  // aligned by an offset from the shared array itself, so that every pointer derived from it
  // stays known as shared memory (queue appends compile to shared stores, not generic ones)
  unsigned char* dyn = dyn_raw + ((1024u - (smem_u32(dyn_raw) & 1023u)) & 1023u);
  constexpr int NS = (MODE == POOL || MODE == GPOOL) ? NST : NST_MAX;  // ring stages
  unsigned char* stages = dyn;                                        // NS * STAGE_BYTES
  float2* qs = reinterpret_cast<float2*>(dyn + NS * STAGE_BYTES);    // [2][BM][kQCap] queues
  // 32-entry pools of the per-value path: lane-parallel heaps ([2][KP][BM] float2, slot-major)
  // and their queues ([2][kHeapQ][BM]) in place of the sorted lists' queues
  constexpr bool HEAP = MODE == POOL && KP == 32 && !VOTE;
  float2* hq = reinterpret_cast<float2*>(dyn + NS * STAGE_BYTES + 2 * KP * BM * sizeof(float2));
  __shared__ Bars bars;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bk = a.tf32 ? BKB / 4 : BKB / 2;  // K elements per stage
  // K blocks per tile (GRAM: three passes over the camera's frame blocks)
  const int gram_kn = MODE == GRAM ? (int)a.gram_knum[blockIdx.z] : (a.d + bk - 1) / bk;
  const int kb_count = (MODE == GRAM || MODE == MUL) ? 3 * gram_kn : (a.d + bk - 1) / bk;
  // MUL: rows of camera s's G_s in the stacked G
  const int mul_b0 = MODE == MUL ? max(0, a.mul_rowcam[blockIdx.y]) * a.n : 0;

  Tiles<MODE> tl;
  tl.rb = (MODE == POOL && a.pair) ? (int)blockIdx.y : (int)blockIdx.x;
  tl.split = (MODE == POOL && a.pair) ? (int)blockIdx.x : (int)blockIdx.y;
  int nitems = 0;
  if (MODE == GPOOL) {
    nitems = *a.n_items;
    if ((int)blockIdx.x >= nitems) return;  // nothing to do: leave before any barrier or TMEM use
    tl.count = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) tl.count += (a.items[it].w + BN - 1) / BN;
  } else if (MODE == POOL) tl.count = max(0, min(a.tps, (a.n + BN - 1) / BN - tl.split * a.tps));
  else if (MODE == BAND) {
    const int U = min(*a.count, a.cap);
    const int tiles = (U + BM - 1) / BM;
    tl.count = max(0, (tiles - (int)blockIdx.y + (int)gridDim.y - 1) / (int)gridDim.y);
    if (tl.count == 0) return;  // no rows for this CTA: leave before any barrier or TMEM use
  } else if (MODE == GRAM) {
    // G_s is symmetric: tiles wholly below the diagonal (every column < every row) are mirrored
    tl.count = ((int)blockIdx.x + 1) * BN <= (int)blockIdx.y * BM ? 0 : 1;
  } else if (MODE == MUL) {
    tl.count = a.mul_rowcam[blockIdx.y] >= 0 ? 1 : 0;
  } else {
    tl.count = max(0, (a.dist_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x);
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&bars.full[s], 1);
      mbar_init(&bars.empty[s], (MODE == POOL && a.mc) ? 2 : 1);
    }
    const int epi_warps = CROSS ? 8 : 4;
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars.tfull[b], 1);
      mbar_init(&bars.tempty[b], epi_warps);
    }
    mbar_init(&bars.drain, 1);
    bars.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars.tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // clusters: every barrier of both CTAs is initialised before either CTA signals the other's
  if (MODE == POOL && a.mc) cluster_sync_all();
  const uint32_t tmem = bars.tmem_base;
  volatile int* abort_flag = &bars.abort_flag;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int it = 0;
      ItemCursor cur;
      if (MODE == GPOOL) cur.start(a, nitems);
      for (int t = 0; t < tl.count && !*abort_flag; ++t) {
        const int r0 = MODE == GPOOL ? cur.w.x : tl.row0(a, t);
        const int c0 = MODE == GPOOL ? cur.w.z + cur.ct * BN : tl.col0(a, t);
        if (MODE == GPOOL) cur.advance(a, nitems);
        for (int kb = 0; kb < kb_count; ++kb, ++it) {
          const int s = it % NS;
          const uint32_t round = it / NS;
          if (!mbar_wait(&bars.empty[s], (round & 1) ^ 1, abort_flag)) break;
          unsigned char* sa = stages + s * STAGE_BYTES;
          mbar_arrive_expect_tx(&bars.full[s], STAGE_BYTES);
          if (MODE == GRAM) {
            const int pass = kb / gram_kn;
            const int x = (int)((a.gram_kstart[blockIdx.z] + kb % gram_kn) * bk);
            tma_load_2d(sa, pass == 2 ? &tmA2 : &tmA, &bars.full[s], x, r0);
            tma_load_2d(sa + A_BYTES, pass == 1 ? &tmB2 : &tmB, &bars.full[s], x, c0);
          } else if (MODE == MUL) {
            const int pass = kb / gram_kn;
            const int x = (kb % gram_kn) * bk;
            tma_load_2d(sa, pass == 2 ? &tmA2 : &tmA, &bars.full[s], x, r0);
            tma_load_2d(sa + A_BYTES, pass == 1 ? &tmB2 : &tmB, &bars.full[s], x, mul_b0 + c0);
          } else {
            tma_load_2d(sa, &tmA, &bars.full[s], kb * bk, r0);
            if (MODE == POOL && a.mc) {
              const uint32_t cr = cluster_rank();
              tma_load_2d_mc(sa + A_BYTES + cr * (B_BYTES / 2), &tmB2, &bars.full[s], kb * bk,
                             c0 + (int)cr * (BN / 2), (uint16_t)0x3);
            } else {
              tma_load_2d(sa + A_BYTES, &tmB, &bars.full[s], kb * bk, c0);
            }
          }
        }
      }
      // in-flight loads land before the CTA can exit: wait for the last armed stages
      if (*abort_flag) {
        for (int back = 1; back <= NS && back <= it; ++back) {
          const int j = it - back;
          const unsigned long long t0 = globaltimer();
          while (!mbar_try_wait(&bars.full[j % NS], (j / NS) & 1) && globaltimer() - t0 < kTimeoutNs) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = 0; t < tl.count && ok; ++t) {
        const int buf = t & 1;
        const uint32_t use = t >> 1;
        if (!mbar_wait(&bars.tempty[buf], (use & 1) ^ 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t dcol = tmem + buf * BN;
        for (int kb = 0; kb < kb_count; ++kb, ++it) {
          const int s = it % NS;
          if (!mbar_wait(&bars.full[s], (it / NS) & 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(stages + s * STAGE_BYTES);
          const uint64_t ad = smem_desc(sa), bd = smem_desc(sa + A_BYTES);
          // four MMAs per stage, +32 bytes (K=16 BF16 or K=8 TF32) inside the swizzle row
          if (a.tf32) {
#pragma unroll
            for (int k = 0; k < 4; ++k) umma_tf32(dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), (kb | k) != 0);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) umma_bf16(dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), (kb | k) != 0);
          }
          if (MODE == POOL && a.mc) umma_commit_mc(&bars.empty[s], (uint16_t)0x3);
          else umma_commit(&bars.empty[s]);
        }
        if (ok) umma_commit(&bars.tfull[buf]);
      }
      // all issued MMAs complete before TMEM is released
      umma_commit(&bars.drain);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(&bars.drain, 0) && globaltimer() - t0 < kTimeoutNs) {
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue warps
    const int ew = warp - 2;                 // 0..7
    const int kind = ew >> 2;                // 0: global graph, 1: cross-camera graph
    const int quad = warp & 3;               // TMEM lanes 32*quad .. 32*quad+31
    const int r = quad * 32 + lane;          // row of the accumulator owned by this thread
    const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
    PoolOwner me;
    int my_row = -1, my_cam = 0;
    float my_thr = 0.f, my_nq = 0.f;
    int my_kind = 0;
    const int qrow = kind * BM + r;
    const int sw = qrow & 31;
    const uint32_t haddr = smem_u32(dyn + NS * STAGE_BYTES) + (uint32_t)((kind * KP * BM + r) * sizeof(float2));
    const uint32_t qaddr = smem_u32(hq) + (uint32_t)((kind * kHeapQ * BM + r) * sizeof(float2));
    float2* const hqp = hq + kind * kHeapQ * BM + r;  // this row's queue, slot s at hqp[s * BM]
    const size_t pbase = ((size_t)tl.split * (CROSS ? 2 : 1) + kind) * a.a_rows * KP;
    float* pv = a.pool_v ? a.pool_v + pbase : nullptr;
    int* pi = a.pool_i ? a.pool_i + pbase : nullptr;
    if (MODE == POOL) {
      my_row = tl.rb * BM + r;
      const bool valid = my_row < a.a_rows;
      pool_init(me, valid, (valid && a.seed) ? a.seed[my_row] : -CUDART_INF_F);
      if (CROSS && valid) my_cam = a.cam[my_row];
    }
    ItemCursor cur;
    if (MODE == GPOOL) cur.start(a, nitems);
    bool g_valid = false;        // GPOOL: this thread's row belongs to the current item
    int g_row0 = 0, g_cend = 0;  // GPOOL: first row of the item, end of its columns
    // paired splits: this row's threshold in the other half's sweep (read before the wait)
    const bool pair_row = HEAP && a.pair && (kind == 0 || CROSS) && my_row < a.a_rows;
    const size_t tx_mine = ((size_t)tl.split * (CROSS ? 2 : 1) + kind) * a.a_rows + (pair_row ? my_row : 0);
    const size_t tx_other = ((size_t)(tl.split ^ 1) * (CROSS ? 2 : 1) + kind) * a.a_rows + (pair_row ? my_row : 0);
    for (int t = 0; t < tl.count; ++t) {
      const int buf = t & 1;
      const uint32_t use = t >> 1;
      const float tau_other = pair_row ? __ldcg(a.tau_x + tx_other) : CUDART_NAN_F;
      if (!mbar_wait(&bars.tfull[buf], use & 1, abort_flag)) break;
      tc_fence_after();
      const int r0 = MODE == GPOOL ? cur.w.x : tl.row0(a, t);
      const int c0 = MODE == GPOOL ? cur.w.z + cur.ct * BN : tl.col0(a, t);
      const bool g_first = MODE == GPOOL && cur.ct == 0;
      const bool g_last = MODE == GPOOL && cur.ct == cur.nt - 1;
      if (g_first) {
        g_row0 = cur.w.x;
        g_cend = cur.w.z + cur.w.w;
        g_valid = r < cur.w.y;
        my_row = g_row0 + r;
        pool_init(me, g_valid);
        if (CROSS && g_valid) my_cam = a.cam[my_row];
      }
      if (MODE == GPOOL) cur.advance(a, nitems);
      int u = -1;
      if (MODE == BAND) {
        u = r0 + r;
        const int U = min(*a.count, a.cap);
        if (u < U) {
          my_row = a.band_row[u];
          my_kind = a.band_kind[u];
          my_thr = a.band_thr[u];
          if (a.cam) my_cam = a.cam[my_row];
        } else {
          u = -1;
        }
      } else if (MODE == DIST) {
        my_row = r0 + r;
        my_nq = my_row < a.a_rows ? a.nrm_q[my_row] : 0.f;
      } else if (MODE == MUL) {
        my_row = r0 + r;
      } else if (MODE == GRAM) {
        my_row = r0 + r;
        my_nq = a.gram_lambda * (float)a.gram_nf[blockIdx.z];  // lambda n_s, added on the diagonal
      }
      const int cend = MODE == GPOOL ? g_cend : a.n;  // end of this tile's valid columns
      const int ncol = min(BN, cend - c0);
      if (MODE == POOL && t == 0 && a.warm && (kind == 0 || CROSS)) {
        const uint32_t ta = tmem + lane_addr + buf * BN;
        const float f = (CROSS && kind == 1)
                            ? warm_floor<KP, true>(ta, c0, ncol, a.n, a.self_excl, my_row, a.cam, my_cam, lane)
                            : warm_floor<KP, false>(ta, c0, ncol, a.n, a.self_excl, my_row, a.cam, my_cam, lane);
        me.floor = fmaxf(me.floor, f);
        me.tau = fmaxf(me.tau, f);
      }
      if (pair_row) {  // fmaxf ignores the NaN of a threshold not yet written
        me.floor = fmaxf(me.floor, tau_other);
        me.tau = fmaxf(me.tau, tau_other);
      }
      // cross-camera pools: the column cameras of chunk ch + 1 are loaded while chunk ch is
      // processed, so one load latency per tile is exposed instead of one per chunk
      int cam_next = 0;
      if (MODE == POOL && CROSS && kind == 1) cam_next = (c0 + lane < a.n) ? a.cam[c0 + lane] : -1;
      for (int ch = 0; ch < BN / 32; ++ch) {
        if (ch * 32 >= ncol) break;
        float v[32];
        tmem_ld32(tmem + lane_addr + buf * BN + ch * 32, v);
        const int cb = c0 + ch * 32;
        int cam_cur = 0;
        if (MODE == POOL && CROSS && kind == 1) {
          cam_cur = cam_next;
          if ((ch + 1) * 32 < ncol) cam_next = (cb + 32 + lane < a.n) ? a.cam[cb + 32 + lane] : -1;
        }
        if (MODE == GPOOL) {
          if (kind == 0 || CROSS) {
            int ccam = 0;
            if (CROSS && kind == 1) ccam = (cb + lane < cend) ? a.cam[cb + lane] : -1;
            const float hb = (cb + lane < cend) ? a.col_bias[cb + lane] : 0.f;
            float2* myq = qs + qrow * kQCap;
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] -= __shfl_sync(GCR_FULL, hb, c);  // biased scores
            const int r0w = g_row0 + quad * 32;  // first row of this warp (rows are not 32-aligned)
            if (cb + 32 > cend || (a.self_excl && cb < r0w + 32 && cb + 32 > r0w)) {
#pragma unroll
              for (int c = 0; c < 32; ++c)
                if (cb + c >= cend || (a.self_excl && cb + c == my_row)) v[c] = -CUDART_INF_F;
            }
            // four values at a time, as in the POOL mode
#pragma unroll
            for (int g = 0; g < 8; ++g) {
              const float m4 = fmaxf(fmaxf(v[4 * g], v[4 * g + 1]), fmaxf(v[4 * g + 2], v[4 * g + 3]));
              if (!VOTE || __any_sync(GCR_FULL, m4 > me.tau)) {
                pool_make_room<KP>(4, lane, me, r0w, kind * BM + quad * 32, qs, pv, pi);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  const int cc = g * 4 + c;
                  const int cj = (CROSS && kind == 1) ? __shfl_sync(GCR_FULL, ccam, cc) : 0;
                  const bool eligible = !(CROSS && kind == 1) || cj != my_cam;
                  if (VOTE) {
                    if (eligible && v[cc] > me.tau) {
                      myq[me.qcnt ^ sw] = make_float2(v[cc], __int_as_float(cb + cc));
                      ++me.qcnt;
                    }
                  } else {
                    pool_push(me, v[cc], cb + cc, eligible, myq, sw);  // branch-free append
                  }
                }
              }
            }
          }
        } else if (MODE == POOL) {
          if (kind == 0 || CROSS) {
            int ccam = 0;
            if (CROSS && kind == 1) ccam = cam_cur;
            float2* myq = qs + qrow * kQCap;
            const int r0w = tl.rb * BM + quad * 32;  // first row of this warp
            if (VOTE) {
              // Where few scores pass (a long sweep for the pool size, or admission floors),
              // most groups of four fall below every row's threshold: one vote over the warp
              // skips them. The chunk on the warp's diagonal (each row meets itself) and the
              // ragged last chunk first get their excluded columns set to -inf. The queues get
              // room every 4 values; votes and shuffles run on every lane.
              if (cb + 32 > a.n || (a.self_excl && cb == r0w)) {
#pragma unroll
                for (int c = 0; c < 32; ++c)
                  if (cb + c >= a.n || (a.self_excl && cb + c == my_row)) v[c] = -CUDART_INF_F;
              }
#pragma unroll
              for (int g = 0; g < 8; ++g) {
                const float m4 = fmaxf(fmaxf(v[4 * g], v[4 * g + 1]), fmaxf(v[4 * g + 2], v[4 * g + 3]));
                if (__any_sync(GCR_FULL, m4 > me.tau)) {
                  pool_make_room<KP>(4, lane, me, r0w, kind * BM + quad * 32, qs, pv, pi);
#pragma unroll
                  for (int c = 0; c < 4; ++c) {
                    const int cc = g * 4 + c;
                    // every lane of the warp (kind is the warp's) takes the camera of column cc
                    const int cj = (CROSS && kind == 1) ? __shfl_sync(GCR_FULL, ccam, cc) : 0;
                    if ((!(CROSS && kind == 1) || cj != my_cam) && v[cc] > me.tau) {
                      myq[me.qcnt ^ sw] = make_float2(v[cc], __int_as_float(cb + cc));
                      ++me.qcnt;
                    }
                  }
                }
              }
            } else if (HEAP) {
              // Per-value path with heap pools: a score that passes goes to the row's queue
              // (a predicated shared store); every 4 values, if any lane's queue could not take
              // 4 more, all lanes drain their queues into their heaps. A group of four that no
              // row of the warp admits (its max at or below every lane's threshold; thresholds
              // only rise, so none of it could enter later) is skipped after one vote: with
              // first-tile floors and the paired halves' exchanged thresholds that is most
              // groups past the first tiles. The excluded columns (past n, and each row itself
              // on the warp's diagonal chunk) are set to -inf once per chunk; the global pool's
              // warps compare against a camera no column has.
              if (cb + 32 > a.n || (a.self_excl && cb == r0w)) {
#pragma unroll
                for (int c = 0; c < 32; ++c)
                  if (cb + c >= a.n || (a.self_excl && cb + c == my_row)) v[c] = -CUDART_INF_F;
              }
              const int cmp_cam = (CROSS && kind == 1) ? my_cam : -2;
#pragma unroll
              for (int g = 0; g < 8; ++g) {
                const float m4 = fmaxf(fmaxf(v[4 * g], v[4 * g + 1]), fmaxf(v[4 * g + 2], v[4 * g + 3]));
                if (!__any_sync(GCR_FULL, m4 > me.tau)) continue;
                if (__any_sync(GCR_FULL, me.qcnt > kHeapQ - 4)) {
                  const HeapState hs = heap_drain<KP>(haddr, qaddr, me.qcnt, me.len, me.tau, me.floor);
                  me.tau = hs.tau;
                  me.len = hs.len;
                  me.qcnt = 0;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  const int cc = g * 4 + c;
                  const int cj = CROSS ? __shfl_sync(GCR_FULL, ccam, cc) : 0;
                  if (cj != cmp_cam && v[cc] > me.tau) {
                    hqp[me.qcnt * BM] = make_float2(v[cc], __int_as_float(cb + cc));
                    ++me.qcnt;
                  }
                }
              }
            } else {
              // Where many scores pass, every value goes through the branch-free append; the
              // queues are checked every 4 values, so they fill to 28 of 32 slots before a merge
              // (every 8: 24; measured 2.82 -> 2.73 ms per TF32 launch, every 2 is slower again).
              // The excluded columns (past n, and each row itself on the warp's diagonal chunk)
              // are set to -inf once per chunk, so the append tests only the score (and, in the
              // cross-camera warps, the column's camera).
              if (cb + 32 > a.n || (a.self_excl && cb == r0w)) {
#pragma unroll
                for (int c = 0; c < 32; ++c)
                  if (cb + c >= a.n || (a.self_excl && cb + c == my_row)) v[c] = -CUDART_INF_F;
              }
              if (CROSS && kind == 1) {  // warp-uniform
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                  pool_make_room<KP>(4, lane, me, r0w, kind * BM + quad * 32, qs, pv, pi);
#pragma unroll
                  for (int c = 0; c < 4; ++c) {
                    const int cc = g * 4 + c;
                    const int cj = __shfl_sync(GCR_FULL, ccam, cc);
                    pool_push(me, v[cc], cb + cc, cj != my_cam, myq, sw);
                  }
                }
              } else {
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                  pool_make_room<KP>(4, lane, me, r0w, kind * BM + quad * 32, qs, pv, pi);
#pragma unroll
                  for (int c = 0; c < 4; ++c) pool_push(me, v[g * 4 + c], cb + g * 4 + c, true, myq, sw);
                }
              }
            }
          }
        } else if (MODE == BAND) {
          if (kind == 0) {
            int ccam = 0;
            if (a.cam) ccam = (cb + lane < a.n) ? a.cam[cb + lane] : -1;
#pragma unroll
            for (int cc = 0; cc < 32; ++cc) {
              const int j = cb + cc;
              const int cjv = __shfl_sync(GCR_FULL, ccam, cc);
              const int cj = a.cam ? cjv : 0;
              if (u < 0 || j >= a.n || (a.self_excl && j == my_row) || v[cc] < my_thr) continue;
              if (my_kind == 1 && cj == my_cam) continue;
              const int pos = atomicAdd(&a.band_cnt[u], 1);
              if (pos < (a.band_lim ? a.band_lim[u] : a.bcap)) {
                const size_t at = (a.band_off ? (size_t)a.band_off[u] : (size_t)u * a.bcap) + pos;
                if (a.band_v) a.band_v[at] = v[cc];
                a.band_i[at] = j;
              }
            }
          }
        } else if (MODE == MUL) {
          if (kind == 0 && my_row < a.a_rows) {
            float* out = a.D + (size_t)my_row * a.n + cb;
#pragma unroll
            for (int cc = 0; cc < 32; ++cc)
              if (cb + cc < a.n) out[cc] = v[cc];
          }
        } else if (MODE == GRAM) {
          if (kind == 0 && my_row < a.a_rows) {
            float* out = a.G + ((size_t)blockIdx.z * a.a_rows + my_row) * a.n + cb;
            const bool none = gram_kn == 0;  // a camera without frames: no MMA wrote the accumulator
#pragma unroll
            for (int cc = 0; cc < 32; ++cc)
              if (cb + cc < a.n) out[cc] = (none ? 0.f : v[cc]) + (cb + cc == my_row ? my_nq : 0.f);
          }
        } else {
          if (kind == 0) {
            const float ngv = (cb + lane < a.n) ? a.nrm_g[cb + lane] : 0.f;
            const bool row_ok = my_row < a.a_rows;
            float* out = a.D + (size_t)(row_ok ? my_row : 0) * a.n + cb;
#pragma unroll
            for (int cc = 0; cc < 32; ++cc) {
              const float g = __shfl_sync(GCR_FULL, ngv, cc);
              if (row_ok && cb + cc < a.n) out[cc] = my_nq + g - 2.f * v[cc];
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.tempty[buf]);
      if (pair_row) __stcg(a.tau_x + tx_mine, me.tau);
      if (g_last && (kind == 0 || CROSS))
        pool_flush<KP>(lane, g_valid, me, g_row0 + quad * 32, kind * BM + quad * 32, qs, pv, pi);
    }
    if (MODE == POOL && (kind == 0 || CROSS) && !*abort_flag) {
      if (HEAP) {
        if (__any_sync(GCR_FULL, me.qcnt > 0)) {
          const HeapState hs = heap_drain<KP>(haddr, qaddr, me.qcnt, me.len, me.tau, me.floor);
          me.len = hs.len;
          me.qcnt = 0;
        }
        if (my_row < a.a_rows) heap_emit<KP>(haddr, me.len, pv + (size_t)my_row * KP, pi + (size_t)my_row * KP);
        if (a.pair) {
          // the list is written: make it visible, count this warp, and merge if it is second
          // (the stage buffers are idle by now and hold the other half's lists)
          __threadfence();
          __syncwarp();
          int prev = 0;
          if (lane == 0) prev = atomicAdd(a.pair_cnt + ((size_t)tl.rb * (CROSS ? 2 : 1) + kind) * 4 + quad, 1);
          prev = __shfl_sync(GCR_FULL, prev, 0);
          if (prev == 1) {
            __threadfence();
            const size_t ro = ((size_t)(tl.split ^ 1) * (CROSS ? 2 : 1) + kind) * a.a_rows * KP;  // the other half
            const size_t r0s = (size_t)kind * a.a_rows * KP;                                   // split 0's pools
            const float2* own = reinterpret_cast<const float2*>(dyn + NS * STAGE_BYTES) + kind * KP * BM + r;
            float2* scratch = reinterpret_cast<float2*>(stages) + kind * KP * BM + r;
            if (my_row < a.a_rows)
              pair_merge_lists<KP>(own, me.len, a.pool_v + ro + (size_t)my_row * KP, a.pool_i + ro + (size_t)my_row * KP,
                                   scratch, a.pool_v + r0s + (size_t)my_row * KP, a.pool_i + r0s + (size_t)my_row * KP);
          }
        }
      } else {
        pool_flush<KP>(lane, my_row < a.a_rows, me, tl.rb * BM + quad * 32, kind * BM + quad * 32, qs, pv, pi);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // clusters: neither CTA leaves while the other may still signal its barriers (its MMAs have
  // drained by now) or write its stages
  if (MODE == POOL && a.mc) cluster_sync_all();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// Self-test of the bounded wait: one warp waits on an mbarrier that nothing signals; the wait
// gives up after limit_ns, counts a timeout (reported by gcr_sync) and the kernel returns.
__global__ void wait_probe_kernel(unsigned long long limit_ns, int* result) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool ok = true;
  if (threadIdx.x == 0) ok = mbar_wait(&bar, 0, &abort_flag, limit_ns);
  __syncthreads();
  if (threadIdx.x == 0 && result) *result = ok ? 1 : 0;
}

// ------------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Row-major matrix [rows][d] (BF16, or TF32 held as FP32) viewed as a 2-D tensor, box = 128
// bytes of K x box_rows; K past d reads as zero.
cudaError_t make_map(CUtensorMap* m, const void* base, Elt elt, int rows, int d, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const size_t es = elt_bytes(elt);
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((size_t)d * es) % 16) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(d * es)};
  cuuint32_t box[2] = {(cuuint32_t)(BKB / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, elt == Elt::TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t smem_bytes(int mode, bool heap = false) {
  if (mode != POOL && mode != GPOOL) return 1024 + (size_t)NST_MAX * STAGE_BYTES;
  size_t s = 1024 + (size_t)NST * STAGE_BYTES;
  if (heap) s += 2 * (32 + kHeapQ) * BM * sizeof(float2);
  else s += 2 * BM * kQCap * (sizeof(float) + sizeof(int));
  return s;
}

template <int MODE, int KP, bool CROSS, bool VOTE = false>
cudaError_t launch(const CUtensorMap& ta, const CUtensorMap& tb, const UmmaArgs& a, dim3 grid, cudaStream_t st,
                   const CUtensorMap* ta2 = nullptr, const CUtensorMap* tb2 = nullptr, dim3 cluster = dim3(1, 1, 1)) {
  auto fn = umma_kernel<MODE, KP, CROSS, VOTE>;
  const size_t smem = smem_bytes(a.mode, MODE == POOL && KP == 32 && !VOTE);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster.x * cluster.y * cluster.z == 1) {
    fn<<<grid, CROSS ? 320 : 192, smem, st>>>(ta, tb, ta2 ? *ta2 : ta, tb2 ? *tb2 : tb, a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(CROSS ? 320 : 192, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster.x;
  at[0].val.clusterDim.y = cluster.y;
  at[0].val.clusterDim.z = cluster.z;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, ta, tb, ta2 ? *ta2 : ta, tb2 ? *tb2 : tb, a);
}

}  // namespace

cudaError_t launch_wait_probe(unsigned long long limit_ns, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(limit_ns, nullptr);
  return cudaGetLastError();
}

int umma_read_and_clear_timeouts() {
  int h = 0, z = 0;
  if (cudaMemcpyFromSymbol(&h, g_umma_timeouts, sizeof(int)) != cudaSuccess) return -1;
  if (h) cudaMemcpyToSymbol(g_umma_timeouts, &z, sizeof(int));
  return h;
}

cudaError_t launch_umma_pool(const void* Ab, int na, const void* Bb, int nb, int d, Elt elt,
                             const int* cam, bool cross, int self_excl, int kp, int splits, float* pool_v,
                             int* pool_i, cudaStream_t st, const float* seed, float* tau_x, int* pair_cnt) {
  CUtensorMap ta, tb;
  cudaError_t e = make_map(&ta, Ab, elt, na, d, BM);
  if (e != cudaSuccess) return e;
  e = make_map(&tb, Bb, elt, nb, d, BN);
  if (e != cudaSuccess) return e;
  const int ntiles = (nb + BN - 1) / BN;
  const int rblocks = (na + BM - 1) / BM;
  // Paired splits (heap pools only) where the A blocks of one CTA per SM would not fit in half
  // the L2: each CTA re-reads its A block for every column tile, and 151 blocks of 128 x 2048
  // TF32 rows (151 MB) would otherwise come from DRAM every time.
  int l2 = 0, nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const double live_a = (double)std::min(rblocks, std::max(nsm, 1)) * BM * d * (double)elt_bytes(elt);
  // expected share of a split's scores that enter a row's pool, in random order: about
  // kp (1 + ln(columns / kp)) / columns; a vote pays where that is small (or with floors)
  auto admit_share = [&](int tiles_per_split) {
    const double cols = (double)std::min(nb, tiles_per_split * BN);
    return cols > kp ? kp * (1.0 + std::log(cols / kp)) / cols : 1.0;
  };
  const bool pair = kp == 32 && !seed && tau_x && pair_cnt && splits <= 1 && ntiles >= 2 && l2 > 0 &&
                    live_a > 0.5 * l2 && admit_share((ntiles + 1) / 2) >= 0.006;
  if (pair) splits = 2;
  if (splits < 1) splits = 1;
  if (splits > ntiles) splits = ntiles;
  const int tps = (ntiles + splits - 1) / splits;
  splits = (ntiles + tps - 1) / tps;  // no split is left without a column tile
  UmmaArgs a{};
  a.mode = POOL;
  a.tf32 = elt == Elt::TF32;
  a.n = nb;
  a.d = d;
  a.a_rows = na;
  a.self_excl = self_excl;
  a.tps = tps;
  a.cam = cam;
  a.pool_v = pool_v;
  a.pool_i = pool_i;
  a.seed = seed;
  a.vote = (seed != nullptr || admit_share(tps) < 0.006) ? 1 : 0;
  a.warm = 1;
  dim3 grid(rblocks, splits);
  // heap pools: 2-CTA clusters over row blocks (an even count: a last block past na has no
  // rows and only loads its half of the shared B tiles)
  const bool heap = kp == 32 && !a.vote;
  const int rb_grid = heap ? (rblocks + 1) & ~1 : rblocks;
  CUtensorMap tb_half;
  dim3 cluster(1, 1, 1);
  if (heap) {
    e = make_map(&tb_half, Bb, elt, nb, d, BN / 2);
    if (e != cudaSuccess) return e;
    a.mc = 1;
    grid = dim3(rb_grid, splits);
    cluster = dim3(2, 1, 1);
  }
  if (pair) {  // no vote: the admission share was checked for these splits
    const int pools = cross ? 2 : 1;
    cudaError_t e2 = cudaMemsetAsync(tau_x, 0xFF, sizeof(float) * 2 * pools * (size_t)na, st);  // NaN
    if (e2 == cudaSuccess) e2 = cudaMemsetAsync(pair_cnt, 0, sizeof(int) * (size_t)rb_grid * pools * 4, st);
    if (e2 != cudaSuccess) return e2;
    a.pair = 1;
    a.tau_x = tau_x;
    a.pair_cnt = pair_cnt;
    grid = dim3(2, rb_grid);
    cluster = dim3(1, 2, 1);
  }
  if (heap) {
    return cross ? launch<POOL, 32, true>(ta, tb, a, grid, st, nullptr, &tb_half, cluster)
                 : launch<POOL, 32, false>(ta, tb, a, grid, st, nullptr, &tb_half, cluster);
  }
  if (a.vote) {
    if (kp == 32) return cross ? launch<POOL, 32, true, true>(ta, tb, a, grid, st) : launch<POOL, 32, false, true>(ta, tb, a, grid, st);
    if (kp == 64) return cross ? launch<POOL, 64, true, true>(ta, tb, a, grid, st) : launch<POOL, 64, false, true>(ta, tb, a, grid, st);
    if (kp == 128) return cross ? launch<POOL, 128, true, true>(ta, tb, a, grid, st) : launch<POOL, 128, false, true>(ta, tb, a, grid, st);
    return cudaErrorInvalidValue;
  }
  if (kp == 32) return cross ? launch<POOL, 32, true>(ta, tb, a, grid, st) : launch<POOL, 32, false>(ta, tb, a, grid, st);
  if (kp == 64) return cross ? launch<POOL, 64, true>(ta, tb, a, grid, st) : launch<POOL, 64, false>(ta, tb, a, grid, st);
  if (kp == 128) return cross ? launch<POOL, 128, true>(ta, tb, a, grid, st) : launch<POOL, 128, false>(ta, tb, a, grid, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_umma_gpool(const void* Y, int rows, int d, Elt elt, const int* gcam, bool cross, int self_excl,
                              int kp, const int4* items, const int* n_items, int max_items, const float* col_bias,
                              float* pool_v, int* pool_i, cudaStream_t st) {
  if (rows < 1 || max_items < 1) return cudaSuccess;
  CUtensorMap ta, tb;
  cudaError_t e = make_map(&ta, Y, elt, rows, d, BM);
  if (e != cudaSuccess) return e;
  e = make_map(&tb, Y, elt, rows, d, BN);
  if (e != cudaSuccess) return e;
  UmmaArgs a{};
  a.mode = GPOOL;
  a.tf32 = elt == Elt::TF32;
  a.n = rows;
  a.d = d;
  a.a_rows = rows;
  a.self_excl = self_excl;
  a.cam = gcam;
  a.pool_v = pool_v;
  a.pool_i = pool_i;
  a.items = items;
  a.n_items = n_items;
  a.col_bias = col_bias;
  a.vote = 1;
  // persistent: one CTA per SM (the POOL shared memory allows one), items strided over the grid
  dim3 grid((unsigned)std::max(1, std::min(max_items, 152)));
  if (kp == 32) return cross ? launch<GPOOL, 32, true, true>(ta, tb, a, grid, st) : launch<GPOOL, 32, false, true>(ta, tb, a, grid, st);
  if (kp == 64) return cross ? launch<GPOOL, 64, true, true>(ta, tb, a, grid, st) : launch<GPOOL, 64, false, true>(ta, tb, a, grid, st);
  if (kp == 128) return cross ? launch<GPOOL, 128, true, true>(ta, tb, a, grid, st) : launch<GPOOL, 128, false, true>(ta, tb, a, grid, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_umma_band(const void* Xb, int n, int d, Elt elt, const int* cam, int self_excl,
                             const void* Ab, const int* count, int cap, const int* band_row,
                             const int* band_kind, const float* band_thr, int bcap, int* band_cnt, float* band_v,
                             int* band_i, cudaStream_t st, const int* band_off, const int* band_lim) {
  CUtensorMap ta, tb;
  cudaError_t e = make_map(&ta, Ab, elt, cap, d, BM);
  if (e != cudaSuccess) return e;
  e = make_map(&tb, Xb, elt, n, d, BN);
  if (e != cudaSuccess) return e;
  UmmaArgs a{};
  a.mode = BAND;
  a.tf32 = elt == Elt::TF32;
  a.n = n;
  a.d = d;
  a.a_rows = cap;
  a.self_excl = self_excl;
  a.cam = cam;
  a.count = count;
  a.cap = cap;
  a.band_row = band_row;
  a.band_kind = band_kind;
  a.band_thr = band_thr;
  a.bcap = bcap;
  a.band_cnt = band_cnt;
  a.band_v = band_v;
  a.band_i = band_i;
  a.band_off = band_off;
  a.band_lim = band_lim;
  // the row tiles (known only on the device) are strided over grid.y so that the grid covers
  // the GPU about twice even when the columns give few tiles
  const int gx = (n + BN - 1) / BN;
  const int gy = std::max(1, std::min(8, (2 * 152 + gx - 1) / gx));
  dim3 grid(gx, gy);
  return launch<BAND, 64, false>(ta, tb, a, grid, st);
}

cudaError_t launch_umma_dist(const __nv_bfloat16* Qb, int nq, const __nv_bfloat16* Gb, int ng, int d,
                             const float* nrm_q, const float* nrm_g, float* D, cudaStream_t st) {
  CUtensorMap ta, tb;
  cudaError_t e = make_map(&ta, Qb, Elt::BF16, nq, d, BM);
  if (e != cudaSuccess) return e;
  e = make_map(&tb, Gb, Elt::BF16, ng, d, BN);
  if (e != cudaSuccess) return e;
  UmmaArgs a{};
  a.mode = DIST;
  a.n = ng;
  a.d = d;
  a.a_rows = nq;
  a.nrm_q = nrm_q;
  a.nrm_g = nrm_g;
  a.D = D;
  // persistent: one CTA per SM walks its tiles, so the MMAs of a tile overlap the epilogue of
  // the previous one (double-buffered accumulators)
  a.dist_nrb = (nq + BM - 1) / BM;
  a.dist_tiles = a.dist_nrb * ((ng + BN - 1) / BN);
  dim3 grid((unsigned)std::max(1, std::min(a.dist_tiles, 152)));
  return launch<DIST, 64, false>(ta, tb, a, grid, st);
}

cudaError_t launch_umma_gram(const __nv_bfloat16* zt_hi, const __nv_bfloat16* zt_lo, int d, int64_t cols,
                             const int64_t* kstart, const int64_t* knum, const int64_t* nf, int ncam, float lambda,
                             float* G, cudaStream_t st) {
  if (cols > INT32_MAX || cols % 8) return cudaErrorInvalidValue;
  CUtensorMap ta, tb, ta2, tb2;
  cudaError_t e = make_map(&ta, zt_hi, Elt::BF16, d, (int)cols, BM);
  if (e != cudaSuccess) return e;
  e = make_map(&tb, zt_hi, Elt::BF16, d, (int)cols, BN);
  if (e != cudaSuccess) return e;
  e = make_map(&ta2, zt_lo, Elt::BF16, d, (int)cols, BM);
  if (e != cudaSuccess) return e;
  e = make_map(&tb2, zt_lo, Elt::BF16, d, (int)cols, BN);
  if (e != cudaSuccess) return e;
  UmmaArgs a{};
  a.mode = GRAM;
  a.n = d;
  a.d = 64;  // unused: the K extent of a tile comes from gram_knum
  a.a_rows = d;
  a.gram_kstart = kstart;
  a.gram_knum = knum;
  a.gram_nf = nf;
  a.gram_lambda = lambda;
  a.G = G;
  dim3 grid((d + BN - 1) / BN, (d + BM - 1) / BM, ncam);
  return launch<GRAM, 64, false>(ta, tb, a, grid, st, &ta2, &tb2);
}

cudaError_t launch_umma_mul(const float* p_hi, const float* p_lo, int rows, const float* g_hi, const float* g_lo,
                            int ncam, int d, const int* rowcam, float* Q, cudaStream_t st) {
  CUtensorMap ta, tb, ta2, tb2;
  cudaError_t e = make_map(&ta, p_hi, Elt::TF32, rows, d, BM);
  if (e != cudaSuccess) return e;
  e = make_map(&ta2, p_lo, Elt::TF32, rows, d, BM);
  if (e != cudaSuccess) return e;
  e = make_map(&tb, g_hi, Elt::TF32, ncam * d, d, BN);
  if (e != cudaSuccess) return e;
  e = make_map(&tb2, g_lo, Elt::TF32, ncam * d, d, BN);
  if (e != cudaSuccess) return e;
  UmmaArgs a{};
  a.mode = MUL;
  a.tf32 = 1;
  a.n = d;
  a.d = d;
  a.a_rows = rows;
  a.mul_rowcam = rowcam;
  a.D = Q;
  dim3 grid((d + BN - 1) / BN, (rows + BM - 1) / BM);
  return launch<MUL, 64, false>(ta, tb, a, grid, st, &ta2, &tb2);
}

}  // namespace gcr
