// Certified kNN search, inside a shared ball and in centred coordinates, of the (row, graph)
// pairs whose candidate pool could not certify the k-th neighbour (N_i of Eq. 4, N_i^cr of
// Eq. 8, graphs rebuilt at every iteration of Eq. 3).
//
// Propagation contracts every cluster towards its mean, so after a few layers the members of
// a large cluster are nearly identical: their scores s_ij = x_i . x_j differ by less than the
// rounding bound of any FP32 or tensor-core dot product, no pool certifies the k-th neighbour
// and a threshold rescan returns the whole cluster. The distances are still well resolved:
// ||x_i - x_j||^2 = ||y_i - y_j||^2 with y = x - c for any centre c, and with c inside the
// cluster the rounding bound of y_i . y_j scales with ||y_i|| ||y_j|| (the cluster's radius
// squared) instead of ||x_i|| ||x_j|| = 1. For the pending pairs of one search:
//  1. groups: the connected components, by a lock-free union-find, of the graph that links a
//     pending pair (i, graph) to each j among the first k entries of its pool whose own k-th
//     distance bound (same graph) is within a factor kScaleRatio of i's: rows of one contracted
//     cluster share a local scale, while a row whose k-th neighbour lies in another cluster
//     (a cluster smaller than k) has a far larger one and does not chain clusters together;
//     Only pairs that can be in a searched ball take part (ball_participates: a dense pair, or
//     one whose k-th distance bound is at most a quarter of its squared norm), and the search
//     runs only when some pair is dense or kMinBallPairs take part;
//  2. group g gets the centre c_g = x_{r_g}, r_g its smallest member, and the radius
//     R_g = max over its pairs of ||x_i - c_g|| + sqrt(Dbar), Dbar an upper bound on the pair's
//     exact k-th squared distance (from its refined pool): by the triangle inequality every
//     exact neighbour of every pair of g lies in the ball B(c_g, R_g);
//  3. a threshold sweep of the centres against all rows (the tensor-core kernel's BAND mode,
//     in two passes: count, then fill at scanned offsets) lists each ball's members, a superset
//     that allows for the sweep's rounding bound; balls holding more than half of the rows, or
//     beyond the gathered capacity, are not searched (their pairs go to the threshold rescan),
//     nor, unless a pair's band is predicted to overflow, groups of fewer than kMinGroupRows
//     pending rows or whose ball is not contracted (R^2 > ||c||^2 / 4): the rescan is cheaper;
//  4. each ball's members are gathered, centred (y = fl(x - c_g)) and rounded to the GEMM's
//     operand type, the group's pending rows first, with per-position norms and per-group
//     maxima for the rounding bounds;
//  5. work items for the grouped pool GEMM: 128 pending rows of a group against its members.
// The grouped GEMM (umma.cu, GPOOL) and the refinement of its pools (refine.cu) follow.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

constexpr double kU32b = 5.9604644775390625e-08;  // 2^-24
constexpr float kScaleRatio = 8.f;  // largest ratio of the k-th distance bounds of linked rows
// A group of fewer pending rows than this, none of them predicted to overflow the band, is left
// to the threshold rescan: its ball sweep and 128-row GEMM tiles cost more than their rows' sweeps.
constexpr int kMinGroupRows = 8;
// With no pair predicted to overflow the band and fewer taking part than this, the whole ball
// search is skipped (its fixed cost, a few sweeps and GEMM tiles, exceeds the rescan of so few
// pairs); every pending pair then goes to the threshold rescan, which certifies them exactly.
constexpr int kMinBallPairs = 1024;

__device__ __forceinline__ bool ball_go(const BallArgs& a) {
  return *a.ndense > 0 || *a.npart >= kMinBallPairs;
}

// Union-find over row indices. Every parent pointer goes to a smaller or equal index, so a find
// ends after at most x steps. Parents are read and written through L2 (ld/st.cg): the atomics
// that link roots live there, and an L1 copy could be stale.
__device__ __forceinline__ int uf_find(int* parent, int x) {
  for (;;) {
    const int p = __ldcg(parent + x);
    if (p == x) return x;
    const int gp = __ldcg(parent + p);
    if (gp != p) __stcg(parent + x, gp);  // path halving: gp is an ancestor of x
    x = p;
  }
}

// Links the trees of a and b (the larger root under the smaller). Lock-free: a failed CAS means
// another thread linked that root, so the number of roots fell; the retry bound is never reached
// in practice and reports an error instead of looping on.
__device__ __forceinline__ bool uf_unite(int* parent, int a, int b) {
  for (int it = 0; it < (1 << 20); ++it) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return true;
    if (a < b) { const int t = a; a = b; b = t; }
    if (atomicCAS(parent + a, a, b) == a) return true;
  }
  return false;
}

// Node ids: the A rows (the rows searched) are nodes 0 .. na-1; in a search against a gallery
// (two = 1) the B rows (the gallery) are nodes na .. na+nb-1, otherwise B is A.
__device__ __forceinline__ int node_count(const BallArgs& a) { return a.two ? a.na + a.nb : a.na; }
__device__ __forceinline__ const float* node_row(const BallArgs& a, int v) {
  return (a.two && v >= a.na) ? a.XB + (size_t)(v - a.na) * a.d : a.XA + (size_t)v * a.d;
}

__global__ void ball_init_kernel(BallArgs a) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < node_count(a)) {
    a.parent[v] = v;
    a.acnt[v] = 0;
    a.rad[v] = 0.f;
    a.active[v] = 0;
    a.seen[v] = 0;
    a.rdense[v] = 0;
  }
  if (v < a.na) {
    a.pend[v] = 0;
    a.pos_of_row[v] = -1;
    a.root_of_row[v] = -1;
  }
  if (a.two && v < a.nb) a.gscale[v] = CUDART_INF_F;
  if (v == 0) {
    *a.npart = 0;
    *a.ndense = 0;
  }
}

__global__ void ball_mark_kernel(BallArgs a) {
  const int U = min(*a.unc_count, a.unc_cap);
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x) {
    const int i = a.unc_row[u];
    if (ball_participates(a.unc_dk[u], a.n64A[i])) {
      atomicOr(a.pend + i, 1 << a.unc_kind[u]);
      atomicAdd(a.npart, 1);
      if (a.unc_dk[u] < 0.f) atomicAdd(a.ndense, 1);
    }
  }
}

// Approximate squared distance of pending row i to its pool entry s (against a gallery).
__device__ __forceinline__ float pool_d2(const BallArgs& a, int i, int kind, int s, int j) {
  const float v = a.pool_v[((size_t)kind * a.na + i) * a.kp + s];
  return fmaxf(0.f, (float)(a.n64A[i] + a.n64B[j]) - 2.f * v);
}

// Against a gallery, a gallery row has no kNN list of its own: its local scale is the smallest
// approximate squared distance at which a pending row lists it among its first k candidates.
__global__ void ball_scale_kernel(BallArgs a) {
  if (!ball_go(a)) return;
  const int lane = threadIdx.x & 31;
  const int U = min(*a.unc_count, a.unc_cap);
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < U; u += nw) {
    const int i = a.unc_row[u], kind = a.unc_kind[u];
    if (!ball_participates(a.unc_dk[u], a.n64A[i])) continue;
    const int* pi = a.pool_i + ((size_t)kind * a.na + i) * a.kp;
    for (int s = lane; s < a.k; s += 32) {
      const int j = pi[s];
      if (j < 0) continue;
      atomicMin(reinterpret_cast<int*>(a.gscale) + j, __float_as_int(pool_d2(a, i, kind, s, j)));
    }
  }
}

// One warp per pending pair: link i with each j of its first k pool entries of a similar local
// scale (within kScaleRatio): among the A rows, the two k-th distance bounds; against a gallery,
// i's distance to j and j's scale.
__global__ void ball_link_kernel(BallArgs a) {
  if (!ball_go(a)) return;
  const int lane = threadIdx.x & 31;
  const int U = min(*a.unc_count, a.unc_cap);
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < U; u += nw) {
    const int i = a.unc_row[u], kind = a.unc_kind[u];
    if (!ball_participates(a.unc_dk[u], a.n64A[i])) continue;
    const int* pi = a.pool_i + ((size_t)kind * a.na + i) * a.kp;
    const float di = a.two ? 0.f : a.dk_all[(size_t)kind * a.na + i];
    for (int s = lane; s < a.k; s += 32) {
      const int j = pi[s];
      if (j < 0 || (!a.two && j == i)) continue;
      bool link;
      if (a.two) {
        link = pool_d2(a, i, kind, s, j) <= kScaleRatio * a.gscale[j];
      } else {
        const float dj = a.dk_all[(size_t)kind * a.na + j];
        link = di <= kScaleRatio * dj && dj <= kScaleRatio * di;
      }
      if (link && !uf_unite(a.parent, i, a.two ? a.na + j : j)) atomicOr(a.err, 1);
    }
  }
}

// One warp per pending pair: the pair's root, its contribution to the group radius
// (||x_i - c|| + sqrt(Dbar), rounded up) and, once per row, the group's pending-row count.
__global__ void ball_root_kernel(BallArgs a) {
  if (!ball_go(a)) return;
  const int lane = threadIdx.x & 31;
  const int U = min(*a.unc_count, a.unc_cap);
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < U; u += nw) {
    const int i = a.unc_row[u], kind = a.unc_kind[u];
    if (!ball_participates(a.unc_dk[u], a.n64A[i])) continue;  // the same value on every lane
    int root = 0;
    if (lane == 0) root = uf_find(a.parent, i);
    root = __shfl_sync(GCR_FULL, root, 0);
    const float4* xi = reinterpret_cast<const float4*>(a.XA + (size_t)i * a.d);
    const float4* xc = reinterpret_cast<const float4*>(node_row(a, root));
    float ss = 0.f;
    for (int v = lane; v < (a.d >> 2); v += 32) {
      const float4 p = xi[v], q = xc[v];
      const float e0 = p.x - q.x, e1 = p.y - q.y, e2 = p.z - q.z, e3 = p.w - q.w;
      ss = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, ss))));
    }
    ss = warp_sum(ss);
    if (lane == 0) {
      // FP32 differences and sums carry a relative error below (d + 2) * 2^-24 <= 2.5e-4 (d <= 4096)
      const double dist = sqrt((double)ss * (1.0 + 1e-3));
      const float dk = a.unc_dk[u];  // negative: the refinement predicted an overflowing band
      const double R = (dist + sqrt((double)fabsf(dk))) * (1.0 + 1e-6) + 1e-12;
      atomicMax(reinterpret_cast<int*>(a.rad) + root, __float_as_int(__double2float_ru(R)));
      a.seen[root] = 1;
      if (dk < 0.f) a.rdense[root] = 1;
      a.root_of_row[i] = root;
      const int pm = a.pend[i];
      if ((pm & ((1 << kind) - 1)) == 0) atomicAdd(a.acnt + root, 1);  // lowest pending graph of the row
    }
  }
}

// The groups searched: roots with a pair whose band the refinement predicted to overflow, or with
// at least kMinGroupRows pending rows in a contracted ball (R^2 <= ||c||^2 / 4: centring shrinks
// the rounding bound by (R / ||c||)^2, so a wider ball gains too little over the rescan); the
// others' pairs go to the threshold rescan.
__global__ void ball_elig_kernel(BallArgs a) {
  const bool go = ball_go(a);
  if (go && blockIdx.x == 0 && threadIdx.x == 0 && a.stats)
    atomicAdd(a.stats + GCR_STAT_BALL_PAIRS, (unsigned long long)*a.npart);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < node_count(a); v += gridDim.x * blockDim.x) {
    const double nc = (a.two && v >= a.na) ? a.n64B[v - a.na] : a.n64A[v];
    const double R = (double)a.rad[v];
    const bool contracted = R * R <= 0.25 * nc;
    a.active[v] = (go && a.seen[v] && (a.rdense[v] || (a.acnt[v] >= kMinGroupRows && contracted))) ? 1 : 0;
  }
}

// Group table from the scanned active flags; the sweep threshold of each centre:
// ||x_j - c||^2 <= R^2 implies s_cj >= (||x_j||^2 + ||c||^2 - R^2) / 2 >= (nmin + ||c||^2 - R^2) / 2,
// and the approximate score is within delta_c (the GEMM bound of row c against the B rows) of s_cj.
__global__ void ball_group_kernel(BallArgs a) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= node_count(a) || !a.active[r]) return;
  const int g = a.gid[r];
  a.groot[g] = r;
  a.ga[g] = a.acnt[r];
  a.gkind[g] = 0;
  const bool on_b = a.two && r >= a.na;
  const int rr = on_b ? r - a.na : r;
  const double n_c = on_b ? a.n64B[rr] : a.n64A[rr];
  const double an = on_b ? a.anrmB[rr] : a.anrmA[rr];
  const double en = on_b ? a.enrmB[rr] : a.enrmA[rr];
  const RowScalars sc = *a.scB;
  const double bmax = sqrt(sc.nmax) * (1.0 + 1e-12);
  const double R = (double)a.rad[r];
  double delta;
  if (a.precision == GCR_PREC_FP32) {
    delta = (a.d * kU32b / (1.0 - a.d * kU32b)) * sqrt(n_c) * bmax;
  } else {
    const double gacc = (a.d + 32.0) * 2.0 * kU32b / (1.0 - (a.d + 32.0) * 2.0 * kU32b);
    delta = an * sc.emax + en * bmax + gacc * an * sc.amax;
  }
  delta *= 1.0 + 1e-6;
  const double thr = 0.5 * (sc.nmin + n_c - R * R) - delta;
  a.gthr[g] = nextafterf(__double2float_rd(thr), -CUDART_INF_F);
}

// The centres' rounded operand rows (from the A or the B copy), 16 bytes per thread.
__global__ void ball_centres_kernel(BallArgs a) {
  const int G = a.gid[node_count(a)];
  const size_t w16 = (size_t)a.d * (a.elt == Elt::TF32 ? 4 : 2) / 16;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < (size_t)G * w16;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t g = t / w16, c = t % w16;
    const int r = a.groot[g];
    const bool on_b = a.two && r >= a.na;
    const uint4* src = static_cast<const uint4*>(on_b ? a.xrB : a.xrA) + (size_t)(on_b ? r - a.na : r) * w16;
    static_cast<uint4*>(a.cent)[g * w16 + c] = src[c];
  }
}

// Groups searched: a ball no larger than half of the B rows (among the A rows it must also hold
// the group's pending rows; anything else is a numerical impossibility, handled as a failure).
// Segment size: the pending rows plus the ball against a gallery, the ball alone otherwise.
__global__ void ball_route_kernel(BallArgs a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = node_count(a);
  if (g >= nn) return;
  const int G = a.gid[nn];
  int sz = 0;
  if (g < G) {
    const int c = a.gsize[g];
    if (a.two) sz = c <= a.nb / 2 ? a.ga[g] + c : 0;
    else sz = (c <= a.na / 2 && c >= a.ga[g]) ? c : 0;
  }
  a.rsize[g] = sz;
  a.gfill[g] = 0;
  a.afill[g] = 0;
  a.bfill[g] = 0;
  a.gfail[g] = 0;
}

// Capacity cut (segments in scan order), fill-pass thresholds (+inf: not searched), and where
// the fill pass lists each ball: after the pending rows against a gallery, else the segment.
__global__ void ball_cut_kernel(BallArgs a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int G = a.gid[node_count(a)];
  if (g >= G) return;
  const bool fits = a.rsize[g] > 0 && a.goff[g] + a.rsize[g] <= a.cap_rows;
  if (!fits) a.rsize[g] = 0;
  a.gthr_fill[g] = fits ? a.gthr[g] : CUDART_INF_F;
  if (!fits) a.gfail[g] = 1;
  a.boff[g] = a.goff[g] + (a.two ? a.ga[g] : 0);
  a.blim[g] = fits ? (a.two ? a.rsize[g] - a.ga[g] : a.rsize[g]) : 0;
}

__device__ __forceinline__ int group_of(const int* goff, int G, int e) {
  int lo = 0, hi = G;  // largest g with goff[g] <= e
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (goff[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Places each listed member in its group's segment. Among the A rows the list holds the
// group's pending rows too, which go first; against a gallery the list already sits after them.
__device__ __forceinline__ void ball_place_one(const BallArgs& a, int G, int e) {
  const int g = group_of(a.goff, G, e);
  if (a.rsize[g] == 0 || e < a.boff[g] || e >= a.boff[g] + a.blim[g]) return;
  if (a.gfill[g] != a.blim[g]) {  // the fill pass listed a different count than the count pass
    a.gfail[g] = 1;
    return;
  }
  const int j = a.ball_j[e];
  if (a.two) {
    a.gmap[e] = j;
    a.ggrp[e] = g;
    return;
  }
  const int root = a.groot[g];
  const bool is_a = a.pend[j] != 0 && a.root_of_row[j] == root;
  int p;
  if (is_a) {
    const int s = atomicAdd(a.afill + g, 1);
    if (s >= a.ga[g]) { a.gfail[g] = 1; return; }
    p = a.goff[g] + s;
    a.pos_of_row[j] = p;
  } else {
    const int s = atomicAdd(a.bfill + g, 1);
    if (s >= a.rsize[g] - a.ga[g]) { a.gfail[g] = 1; return; }
    p = a.goff[g] + a.ga[g] + s;
  }
  a.gmap[p] = j;
  a.ggrp[p] = g;
}

__global__ void ball_place_kernel(BallArgs a) {
  const int G = a.gid[node_count(a)];
  if (G == 0) return;
  const int E = min(a.goff[G], a.cap_rows);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
    ball_place_one(a, G, e);
}
// Against a gallery: the pending rows of each searched group at the head of its segment.
__global__ void ball_place_rows_kernel(BallArgs a) {
  const int U = min(*a.unc_count, a.unc_cap);
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x) {
    const int i = a.unc_row[u], kind = a.unc_kind[u];
    if (!ball_participates(a.unc_dk[u], a.n64A[i])) continue;
    if ((a.pend[i] & ((1 << kind) - 1)) != 0) continue;  // once per row
    const int root = a.root_of_row[i];
    if (root < 0 || !a.active[root]) continue;            // no group, or one left to the rescan
    const int g = a.gid[root];
    if (a.rsize[g] == 0) continue;
    const int s = atomicAdd(a.afill + g, 1);
    if (s >= a.ga[g]) { a.gfail[g] = 1; continue; }
    const int p = a.goff[g] + s;
    a.pos_of_row[i] = p;
    a.gmap[p] = i;
    a.ggrp[p] = g;
  }
}

// Every pending row of a group must have been placed; work items of the searched groups.
__global__ void ball_items_count_kernel(BallArgs a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = node_count(a);
  if (g >= nn) return;
  const int G = a.gid[nn];
  int c = 0;
  if (g < G && a.rsize[g] > 0) {
    if (a.afill[g] != a.ga[g]) a.gfail[g] = 1;
    if (!a.gfail[g]) c = (a.ga[g] + 127) / 128;
  }
  a.icnt[g] = c;
  if (c > 0 && a.stats) {
    atomicAdd(a.stats + GCR_STAT_BALL_GROUPS, 1ull);
    atomicAdd(a.stats + GCR_STAT_BALL_ROWS, (unsigned long long)a.rsize[g]);
  }
  if (g < G) {  // neutral per-group maxima for the centring pass
    a.gsc[g].nmin = 1e300;
    a.gsc[g].nmax = 0.0;
    a.gsc[g].emax = 0.0;
    a.gsc[g].amax = 0.0;
  }
}

__global__ void ball_items_kernel(BallArgs a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int G = a.gid[node_count(a)];
  if (g >= G || a.icnt[g] == 0) return;
  const int o = a.ioff[g];
  for (int b = 0; b < a.icnt[g]; ++b)
    a.items[o + b] = make_int4(a.goff[g] + 128 * b, min(128, a.ga[g] - 128 * b), a.boff[g], a.blim[g]);
}

__device__ __forceinline__ unsigned long long dbits_b(double v) { return (unsigned long long)__double_as_longlong(v); }

// One warp per position of a searched group: y = fl(x - c_g), its rounded operand copy, the
// squared norm (float-float, combined in FP64), the bias ||y||^2 / 2 of the pool scores, the
// rounding-error norms (rounded up as in the row statistics) and the group maxima.
template <Elt E>
__device__ __forceinline__ void ball_center_one(const BallArgs& a, int p, int lane);

template <Elt E>
__global__ void __launch_bounds__(256) ball_center_kernel(BallArgs a) {
  const int lane = threadIdx.x & 31;
  const int G = a.gid[node_count(a)];
  if (G == 0) return;
  const int P = min(a.goff[G], a.cap_rows);
  for (int p = blockIdx.x * 8 + (threadIdx.x >> 5); p < P; p += gridDim.x * 8) ball_center_one<E>(a, p, lane);
}

template <Elt E>
__device__ __forceinline__ void ball_center_one(const BallArgs& a, int p, int lane) {
  const int g = a.ggrp[p];
  if (g < 0 || a.gfail[g] || a.rsize[g] == 0) return;
  const int j = a.gmap[p];
  const bool on_b = a.two && p >= a.goff[g] + a.ga[g];
  const float4* xj = reinterpret_cast<const float4*>(on_b ? a.XB + (size_t)j * a.d : a.XA + (size_t)j * a.d);
  const float4* xc = reinterpret_cast<const float4*>(node_row(a, a.groot[g]));
  float4* y = reinterpret_cast<float4*>(a.Y + (size_t)p * a.d);
  FF acc;
  float ee = 0.f, aa = 0.f;
  for (int v = lane; v < (a.d >> 2); v += 32) {
    const float4 q = xj[v], c = xc[v];
    const float4 t = make_float4(q.x - c.x, q.y - c.y, q.z - c.z, q.w - c.w);
    y[v] = t;
    acc.add_sq(t.x); acc.add_sq(t.y); acc.add_sq(t.z); acc.add_sq(t.w);
    float f0, f1, f2, f3;
    if constexpr (E == Elt::BF16) {
      __nv_bfloat16 b0 = __float2bfloat16_rn(t.x), b1 = __float2bfloat16_rn(t.y);
      __nv_bfloat16 b2 = __float2bfloat16_rn(t.z), b3 = __float2bfloat16_rn(t.w);
      __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(a.Yr) + (size_t)p * a.d + 4 * v);
      o[0] = __halves2bfloat162(b0, b1);
      o[1] = __halves2bfloat162(b2, b3);
      f0 = __bfloat162float(b0); f1 = __bfloat162float(b1);
      f2 = __bfloat162float(b2); f3 = __bfloat162float(b3);
    } else {
      f0 = round_tf32(t.x); f1 = round_tf32(t.y);
      f2 = round_tf32(t.z); f3 = round_tf32(t.w);
      reinterpret_cast<float4*>(static_cast<float*>(a.Yr) + (size_t)p * a.d)[v] = make_float4(f0, f1, f2, f3);
    }
    const float e0 = f0 - t.x, e1 = f1 - t.y, e2 = f2 - t.z, e3 = f3 - t.w;
    ee = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, ee))));
    aa = fmaf(f0, f0, fmaf(f1, f1, fmaf(f2, f2, fmaf(f3, f3, aa))));
  }
  const double ss = warp_sum_d(acc.value());
  const float en = sqrtf(warp_sum(ee) * 1.002f) * 1.0001f;
  const float an = sqrtf(warp_sum(aa) * 1.002f) * 1.0001f;
  if (lane != 0) return;
  a.n64y[p] = ss;
  a.hy[p] = (float)(0.5 * ss);
  a.enrm_y[p] = en;
  a.anrm_y[p] = an;
  if (a.gcam) a.gcam[p] = a.cam[j];
  RowScalars* sc = a.gsc + g;
  atomicMin(reinterpret_cast<unsigned long long*>(&sc->nmin), dbits_b(ss));
  atomicMax(reinterpret_cast<unsigned long long*>(&sc->nmax), dbits_b(ss));
  atomicMax(reinterpret_cast<unsigned long long*>(&sc->emax), dbits_b((double)en));
  atomicMax(reinterpret_cast<unsigned long long*>(&sc->amax), dbits_b((double)an));
}

// ---------------------------------------------------------------- cluster order of the rows
// Propagation gathers each row's neighbour rows; it hits in L2 when the rows in flight share
// their neighbours, i.e. when rows are walked cluster by cluster. Clusters here are the
// components of the graph linking each row to its first kOrderLinks neighbours at a similar local
// scale (the k-th distances within kScaleRatio of each other, so that a row whose neighbours lie
// in other clusters does not chain clusters together), among contracted rows (k-th distance at
// most a quarter of the squared norm). A component of two or more rows that fit in half of L2
// is walked as one run (key = its root); the rows of a larger one (which no order keeps in L2,
// and whose single run would only serialise unrelated gathers) and the rows left alone keep
// their previous key. Rows are counting-sorted by key.
constexpr int kOrderLinks = 4;

__global__ void order_init_kernel(int* parent, int* cnt, int* fill, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    parent[i] = i;
    cnt[i] = 0;
    fill[i] = 0;
  }
}

__global__ void order_link_kernel(const int32_t* nbr, const float* d2, const double* n64, int n, int k, int* parent,
                                  int* err) {
  const int links = min(k, kOrderLinks);
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < (long)n * links; t += (long)gridDim.x * blockDim.x) {
    const int i = (int)(t / links), s = (int)(t % links);
    const float di = d2[(size_t)i * k + k - 1];
    if (!((double)di <= 0.25 * n64[i])) continue;  // not contracted: the row keeps its key
    const int j = nbr[(size_t)i * k + s];
    if (j < 0) continue;
    const float dj = d2[(size_t)j * k + k - 1];
    if (di <= kScaleRatio * dj && dj <= kScaleRatio * di && !uf_unite(parent, i, j)) atomicOr(err, 1);
  }
}

__global__ void order_count_kernel(int* parent, int n, int* root, int* cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int r = uf_find(parent, i);
    root[i] = r;
    atomicAdd(cnt + r, 1);
  }
}

// key[i] = root[i] for rows of components of 2 to max_run rows, else prev_key[i]; counted.
__global__ void order_key2_kernel(const int* root, const int* csize, const int* prev_key, int n, int max_run,
                                  int* key, int* cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int r = root[i];
    const int kk = (csize[r] > 1 && csize[r] <= max_run) ? r : prev_key[i];
    key[i] = kk;
    atomicAdd(cnt + kk, 1);
  }
}

__global__ void order_scatter_kernel2(const int* root, const int* off, int n, int* fill, int* order) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int r = root[i];
    order[off[r] + atomicAdd(fill + r, 1)] = i;
  }
}

}  // namespace

cudaError_t launch_cluster_order(const int32_t* nbr, const float* d2, const double* n64, int n, int d, int k,
                                 const int* prev_key, int* parent, int* root, int* csize, int* cnt, int* off,
                                 int* fill, int* order, int* err, cudaStream_t st) {
  if (n < 1 || k < 1) return cudaSuccess;
  int dev = 0, l2 = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  if (e != cudaSuccess) return e;
  const int max_run = (int)std::max<long>(1, (long)l2 / 2 / ((long)d * 4));
  const int nb = std::min((n + 255) / 256, 152 * 8);
  order_init_kernel<<<nb, 256, 0, st>>>(parent, csize, fill, n);
  e = cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), st);
  if (e != cudaSuccess) return e;
  order_link_kernel<<<nb, 256, 0, st>>>(nbr, d2, n64, n, k, parent, err);
  order_count_kernel<<<nb, 256, 0, st>>>(parent, n, root, csize);
  order_key2_kernel<<<nb, 256, 0, st>>>(root, csize, prev_key, n, max_run, root, cnt);
  e = launch_scan(cnt, off, n, st);
  if (e != cudaSuccess) return e;
  order_scatter_kernel2<<<nb, 256, 0, st>>>(root, off, n, fill, order);
  return cudaGetLastError();
}

size_t carve_ball(Carve& c, int n, int d, int kinds, int kp, Elt elt, int cap_rows, BallArgs* out, int nb) {
  // n: nodes (the A rows, plus the nb gallery rows of a search against a gallery)
  BallArgs t{};
  t.parent = c.take<int>(n);
  t.pend = c.take<int>(n);
  t.acnt = c.take<int>(n);
  t.rad = c.take<float>(n);
  t.rdense = c.take<int>(n);
  t.seen = c.take<int>(n);
  t.active = c.take<int>(n + 1);
  t.gid = c.take<int>(n + 1);
  t.pos_of_row = c.take<int>(n);
  t.root_of_row = c.take<int>(n);
  t.groot = c.take<int>(n);
  t.ga = c.take<int>(n);
  t.gkind = c.take<int>(n);
  t.gthr = c.take<float>(n);
  t.gthr_fill = c.take<float>(n);
  t.gsize = c.take<int>(n + 1);
  t.rsize = c.take<int>(n + 1);
  t.goff = c.take<int>(n + 1);
  t.boff = c.take<int>(n);
  t.blim = c.take<int>(n);
  t.gscale = c.take<float>(nb > 0 ? nb : 1);
  t.npart = c.take<int>(1);
  t.ndense = c.take<int>(1);
  t.gfill = c.take<int>(n);
  t.afill = c.take<int>(n);
  t.bfill = c.take<int>(n);
  t.gfail = c.take<int>(n);
  t.icnt = c.take<int>(n + 1);
  t.ioff = c.take<int>(n + 1);
  t.gsc = c.take<RowScalars>(n);
  t.max_items = cap_rows / 128 + n + 1;  // sum over groups of ceil(pending rows / 128)
  t.items = c.take<int4>((size_t)t.max_items);
  t.ball_j = c.take<int>(cap_rows);
  t.gmap = c.take<int>(cap_rows);
  t.ggrp = c.take<int>(cap_rows);
  t.n64y = c.take<double>(cap_rows);
  t.hy = c.take<float>(cap_rows);
  t.enrm_y = c.take<float>(cap_rows);
  t.anrm_y = c.take<float>(cap_rows);
  t.gcam = kinds == 2 ? c.take<int>(cap_rows) : nullptr;
  t.Y = c.take<float>((size_t)cap_rows * d);
  t.Yr = c.take<char>((size_t)cap_rows * d * elt_bytes(elt));
  t.gpool_v = c.take<float>((size_t)kinds * cap_rows * kp);
  t.gpool_i = c.take<int>((size_t)kinds * cap_rows * kp);
  t.cap_rows = cap_rows;
  if (out) {
    BallArgs& a = *out;
#define GCR_BALL_TAKE(f) a.f = t.f
    GCR_BALL_TAKE(parent); GCR_BALL_TAKE(pend); GCR_BALL_TAKE(acnt); GCR_BALL_TAKE(rad); GCR_BALL_TAKE(rdense); GCR_BALL_TAKE(seen); GCR_BALL_TAKE(active);
    GCR_BALL_TAKE(gid); GCR_BALL_TAKE(pos_of_row); GCR_BALL_TAKE(root_of_row); GCR_BALL_TAKE(groot);
    GCR_BALL_TAKE(ga); GCR_BALL_TAKE(gkind); GCR_BALL_TAKE(gthr); GCR_BALL_TAKE(gthr_fill); GCR_BALL_TAKE(gsize);
    GCR_BALL_TAKE(rsize); GCR_BALL_TAKE(goff); GCR_BALL_TAKE(boff); GCR_BALL_TAKE(blim); GCR_BALL_TAKE(gscale);
    GCR_BALL_TAKE(npart); GCR_BALL_TAKE(ndense); GCR_BALL_TAKE(gfill); GCR_BALL_TAKE(afill); GCR_BALL_TAKE(bfill);
    GCR_BALL_TAKE(gfail); GCR_BALL_TAKE(icnt); GCR_BALL_TAKE(ioff); GCR_BALL_TAKE(gsc); GCR_BALL_TAKE(max_items);
    GCR_BALL_TAKE(items); GCR_BALL_TAKE(ball_j); GCR_BALL_TAKE(gmap); GCR_BALL_TAKE(ggrp); GCR_BALL_TAKE(n64y);
    GCR_BALL_TAKE(hy); GCR_BALL_TAKE(enrm_y); GCR_BALL_TAKE(anrm_y); GCR_BALL_TAKE(gcam); GCR_BALL_TAKE(Y);
    GCR_BALL_TAKE(Yr); GCR_BALL_TAKE(gpool_v); GCR_BALL_TAKE(gpool_i); GCR_BALL_TAKE(cap_rows);
#undef GCR_BALL_TAKE
  }
  return c.off;
}

// Steps 1-5 (see the top of this file). The caller then runs the grouped GEMM and the
// refinement of its pools.
cudaError_t launch_ball_prepare(const BallArgs& a, cudaStream_t st) {
  const int nn = a.two ? a.na + a.nb : a.na;
  if (a.na < 1 || a.unc_cap < 1) return cudaSuccess;
  const int nb = (nn + 255) / 256;
  const int wb = std::min((a.unc_cap + 7) / 8, 152 * 8);   // grid-stride loops over the pending pairs
  ball_init_kernel<<<nb, 256, 0, st>>>(a);
  ball_mark_kernel<<<std::min((a.unc_cap + 255) / 256, 152 * 4), 256, 0, st>>>(a);
  if (a.two) ball_scale_kernel<<<wb, 256, 0, st>>>(a);
  ball_link_kernel<<<wb, 256, 0, st>>>(a);
  ball_root_kernel<<<wb, 256, 0, st>>>(a);
  ball_elig_kernel<<<std::min(nb, 152 * 8), 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan(a.active, a.gid, nn, st);  // group ids; gid[nn] = number of groups
  if (e != cudaSuccess) return e;
  ball_group_kernel<<<nb, 256, 0, st>>>(a);
  ball_centres_kernel<<<152 * 4, 256, 0, st>>>(a);
  // sweep pass 1: ball sizes (the centre rows: at most cent_rows groups, one per pending row)
  e = cudaMemsetAsync(a.gsize, 0, sizeof(int) * (nn + 1), st);
  if (e != cudaSuccess) return e;
  const int B_rows = a.two ? a.nb : a.na;
  const void* xrB = a.two ? a.xrB : a.xrA;
  e = launch_umma_band(xrB, B_rows, a.d, a.elt, nullptr, 0, a.cent, a.gid + nn, a.cent_rows, a.groot, a.gkind,
                       a.gthr, 0, a.gsize, nullptr, a.ball_j, st);
  if (e != cudaSuccess) return e;
  ball_route_kernel<<<nb, 256, 0, st>>>(a);
  e = launch_scan(a.rsize, a.goff, nn, st);
  if (e != cudaSuccess) return e;
  ball_cut_kernel<<<nb, 256, 0, st>>>(a);
  // sweep pass 2: members of the searched balls at their offsets
  e = launch_umma_band(xrB, B_rows, a.d, a.elt, nullptr, 0, a.cent, a.gid + nn, a.cent_rows, a.groot, a.gkind,
                       a.gthr_fill, 0, a.gfill, nullptr, a.ball_j, st, a.boff, a.blim);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.ggrp, 0xff, sizeof(int) * a.cap_rows, st);
  if (e != cudaSuccess) return e;
  ball_place_kernel<<<std::min((a.cap_rows + 255) / 256, 152 * 8), 256, 0, st>>>(a);
  if (a.two) ball_place_rows_kernel<<<std::min((a.unc_cap + 255) / 256, 152 * 4), 256, 0, st>>>(a);
  ball_items_count_kernel<<<nb, 256, 0, st>>>(a);
  e = launch_scan(a.icnt, a.ioff, nn, st);
  if (e != cudaSuccess) return e;
  ball_items_kernel<<<nb, 256, 0, st>>>(a);
  const unsigned cb = (unsigned)std::min((a.cap_rows + 7) / 8, 152 * 4);
  if (a.elt == Elt::TF32) ball_center_kernel<Elt::TF32><<<cb, 256, 0, st>>>(a);
  else ball_center_kernel<Elt::BF16><<<cb, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace gcr
