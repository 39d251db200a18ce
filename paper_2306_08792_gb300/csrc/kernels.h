// Internal declarations shared by the GCR translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace gcr {

struct Carve;     // bump allocator over a caller's workspace (common.cuh)
struct BallArgs;  // ball search of the pairs a pool could not certify (below)

// Element type of the tensor-core GEMM operands: BF16 copies of the rows, or FP32 rows
// rounded to TF32 (10 explicit mantissa bits, low 13 bits zero).
enum class Elt : int { BF16 = 0, TF32 = 1 };
inline size_t elt_bytes(Elt e) { return e == Elt::TF32 ? 4 : 2; }

// Per-call scalars reduced over the rows of X (device memory).
struct RowScalars {
  double nmin, nmax;   // min / max of ||x_j||^2
  double bmax;         // max ||x_j||: formed by the reader from nmax
  double emax;         // max ||round(x_j) - x_j||   (tensor-core paths)
  double amax;         // max ||round(x_j)||         (tensor-core paths)
};

// ---- prep.cu
cudaError_t launch_normalize(const float* X_in, float* X_out, int64_t n, int d, cudaStream_t st);
// xr (may be NULL): the rounded operand copy (BF16, or TF32 held as FP32) written alongside
// the rounding-error norms enrm and the norms of the rounded rows anrm.
cudaError_t launch_row_stats(const float* X, int n, int d, double* n64, float* n32,
                             void* xr, Elt elt, float* enrm, float* anrm, RowScalars* sc,
                             cudaStream_t st);
cudaError_t launch_split3(const float* X, int n, int d, int gallery_order, __nv_bfloat16* out, cudaStream_t st);

// ---- sgemm.cu
size_t sgemm_pool_smem();
// Pools of S = A . B^T rows: [split][kind][na][kp]; self_excl skips j == i (A == B).
cudaError_t launch_sgemm_pool(const float* A, int na, const float* B, int nb, int d, const int* cam, int kp,
                              bool cross, int self_excl, int splits, float* pool_v, int* pool_i, cudaStream_t st);
// Threshold rescan: rows X[band_row[u]] against all rows of Bm (n of them).
cudaError_t launch_sgemm_band(const float* X, const float* Bm, int n, int d, const int* cam, int self_excl,
                              const int* count, int cap, const int* band_row, const int* band_kind,
                              const float* band_thr, int bcap, int* band_cnt, float* band_v, int* band_i,
                              cudaStream_t st);
cudaError_t launch_sgemm_dist(const float* Xq, int nq, const float* Xg, int ng, int d,
                              const float* nrm_q, const float* nrm_g, float* D, cudaStream_t st);

// ---- umma.cu (tcgen05 path; operands BF16 or TF32)
// Pools of S = A . B^T rows: [split][kind][na][kp], kp = 32, 64 or 128.
// seed (may be NULL): per row of A an admission floor; every split keeps only scores above it,
// so a merged pool may hold fewer than kp entries, and every score left out of it is <= the
// floor or <= its last entry.
// tau_x ([2][kinds][na] floats) and pair_cnt ([2 ceil(na / 256)][kinds][4] ints), both may be
// NULL: for 32-entry pools without a seed and with splits = 1, where one 128-row A block per SM
// would not fit in half the L2, two CTAs sweep the two column halves of each row block; pool_v
// and pool_i then need room for two [kind][na][kp] regions, and the pools end in the first.
cudaError_t launch_umma_pool(const void* Ab, int na, const void* Bb, int nb, int d, Elt elt,
                             const int* cam, bool cross, int self_excl, int kp, int splits, float* pool_v,
                             int* pool_i, cudaStream_t st, const float* seed = nullptr, float* tau_x = nullptr,
                             int* pair_cnt = nullptr);
// Pools of row blocks of the gathered matrix Y (rows x d, rounded operand) against column ranges
// of Y: work item w = {first row, rows <= 128, first column, columns} of *n_items (<= max_items);
// pool entry (s - col_bias[j], j), j a position in Y; column j == row skipped when self_excl;
// gcam: camera per position (cross-camera pools). Pools [kind][rows][kp].
cudaError_t launch_umma_gpool(const void* Y, int rows, int d, Elt elt, const int* gcam, bool cross, int self_excl,
                              int kp, const int4* items, const int* n_items, int max_items, const float* col_bias,
                              float* pool_v, int* pool_i, cudaStream_t st);
// Threshold rescan: gathered rows Ab (cap rows, *count valid) against the n rows of Xb. Row u
// counts every column whose score reaches band_thr[u] in band_cnt[u] and writes the first
// band_lim[u] (NULL: bcap) of them at band_off[u] (NULL: u * bcap); band_v may be NULL.
cudaError_t launch_umma_band(const void* Xb, int n, int d, Elt elt, const int* cam, int self_excl,
                             const void* Ab, const int* count, int cap, const int* band_row,
                             const int* band_kind, const float* band_thr, int bcap, int* band_cnt, float* band_v,
                             int* band_i, cudaStream_t st, const int* band_off = nullptr,
                             const int* band_lim = nullptr);
cudaError_t launch_umma_dist(const __nv_bfloat16* Qb, int nq, const __nv_bfloat16* Gb, int ng, int d,
                             const float* nrm_q, const float* nrm_g, float* D, cudaStream_t st);
// G_s = Z_s Z_s^T + lambda n_s I for every camera s (d x d, FP32, [ncam][d][d]), Z the
// transposed normalised frames (d rows, cols columns), split hi + lo in BF16 (hi.hi + hi.lo +
// lo.hi); camera s owns the column blocks of 64 [kstart[s], kstart[s] + knum[s]).
cudaError_t launch_umma_gram(const __nv_bfloat16* zt_hi, const __nv_bfloat16* zt_lo, int d, int64_t cols,
                             const int64_t* kstart, const int64_t* knum, const int64_t* nf, int ncam, float lambda,
                             float* G, cudaStream_t st);
// Q = P G_s for each 128-row block of P (camera s = rowcam[block]; blocks with s < 0 are
// skipped), TF32 operands split hi + lo (hi.hi + hi.lo + lo.hi); G stacked as ncam*d rows of d
// (symmetric, so its rows are the K-major B operand).
cudaError_t launch_umma_mul(const float* p_hi, const float* p_lo, int rows, const float* g_hi, const float* g_lo,
                            int ncam, int d, const int* rowcam, float* Q, cudaStream_t st);
int umma_read_and_clear_timeouts();
cudaError_t launch_wait_probe(unsigned long long limit_ns, cudaStream_t st);  // bounded waits that ran out since the last call (-1: error)

// ---- refine.cu
struct RefineArgs {
  const float* X;           // rows whose neighbours are refined (n x d)
  const float* XB;          // rows the candidates index (equal to X for the offline graph)
  int n, d, k, kinds;
  int precision;            // GCR_PREC_FP32 / GCR_PREC_BF16 / GCR_PREC_TF32
  const double* n64;        // ||x_i||^2 of the rows of X
  const double* n64B;       // ||x_j||^2 of the rows of XB
  const float* enrm;        // rounding statistics of the rows of X (tensor-core paths)
  const float* anrm;
  const RowScalars* sc;     // maxima over the rows of XB
  const float* pool_v;      // [kinds][n][kp]
  const int* pool_i;
  int kp;
  int32_t* nbr[2];
  float* d2[2];
  int* unc_count;           // uncertified (row, kind) pairs for the band rescan
  int* unc_row;
  int* unc_kind;
  float* unc_thr;
  float* unc_dk;            // per queued pair (may be NULL): an upper bound on its exact k-th
                            // squared distance, negated when the pair's band is predicted to
                            // overflow the band capacity
  float* dk_all;            // [kinds][n] (may be NULL): the same bound for every (row, graph)
  int skip_saturated;       // 1: pairs whose pool is saturated with near-ties are not queued
  int* bq_count;            // ball refinement: pairs handed on to the band rescan, in the
  int* bq_row;              // pending queue's order (bq_flag per pending pair, bq_pos its
  int* bq_kind;             // scan: cap + 1 entries)
  float* bq_thr;
  int* bq_flag;
  int* bq_pos;
  unsigned long long* stats;
  // band rescan results
  const int* band_cnt;
  const float* band_v;
  const int* band_i;
  int bcap;
  int band_rows;            // capacity of the band buffers (rows beyond it are not rescanned)
  const int* order;         // processing order of the rows (NULL: 0..n-1); results do not depend on it
  const float* floor;       // per row (kinds == 1), or NULL: the admission floor the pools were
                            // searched with (a bound on every score left out of a short pool)
};
cudaError_t launch_refine_pool(const RefineArgs& a, cudaStream_t st);
// Refinement of the grouped pools of the ball search (ball.cu): each queued pair of a searched
// group is certified in the centred coordinates of its ball (result written, counted in
// GCR_STAT_BALL) or handed on to the band queue bq_* with its original threshold.
cudaError_t launch_refine_ball(const RefineArgs& a, const BallArgs& b, cudaStream_t st);
// Split-pool seeds of the serving search (see refine.cu): for each of the b query rows of xq,
// an admission floor for its search against the gallery G, from the FP32 scores of the distinct
// rows of the row's previous pool (prev_kp entries of pool_i), of their hop lists (hop_k per
// gallery row, when hop != NULL) and of the sample rows floor(i * ng / sample), i < sample:
// below the approximate score of every candidate among the best min(valid, kp), so that the
// search keeps at least that many. -inf when fewer than k distinct candidates.
constexpr int kSeedCandidates = 4096;  // prev_kp * (1 + hop_k) + sample must not exceed this
struct SeedArgs {
  const float* xq;          // b x d query rows of this search (FP32)
  const float* G;           // ng x d gallery rows of this search (FP32)
  int b, ng, d, precision;
  const double* n64q;       // ||x_q||^2
  const float* enrm;        // rounding statistics of the query rows (tensor-core modes)
  const float* anrm;
  const RowScalars* gsc;    // maxima over the gallery rows
  const int* pool_i;        // b x prev_kp (NULL when prev_kp == 0)
  int prev_kp;
  const int32_t* hop;       // ng x hop_k, or NULL
  int hop_k;
  int sample;               // evenly spaced gallery rows added to the candidates (0..ng)
  int k;                    // neighbours this search must certify
  int kp;                   // pool size of this search
  float* seed;              // b
};
cudaError_t launch_serve_seed(const SeedArgs& a, cudaStream_t st);
cudaError_t launch_refine_band(const RefineArgs& a, cudaStream_t st);
// Cluster-local row order from the pools (first k candidates): order[0..n) is a permutation.
cudaError_t launch_row_order(const int* pool_i, int n, int kp, int k, int* key, int* cnt, int* off, int* fill,
                             int* order, cudaStream_t st);
// Copies rows[u] of src (row_bytes each, a multiple of 16) to row u of out, u < min(*count, max_rows).
cudaError_t launch_gather_rows(const void* src, size_t row_bytes, const int* count, const int* rows,
                               int max_rows, void* out, cudaStream_t st);

// ---- ball.cu: certified search of the pending (row, graph) pairs inside balls shared by
// groups of them, in coordinates centred on each ball (see ball.cu)
struct BallArgs {
  // inputs. The A rows are the rows searched; the B rows the candidates: the A rows themselves
  // (two = 0, an offline graph) or a gallery (two = 1, a search against it)
  int two;
  const float* XA;          // na x d FP32 rows
  const float* XB;          // nb x d (two = 1)
  const void* xrA;          // rounded operand copies (BF16, or TF32 held as FP32)
  const void* xrB;
  Elt elt;
  int na, nb, d, k, kp, kinds, precision;
  const double* n64A;       // ||x||^2 per row
  const double* n64B;
  const float* enrmA;       // rounding statistics per row
  const float* anrmA;
  const float* enrmB;
  const float* anrmB;
  const RowScalars* scB;    // maxima over the B rows
  const int* cam;           // camera per row (cross-camera graph, two = 0), or NULL
  const int* pool_i;        // [kinds][na][kp] pools of the first search (indices of B rows)
  const float* pool_v;      //                 and their approximate scores
  const int* unc_count;     // pending pairs (device count), capacity unc_cap
  const int* unc_row;
  const int* unc_kind;
  const float* unc_dk;      // per pair: an upper bound on its exact k-th squared distance
                            // (negated: the pair's band is predicted to overflow)
  const float* dk_all;      // [kinds][na]: that bound for every (row, graph) (two = 0)
  int unc_cap;
  void* cent;               // scratch: cent_rows rounded rows (the centres' operand copies)
  int cent_rows;            // >= the number of groups (at most one per pending row)
  int* err;                 // set when a union-find link gives up
  unsigned long long* stats;  // GCR_STAT_BALL_PAIRS / _GROUPS / _ROWS counters (may be NULL)
  // workspace (carve_ball)
  int *parent, *pend, *acnt, *active, *gid, *pos_of_row, *root_of_row;
  int* rdense;              // per root: a pair of the group was predicted to overflow the band
  int* seen;                // per root: the root of some pending pair
  float* rad;
  float* gscale;            // per B row (two = 1): its local scale
  int* npart;               // pending pairs taking part, and those predicted dense
  int* ndense;
  int *groot, *ga, *gkind, *gsize, *rsize, *goff, *boff, *blim, *gfill, *afill, *bfill, *gfail, *icnt, *ioff;
  float *gthr, *gthr_fill;
  RowScalars* gsc;          // per group: maxima over its positions
  int4* items;
  int max_items;
  int* ball_j;              // listed members, cap_rows
  int* gmap;                // position -> row (of A, or of B for the ball members when two = 1)
  int* ggrp;                // position -> group (-1: unused)
  double* n64y;             // per position: ||y||^2
  float* hy;                //               ||y||^2 / 2 (the pool scores' bias)
  float* enrm_y;
  float* anrm_y;
  int* gcam;                // camera per position (cross-camera graph)
  float* Y;                 // centred rows, cap_rows x d
  void* Yr;                 // their rounded operand copy
  float* gpool_v;           // [kinds][cap_rows][kp] pools of the grouped search
  int* gpool_i;
  int cap_rows;
};
// Whether a pending pair enters the ball search: its band is predicted to overflow (dk < 0), or
// its k-th distance bound is at most a quarter of its squared norm (dk <= n_i / 4). A ball holds
// the pair's k-th neighbour, so R^2 >= dk and a pair above that bound could only be in a ball
// too wide to be searched; such a pair goes to the threshold rescan, even when its row is
// placed in a ball for another graph (the ball was sized without it).
__device__ __forceinline__ bool ball_participates(float dk, double n_i) {
  return dk < 0.f || (double)dk <= 0.25 * n_i;
}
// n: nodes (the A rows, plus the nb B rows when two = 1); cap_rows: gathered positions.
size_t carve_ball(Carve& c, int n, int d, int kinds, int kp, Elt elt, int cap_rows, BallArgs* out, int nb = 0);
cudaError_t launch_ball_prepare(const BallArgs& a, cudaStream_t st);
// Cluster order of the rows for the propagation: order[0..n) lists the rows component by
// component of the graph of each row's first few neighbours at a similar scale (nbr, d2: n x k
// lists by ascending distance; n64 the rows' squared norms), for components of contracted rows
// that fit in half of L2 (d floats a row); the other rows are ordered by prev_key. Scratch: parent, root, csize, fill (n),
// cnt, off (n + 1).
cudaError_t launch_cluster_order(const int32_t* nbr, const float* d2, const double* n64, int n, int d, int k,
                                 const int* prev_key, int* parent, int* root, int* csize, int* cnt, int* off,
                                 int* fill, int* order, int* err, cudaStream_t st);

// ---- graph.cu
struct GraphArgs {
  int n, k, kinds, symmetric;
  float gamma, alpha;
  const int32_t* nbr[2];
  const float* d2[2];
  float* w[2];              // [n*k] weights
  float* deg_r[2];
  float* deg_c[2];
  int* cnt[2];              // [n+1] in-degree counts -> transposed row pointers
  int* fill[2];             // [n]
  int* t_src[2];            // [n*k]
  float* t_w[2];
  int* op_rowptr;           // [n+1]
  int* op_len;              // [n]
  int* op_col;              // [op_cap] (also the unsorted transpose while building)
  float* op_val;            // [op_cap]
  int* raw_col;             // [op_cap] scratch
  float* raw_val;           // [op_cap] scratch
  int* op_cnt;              // [n] scratch
  int* scan_tmp;            // [n+1] scratch
  double* inv;              // [2*kinds][n] scratch: inverse square roots of the degrees
  int* long_list;           // [n] scratch: transposed rows of a hub's length
  int* long_count;          // [2] scratch
  int* scan_tmp2;           // [n+1], [n]: the second graph's scan temporary and hub list (its
  int* long_list2;          //   transpose is built on a second stream)
};
cudaError_t launch_build_operator(const GraphArgs& g, cudaStream_t st);
cudaError_t launch_scan(const int* in, int* out, int n, cudaStream_t st);

// ---- propagate.cu
// order (may be NULL): the rows in processing order; results do not depend on it.
cudaError_t launch_propagate(const int* rowptr, const int* len, const int* col, const float* val,
                             const float* X_in, float* X_out, int n, int d, const int* order, cudaStream_t st);

// ---- gcrv.cu
struct GcrvWs {
  int rows_cap;
  float* inv;
  int* cam_cnt;
  int64_t* cam_nf;
  int* blk0;
  int* perm;
  int* pos;
  int64_t* fstart;
  int64_t* foff;
  int* row_cam;
  int* flist;
  float* mu;
  float* mu_cam;
  float* G;
  __nv_bfloat16* zt_hi;     // [d][cols] transposed normalised frames, camera blocks padded to 64
  __nv_bfloat16* zt_lo;
  int64_t zt_cols;
  float* g_hi;              // [ncam][d][d] G in TF32 hi + lo
  float* g_lo;
  float* p_hi;              // [rows_cap][d] the CG direction in TF32 hi + lo
  float* p_lo;
  int64_t* kstart;          // [kMaxCams] first 64-column block of each camera
  int64_t* knum;            // [kMaxCams] 64-column blocks of each camera
  float* X;
  float* R;
  float* P;
  float* Q;
  double* rr;
};
int gcrv_iterations(float lambda);
// Eq. 10 alone: W[c] = mean of tracklet c's L2-normalised frames (inv: F floats of scratch).
cudaError_t launch_gcrv_means(const float* frames, int64_t F, int d, const int64_t* off, int C, float* inv, float* W,
                              cudaStream_t st);
cudaError_t launch_gcrv(const float* frames, int64_t F, int d, const int64_t* off, const int32_t* cam, int C,
                        int ncam, float lambda, float* W, const GcrvWs& w, cudaStream_t st);

// ---- serve.cu
cudaError_t launch_merge_splits(const float* pv, const int* pi, int S, int kinds, int na, int kp, float* ov, int* oi,
                                cudaStream_t st);
cudaError_t launch_query_step(const float* xq, int b, int d, const float* G, const float* deg, const int32_t* nbr,
                              const float* d2, int k, float gamma, int symmetric, float* out, cudaStream_t st);
cudaError_t launch_layer_degree(const float* dr, const float* dc, int n, int symmetric, float* out, cudaStream_t st);

// ---- dsfp.cu
// Local propagation of Algorithm 1 for every row of the normalised X (n x d, d % 4 == 0)
// over its neighbour lists nbr (n x k, entries < 0 absent; k <= kDsfpMaxK); out: n x d.
cudaError_t launch_dsfp(const float* X, int n, int d, const int32_t* nbr, int k, float gamma, int T, float* out,
                        cudaStream_t st);

// ---- eval.cu
cudaError_t launch_eval(const int32_t* idx, int nq, long K, const int32_t* q_label, const int32_t* q_cam,
                        const int32_t* g_label, const int32_t* g_cam, int ng, int protocol, double* ap_out,
                        int32_t* first_out, cudaStream_t st);

// ---- sort.cu
cudaError_t launch_rank_rows(const float* D, int nq, int ng, int K, int32_t* idx_out,
                             float* dist_out, cudaStream_t st);

}  // namespace gcr
