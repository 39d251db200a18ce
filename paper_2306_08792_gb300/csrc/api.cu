// Host entry points of the C ABI declared in include/gcr.h.
//
// Every entry point validates its arguments on the host, carves its scratch from the
// caller's workspace and enqueues kernels on the caller's stream. Nothing here allocates
// device memory or synchronises (except gcr_sync).
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

using namespace gcr;

namespace {

// ---------------------------------------------------------------------------------------------
// Stage profiler: CUDA events recorded on the launching stream around each stage, summed on read.
struct StageProfiler {
  bool on = false;
  static constexpr int kMaxRec = 4096;
  cudaEvent_t ev[kMaxRec][2];
  int stage[kMaxRec];
  int launches[kMaxRec];
  int used = 0;
  bool created = false;
};
StageProfiler g_prof;

struct StageScope {
  int slot = -1;
  cudaStream_t st;
  StageScope(int stage, cudaStream_t s, int nlaunch = 1) : st(s) {
    if (!g_prof.on || g_prof.used >= StageProfiler::kMaxRec) return;
    slot = g_prof.used++;
    g_prof.stage[slot] = stage;
    g_prof.launches[slot] = nlaunch;
    cudaEventRecord(g_prof.ev[slot][0], st);
  }
  ~StageScope() {
    if (slot >= 0) cudaEventRecord(g_prof.ev[slot][1], st);
  }
};

constexpr int kBandCap = 512;        // band entries kept per rescanned (row, graph)

struct Resolved {
  int kp;
  int kinds;
};

// The tensor-core modes (BF16, TF32) search on rounded operand copies; FP32 runs on the CUDA cores.
bool tensor_mode(const gcr_params* p) { return p->precision != GCR_PREC_FP32; }
Elt elt_of(const gcr_params* p) { return p->precision == GCR_PREC_TF32 ? Elt::TF32 : Elt::BF16; }
size_t elt_size(const gcr_params* p) { return elt_bytes(elt_of(p)); }

int check_precision(const gcr_params* p, int32_t d) {
  if (p->precision != GCR_PREC_FP32 && p->precision != GCR_PREC_BF16 && p->precision != GCR_PREC_TF32)
    return GCR_E_INVALID;
  // BF16 rows (and the compensated BF16 distance operands of both modes) need 16-byte rows
  if (tensor_mode(p) && d % 8 != 0) return GCR_E_UNSUPPORTED;
  return GCR_OK;
}

// Default candidate pool: room for a margin of max(12, k/2) candidates past the k-th, which
// the certification needs when the k-th neighbour sits in a dense region; BF16 at least 64.
int default_pool(const gcr_params* p) {
  const int want = p->k + std::max(12, p->k / 2);
  int kp = want <= 32 ? 32 : (want <= 64 ? 64 : 128);
  if (p->precision == GCR_PREC_BF16) kp = std::max(kp, 64);
  return kp;
}

// Feature matrices are read and written as 16-byte vectors: their base must be 16-byte aligned
// (rows then are too, d being a multiple of 4).
bool misaligned(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) != 0; }

int check_params(const gcr_params* p, int64_t n, int32_t d, Resolved* r) {
  if (!p || n < 1 || n > (1 << 24)) return GCR_E_INVALID;
  if (d < 4 || d > kMaxD) return GCR_E_INVALID;
  if (d % 4 != 0) return GCR_E_UNSUPPORTED;
  const int pc = check_precision(p, d);
  if (pc != GCR_OK) return pc;
  if (!(p->gamma > 0.f) || !std::isfinite(p->gamma)) return GCR_E_INVALID;
  if (p->symmetric != 0 && p->symmetric != 1) return GCR_E_INVALID;
  if (p->cross_camera != 0 && p->cross_camera != 1) return GCR_E_INVALID;
  if (p->cross_camera && !(p->alpha >= 0.f && p->alpha <= 1.f)) return GCR_E_INVALID;
  int kp = p->pool ? p->pool : default_pool(p);
  if (kp != 32 && kp != 64 && kp != 128) return GCR_E_INVALID;
  if (p->k < 0 || p->k >= kp) return GCR_E_INVALID;
  // the BF16 rounding bound is too loose for a 32-entry pool to certify most rows
  if (p->precision == GCR_PREC_BF16 && kp == 32) return GCR_E_UNSUPPORTED;
  r->kp = kp;
  r->kinds = p->cross_camera ? 2 : 1;
  return GCR_OK;
}

size_t op_capacity(int64_t n, const gcr_params* p, int kinds) {
  const int64_t per = 1 + (int64_t)p->k * kinds * (p->symmetric ? 2 : 1);
  return (size_t)(n * per);
}

struct BuildWs {
  double* n64;
  float* n32;
  RowScalars* sc;
  void* xr;            // rounded operand copy (tensor-core modes)
  float* enrm;
  float* anrm;
  float* pool_v;
  int* pool_i;
  float* tau_x;        // paired GEMM splits: per-row thresholds of the two column halves
  int* pair_cnt;
  int* unc_count;
  int* unc_row;
  int* unc_kind;
  float* unc_thr;
  float* unc_dk;
  float* dk_all;       // k-th distance bound of every (row, graph)
  int* bq_count;       // pairs the ball search hands on to the band rescan
  int* bq_row;
  int* bq_kind;
  float* bq_thr;
  int* bq_flag;
  int* bq_pos;
  int* band_cnt;
  float* band_v;
  int* band_i;
  void* band_a;        // gathered rounded rows of the band rescan (also the ball centres)
  BallArgs ball;       // workspace of the ball search (tensor-core modes)
  float* w;
  int* cnt;
  int* fill;
  int* t_src;
  float* t_w;
  int* raw_col;
  float* raw_val;
  int* op_cnt;
  int* scan_tmp;
  double* inv;
  int* long_list;
  int* long_count;
  int* scan_tmp2;      // the second graph's transpose scratch (built on a second stream)
  int* long_list2;
  unsigned long long* stats;
  int* err;
  int* okey;
  int* ocnt;
  int* ooff;
  int* ofill;
  int* order;
  int band_rows;
};

size_t carve_build(Carve& c, int64_t n, int32_t d, const gcr_params* p, const Resolved& r, BuildWs* w) {
  const size_t nn = (size_t)n;
  const int kinds = r.kinds;
  const bool bf = tensor_mode(p);
  const size_t es = elt_size(p);
  // every (row, graph) pair fits in the band buffers, so no uncertified pair goes unrescanned
  const int band_rows = (int)((int64_t)kinds * n);
  const size_t cap = op_capacity(n, p, kinds);
  BuildWs t;
  t.n64 = c.take<double>(nn);
  t.n32 = c.take<float>(nn);
  t.sc = c.take<RowScalars>(1);
  t.xr = bf ? c.take<char>(nn * d * es) : nullptr;
  t.enrm = bf ? c.take<float>(nn) : nullptr;
  t.anrm = bf ? c.take<float>(nn) : nullptr;
  // 32-entry pools on the tensor-core path: room for the two column halves of paired GEMM splits
  const bool pairable = bf && r.kp == 32;
  t.pool_v = c.take<float>((size_t)(pairable ? 2 : 1) * kinds * nn * r.kp);
  t.pool_i = c.take<int>((size_t)(pairable ? 2 : 1) * kinds * nn * r.kp);
  t.tau_x = pairable ? c.take<float>((size_t)2 * kinds * nn) : nullptr;
  t.pair_cnt = pairable ? c.take<int>((size_t)kinds * 4 * 2 * ((nn + 255) / 256)) : nullptr;
  t.unc_count = c.take<int>(4);
  t.unc_row = c.take<int>((size_t)kinds * nn);
  t.unc_kind = c.take<int>((size_t)kinds * nn);
  t.unc_thr = c.take<float>((size_t)kinds * nn);
  t.unc_dk = c.take<float>((size_t)kinds * nn);
  t.dk_all = c.take<float>((size_t)kinds * nn);
  t.bq_count = c.take<int>(4);
  t.bq_row = c.take<int>((size_t)kinds * nn);
  t.bq_kind = c.take<int>((size_t)kinds * nn);
  t.bq_thr = c.take<float>((size_t)kinds * nn);
  t.bq_flag = c.take<int>((size_t)kinds * nn);
  t.bq_pos = c.take<int>((size_t)kinds * nn + 1);
  t.band_cnt = c.take<int>(band_rows);
  t.band_v = c.take<float>((size_t)band_rows * kBandCap);
  t.band_i = c.take<int>((size_t)band_rows * kBandCap);
  t.band_a = bf ? c.take<char>((size_t)band_rows * d * es) : nullptr;
  std::memset(&t.ball, 0, sizeof(t.ball));
  // ball search: up to 2n gathered members (centred rows and their operand copies); balls of
  // one contracted cluster overlap, so their total can exceed n
  if (bf && p->k > 0) carve_ball(c, (int)n, d, kinds, r.kp, elt_of(p), (int)std::min<int64_t>(2 * n, INT32_MAX / 2), &t.ball);
  t.w = c.take<float>((size_t)kinds * nn * p->k);
  t.cnt = c.take<int>((size_t)kinds * (nn + 1));
  t.fill = c.take<int>((size_t)kinds * nn);
  t.t_src = c.take<int>((size_t)kinds * nn * p->k);
  t.t_w = c.take<float>((size_t)kinds * nn * p->k);
  t.raw_col = c.take<int>(cap);
  t.raw_val = c.take<float>(cap);
  t.op_cnt = c.take<int>(nn);
  t.scan_tmp = c.take<int>(nn + 1);
  t.inv = c.take<double>((size_t)2 * kinds * nn);
  t.long_list = c.take<int>(nn);
  t.long_count = c.take<int>(4);
  t.scan_tmp2 = c.take<int>(nn + 1);
  t.long_list2 = c.take<int>(nn);
  t.stats = c.take<unsigned long long>(GCR_STATS_LEN);
  t.err = c.take<int>(4);
  t.okey = c.take<int>(nn);
  t.ocnt = c.take<int>(nn + 1);
  t.ooff = c.take<int>(nn + 1);
  t.ofill = c.take<int>(nn);
  t.order = c.take<int>(nn);
  t.band_rows = band_rows;
  if (w) *w = t;
  return c.off;
}

// The certified kNN search of Eq. 4 / Eq. 8 (S1-S3): writes g->nbr / nbr_d2 (and the
// cross-camera lists), g->row_order when given, and the search counters.
int knn_impl(const float* X, int64_t n64_, int32_t d, const int32_t* cam, const gcr_params* p, const Resolved& r,
             gcr_graph* g, const BuildWs& w, cudaStream_t st) {
  const int n = (int)n64_;
  const int kinds = r.kinds;
  const bool bf = tensor_mode(p);
  const Elt elt = elt_of(p);
  unsigned long long* stats = g->stats ? reinterpret_cast<unsigned long long*>(g->stats) : w.stats;
  if (!g->stats) GCR_CUDA_TRY(cudaMemsetAsync(w.stats, 0, sizeof(unsigned long long) * GCR_STATS_LEN, st));

  {
    StageScope sc_(GCR_STAGE_PREP, st, 2);
    GCR_CUDA_TRY(launch_row_stats(X, n, d, w.n64, w.n32, bf ? w.xr : nullptr, elt, w.enrm, w.anrm, w.sc, st));
  }
  GCR_CUDA_TRY(cudaMemsetAsync(w.unc_count, 0, sizeof(int) * 4, st));
  GCR_CUDA_TRY(cudaMemsetAsync(w.band_cnt, 0, sizeof(int) * w.band_rows, st));
  GCR_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int) * 4, st));
  const int* camp = p->cross_camera ? cam : nullptr;

  if (p->k > 0) {
    StageScope sc_(GCR_STAGE_SIM_GEMM, st);
    if (bf) {
      GCR_CUDA_TRY(launch_umma_pool(w.xr, n, w.xr, n, d, elt, camp, p->cross_camera != 0, 1, r.kp, 1, w.pool_v,
                                    w.pool_i, st, nullptr, w.tau_x, w.pair_cnt));
    } else {
      GCR_CUDA_TRY(launch_sgemm_pool(X, n, X, n, d, camp, r.kp, p->cross_camera != 0, 1, 1, w.pool_v, w.pool_i, st));
    }
  }

  RefineArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  ra.X = X; ra.XB = X; ra.n = n; ra.d = d; ra.k = p->k; ra.kinds = kinds; ra.precision = p->precision;
  ra.n64 = w.n64; ra.n64B = w.n64; ra.enrm = w.enrm; ra.anrm = w.anrm; ra.sc = w.sc;
  ra.pool_v = w.pool_v; ra.pool_i = w.pool_i; ra.kp = r.kp;
  ra.nbr[0] = g->nbr; ra.d2[0] = g->nbr_d2;
  ra.nbr[1] = kinds == 2 ? g->nbr_cr : g->nbr;
  ra.d2[1] = kinds == 2 ? g->nbr_cr_d2 : g->nbr_d2;
  ra.unc_count = w.unc_count; ra.unc_row = w.unc_row; ra.unc_kind = w.unc_kind; ra.unc_thr = w.unc_thr;
  ra.stats = stats;
  ra.band_cnt = w.band_cnt; ra.band_v = w.band_v; ra.band_i = w.band_i; ra.bcap = kBandCap;
  ra.band_rows = w.band_rows;
  // cluster-local processing order for the refinement and the propagation of this graph; it
  // is always written when the caller provides row_order (the identity when k = 0)
  int* order = g->row_order ? g->row_order : w.order;
  if (p->k == 0 && g->row_order)
    GCR_CUDA_TRY(launch_row_order(w.pool_i, n, r.kp, 0, w.okey, w.ocnt, w.ooff, w.ofill, order, st));
  if (p->k > 0) {
    ra.unc_dk = w.unc_dk;
    ra.dk_all = bf ? w.dk_all : nullptr;
    // the tensor-core modes queue every uncertified pair for the ball search; FP32 keeps the
    // prediction of saturated pools (no ball search on the CUDA-core path)
    ra.skip_saturated = bf ? 0 : 1;
    {
      StageScope sc_(GCR_STAGE_REFINE, st, 5);
      GCR_CUDA_TRY(launch_row_order(w.pool_i, n, r.kp, p->k, w.okey, w.ocnt, w.ooff, w.ofill, order, st));
      ra.order = order;
      GCR_CUDA_TRY(launch_refine_pool(ra, st));
    }
    // the queue the band rescan takes: the ball search's leftovers, or the refinement's queue
    RefineArgs rb = ra;
    if (bf) {
      StageScope sc_(GCR_STAGE_BALL, st, 20);
      BallArgs b = w.ball;
      b.two = 0; b.XA = b.XB = X; b.xrA = b.xrB = w.xr; b.elt = elt; b.na = n; b.nb = n; b.d = d; b.k = p->k;
      b.kp = r.kp; b.kinds = kinds; b.precision = p->precision; b.n64A = b.n64B = w.n64;
      b.enrmA = b.enrmB = w.enrm; b.anrmA = b.anrmB = w.anrm; b.scB = w.sc; b.cam = camp;
      b.pool_i = w.pool_i; b.pool_v = w.pool_v; b.unc_count = w.unc_count; b.unc_row = w.unc_row;
      b.unc_kind = w.unc_kind; b.unc_dk = w.unc_dk; b.dk_all = w.dk_all; b.unc_cap = kinds * n;
      b.cent = w.band_a; b.cent_rows = w.band_rows; b.err = w.err; b.stats = stats;
      GCR_CUDA_TRY(launch_ball_prepare(b, st));
      GCR_CUDA_TRY(launch_umma_gpool(b.Yr, b.cap_rows, d, elt, b.gcam, kinds == 2, 1, r.kp, b.items, b.ioff + n,
                                     b.max_items, b.hy, b.gpool_v, b.gpool_i, st));
      ra.bq_count = w.bq_count; ra.bq_row = w.bq_row; ra.bq_kind = w.bq_kind; ra.bq_thr = w.bq_thr;
      ra.bq_flag = w.bq_flag; ra.bq_pos = w.bq_pos;
      GCR_CUDA_TRY(launch_refine_ball(ra, b, st));
      rb.unc_count = w.bq_count; rb.unc_row = w.bq_row; rb.unc_kind = w.bq_kind; rb.unc_thr = w.bq_thr;
    }
    // threshold rescan of the pairs still uncertified
    StageScope sc_(GCR_STAGE_BAND, st, bf ? 3 : 2);
    if (bf) {
      GCR_CUDA_TRY(launch_gather_rows(w.xr, (size_t)d * elt_bytes(elt), rb.unc_count, rb.unc_row, w.band_rows,
                                      w.band_a, st));
      GCR_CUDA_TRY(launch_umma_band(w.xr, n, d, elt, camp, 1, w.band_a, rb.unc_count, w.band_rows, rb.unc_row,
                                    rb.unc_kind, rb.unc_thr, kBandCap, w.band_cnt, w.band_v, w.band_i, st));
    } else {
      GCR_CUDA_TRY(launch_sgemm_band(X, X, n, d, camp, 1, rb.unc_count, w.band_rows, rb.unc_row, rb.unc_kind,
                                     rb.unc_thr, kBandCap, w.band_cnt, w.band_v, w.band_i, st));
    }
    GCR_CUDA_TRY(launch_refine_band(rb, st));
  }
  return GCR_OK;
}

// The propagation's row order (clusters of the final lists, so that its gathers hit in L2) is
// computed on a side stream while the operator is built: one stream and two events per device,
// the mutex keeping a call's fork, order and join together.
struct OrderStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kMaxOrderDevices = 64;
OrderStream g_order_side[kMaxOrderDevices];
std::mutex g_order_mu;

int build_graph_impl(const float* X, int64_t n64_, int32_t d, const int32_t* cam, const gcr_params* p,
                     const Resolved& r, gcr_graph* g, const BuildWs& w, cudaStream_t st) {
  const int n = (int)n64_;
  const int kinds = r.kinds;
  const int s = knn_impl(X, n64_, d, cam, p, r, g, w, st);
  if (s != GCR_OK) return s;

  GraphArgs ga;
  std::memset(&ga, 0, sizeof(ga));
  ga.n = n; ga.k = p->k; ga.kinds = kinds; ga.symmetric = p->symmetric;
  ga.gamma = p->gamma; ga.alpha = p->alpha;
  ga.nbr[0] = g->nbr; ga.d2[0] = g->nbr_d2;
  ga.nbr[1] = g->nbr_cr; ga.d2[1] = g->nbr_cr_d2;
  ga.deg_r[0] = g->deg_r; ga.deg_c[0] = g->deg_c;
  ga.deg_r[1] = g->deg_r_cr; ga.deg_c[1] = g->deg_c_cr;
  for (int q = 0; q < kinds; ++q) {
    ga.w[q] = w.w + (size_t)q * n * p->k;
    ga.cnt[q] = w.cnt + (size_t)q * (n + 1);
    ga.fill[q] = w.fill + (size_t)q * n;
    ga.t_src[q] = w.t_src + (size_t)q * n * p->k;
    ga.t_w[q] = w.t_w + (size_t)q * n * p->k;
  }
  ga.op_rowptr = g->op_rowptr; ga.op_len = g->op_len; ga.op_col = g->op_col; ga.op_val = g->op_val;
  ga.raw_col = w.raw_col; ga.raw_val = w.raw_val; ga.op_cnt = w.op_cnt; ga.scan_tmp = w.scan_tmp;
  ga.inv = w.inv; ga.long_list = w.long_list; ga.long_count = w.long_count;
  ga.scan_tmp2 = w.scan_tmp2; ga.long_list2 = w.long_list2;
  const bool want_order = g->row_order != nullptr && p->k > 0;
  std::unique_lock<std::mutex> olock;
  OrderStream* os = nullptr;
  if (want_order) {
    int dev = 0;
    GCR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxOrderDevices) return GCR_E_UNSUPPORTED;
    olock = std::unique_lock<std::mutex>(g_order_mu);
    os = &g_order_side[dev];
    if (!os->s) {
      GCR_CUDA_TRY(cudaStreamCreateWithFlags(&os->s, cudaStreamNonBlocking));
      GCR_CUDA_TRY(cudaEventCreateWithFlags(&os->fork, cudaEventDisableTiming));
      GCR_CUDA_TRY(cudaEventCreateWithFlags(&os->join, cudaEventDisableTiming));
    }
  }
  {
    StageScope sc_(GCR_STAGE_GRAPH, st, 7 * kinds + 3 + (want_order ? 5 : 0));
    if (want_order) {
      GCR_CUDA_TRY(cudaEventRecord(os->fork, st));
      GCR_CUDA_TRY(cudaStreamWaitEvent(os->s, os->fork, 0));
      // scratch: the search's pending-pair queues, free once the search is done; w.okey holds
      // the pools' keys (the order of the rows outside any cluster)
      GCR_CUDA_TRY(launch_cluster_order(g->nbr, g->nbr_d2, w.n64, n, d, p->k, w.okey, w.unc_row, w.unc_kind,
                                        w.bq_row, w.ocnt, w.ooff, w.ofill, g->row_order, w.err, os->s));
      GCR_CUDA_TRY(cudaEventRecord(os->join, os->s));
    }
    GCR_CUDA_TRY(launch_build_operator(ga, st));
    if (want_order) GCR_CUDA_TRY(cudaStreamWaitEvent(st, os->join, 0));
  }
  return GCR_OK;
}

int check_graph(const gcr_graph* g, int kinds, int k) {
  if (!g || !g->deg_r || !g->deg_c || !g->op_rowptr || !g->op_len || !g->op_col || !g->op_val)
    return GCR_E_INVALID;
  if (k > 0 && (!g->nbr || !g->nbr_d2)) return GCR_E_INVALID;
  if (kinds == 2 && (!g->deg_r_cr || !g->deg_c_cr)) return GCR_E_INVALID;
  if (kinds == 2 && k > 0 && (!g->nbr_cr || !g->nbr_cr_d2)) return GCR_E_INVALID;
  return GCR_OK;
}

struct RerankWs {
  float* D;
  double* n64q;
  double* n64g;
  float* nq;
  float* ng;
  RowScalars* sc;
  __nv_bfloat16* qb;
  __nv_bfloat16* gb;
  float* dummy;
  int* err;
};

// Top-K re-ranking through the certified pool search: used when 1 <= topk_out <= 127 and
// topk_out < ng (any gallery size); the full ranking uses the distance GEMM + sort.
bool rerank_uses_pool(const gcr_params* p, int64_t ng) {
  return p->topk_out >= 1 && p->topk_out <= 127 && p->topk_out < ng;
}

size_t carve_rerank(Carve& c, int64_t nq, int64_t ng, int32_t d, bool bf, RerankWs* w) {
  RerankWs t;
  t.D = c.take<float>((size_t)nq * ng);
  t.n64q = c.take<double>(nq);
  t.n64g = c.take<double>(ng);
  t.nq = c.take<float>(nq);
  t.ng = c.take<float>(ng);
  t.sc = c.take<RowScalars>(2);
  t.qb = bf ? c.take<__nv_bfloat16>((size_t)nq * 3 * d) : nullptr;
  t.gb = bf ? c.take<__nv_bfloat16>((size_t)ng * 3 * d) : nullptr;
  t.dummy = c.take<float>(2 * (size_t)std::max(nq, ng));
  t.err = c.take<int>(4);
  if (w) *w = t;
  return c.off;
}

// Optional delivery of the ranking to host memory in query chunks: after each chunk is
// sorted, its rows are copied on a second stream while the next chunks are computed.
struct HostDelivery {
  int32_t* idx_host;
  float* dist_host;
  int chunk_rows;         // queries per chunk (a multiple of the GEMM's 128-row tile)
  cudaStream_t copy;      // copy stream
  cudaEvent_t* ready;     // one event per chunk
  int n_events;
};

int rerank_impl(const float* Xq, int64_t nq, const float* Xg, int64_t ng, int32_t d, const gcr_params* p,
                int32_t* idx_out, float* dist_out, const RerankWs& w, cudaStream_t st,
                const HostDelivery* hd = nullptr) {
  // the distance GEMM of both tensor-core modes runs on compensated BF16 operands
  const bool bf = tensor_mode(p);
  const int K = p->topk_out > 0 ? (int)std::min<int64_t>(p->topk_out, ng) : (int)ng;
  const size_t mx = (size_t)std::max(nq, ng);
  {
    StageScope sc_(GCR_STAGE_PREP, st, bf ? 6 : 4);
    GCR_CUDA_TRY(launch_row_stats(Xq, (int)nq, d, w.n64q, w.nq, nullptr, Elt::BF16, w.dummy, w.dummy + mx, w.sc, st));
    GCR_CUDA_TRY(
        launch_row_stats(Xg, (int)ng, d, w.n64g, w.ng, nullptr, Elt::BF16, w.dummy, w.dummy + mx, w.sc + 1, st));
    if (bf) {
      GCR_CUDA_TRY(launch_split3(Xq, (int)nq, d, 0, w.qb, st));
      GCR_CUDA_TRY(launch_split3(Xg, (int)ng, d, 1, w.gb, st));
    }
  }
  if (bf) GCR_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int) * 4, st));
  const int64_t chunk = hd ? hd->chunk_rows : nq;
  for (int64_t q0 = 0, c = 0; q0 < nq; q0 += chunk, ++c) {
    const int nc = (int)std::min<int64_t>(chunk, nq - q0);
    {
      StageScope sc_(GCR_STAGE_DIST_GEMM, st);
      if (bf) {
        GCR_CUDA_TRY(launch_umma_dist(w.qb + (size_t)q0 * 3 * d, nc, w.gb, (int)ng, 3 * d, w.nq + q0, w.ng,
                                      w.D + (size_t)q0 * ng, st));
      } else {
        GCR_CUDA_TRY(launch_sgemm_dist(Xq + (size_t)q0 * d, nc, Xg, (int)ng, d, w.nq + q0, w.ng,
                                       w.D + (size_t)q0 * ng, st));
      }
    }
    {
      StageScope sc_(GCR_STAGE_SORT, st);
      GCR_CUDA_TRY(launch_rank_rows(w.D + (size_t)q0 * ng, nc, (int)ng, K, idx_out + (size_t)q0 * K,
                                    dist_out + (size_t)q0 * K, st));
    }
    if (hd) {
      if (c >= hd->n_events) return GCR_E_INVALID;
      const size_t off = (size_t)q0 * K, cnt = (size_t)nc * K;
      GCR_CUDA_TRY(cudaEventRecord(hd->ready[c], st));
      GCR_CUDA_TRY(cudaStreamWaitEvent(hd->copy, hd->ready[c], 0));
      GCR_CUDA_TRY(cudaMemcpyAsync(hd->idx_host + off, idx_out + off, cnt * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                   hd->copy));
      GCR_CUDA_TRY(cudaMemcpyAsync(hd->dist_host + off, dist_out + off, cnt * sizeof(float), cudaMemcpyDeviceToHost,
                                   hd->copy));
    }
  }
  return GCR_OK;
}

int check_rerank(int64_t nq, int64_t ng, int32_t d, const gcr_params* p) {
  if (!p || nq < 1 || ng < 1 || ng > (1 << 24) || nq > (1 << 24)) return GCR_E_INVALID;
  if (d < 4 || d > kMaxD) return GCR_E_INVALID;
  if (d % 4 != 0) return GCR_E_UNSUPPORTED;
  const int pc = check_precision(p, d);
  if (pc != GCR_OK) return pc;
  if (p->topk_out < 0) return GCR_E_INVALID;
  if (ng > 16384 && !(p->topk_out >= 1 && p->topk_out <= 127)) return GCR_E_UNSUPPORTED;
  return GCR_OK;
}

struct TopkRerankWs;
size_t carve_topk_rerank(Carve& c, int64_t nq, int64_t ng, int32_t d, const gcr_params* p, TopkRerankWs* w);
int topk_rerank_impl(const float* Xq, int64_t nq, const float* Xg, int64_t ng, int32_t d, const gcr_params* p,
                     int32_t* idx_out, float* dist_out, const TopkRerankWs& w, cudaStream_t st);

struct PipeWs {
  float* Xa;
  float* Xb;
  gcr_graph g;
  char* inner;
  size_t inner_bytes;
};

size_t carve_pipe(Carve& c, int64_t n, int64_t nq, int32_t d, const gcr_params* p, const Resolved& r, PipeWs* w) {
  const size_t nn = (size_t)n;
  const int kinds = r.kinds;
  PipeWs t;
  std::memset(&t, 0, sizeof(t));
  t.Xa = c.take<float>(nn * d);
  t.Xb = c.take<float>(nn * d);
  t.g.nbr = c.take<int32_t>(nn * p->k);
  t.g.nbr_d2 = c.take<float>(nn * p->k);
  t.g.nbr_cr = kinds == 2 ? c.take<int32_t>(nn * p->k) : nullptr;
  t.g.nbr_cr_d2 = kinds == 2 ? c.take<float>(nn * p->k) : nullptr;
  t.g.deg_r = c.take<float>(nn);
  t.g.deg_c = c.take<float>(nn);
  t.g.deg_r_cr = kinds == 2 ? c.take<float>(nn) : nullptr;
  t.g.deg_c_cr = kinds == 2 ? c.take<float>(nn) : nullptr;
  t.g.op_rowptr = c.take<int32_t>(nn + 1);
  t.g.op_len = c.take<int32_t>(nn);
  const size_t cap = op_capacity(n, p, kinds);
  t.g.op_col = c.take<int32_t>(cap);
  t.g.op_val = c.take<float>(cap);
  t.g.row_order = c.take<int32_t>(nn);
  t.g.stats = nullptr;
  // the build and re-rank scratch run one after the other: they share one region
  Carve cb(nullptr, 0);
  const size_t b = carve_build(cb, n, d, p, r, nullptr);
  Carve cr(nullptr, 0);
  const size_t rr = rerank_uses_pool(p, n - nq) ? carve_topk_rerank(cr, nq, n - nq, d, p, nullptr)
                                                : carve_rerank(cr, nq, n - nq, d, tensor_mode(p), nullptr);
  t.inner_bytes = std::max(b, rr);
  t.inner = c.take<char>(t.inner_bytes);
  if (w) *w = t;
  return c.off;
}


// ------------------------------------------------------------------------------------ serving
struct GalleryView {
  float* layers;   // (T+1) x ng x d
  float* deg;      // T x ng
  double* n64;     // (T+1) x ng
  float* n32;      // (T+1) x ng
  char* xr;        // (T+1) x ng x d rounded operand copies (tensor-core modes)
  float* enrm;     // (T+1) x ng
  float* anrm;     // (T+1) x ng
  RowScalars* sc;  // T+1
  int32_t* nbr;    // ng x k: the kNN lists of the last layer's graph (T >= 1, k >= 1); candidates
                   // for the seeds of the final search's split pools
};

int check_serve_params(const gcr_params* p, int64_t ng, int32_t d, Resolved* r) {
  int s = check_params(p, ng, d, r);
  if (s != GCR_OK) return s;
  if (p->cross_camera) return GCR_E_UNSUPPORTED;  // the resident gallery carries no camera graph
  if (p->T < 0 || p->T > 16) return GCR_E_INVALID;
  if (p->topk_out < 1 || p->topk_out > 127 || p->topk_out > ng) return GCR_E_INVALID;
  if (p->k > ng) return GCR_E_INVALID;
  return GCR_OK;
}

size_t carve_gallery(Carve& c, int64_t ng, int32_t d, const gcr_params* p, GalleryView* v) {
  const size_t L = (size_t)p->T + 1, n = (size_t)ng;
  const bool bf = tensor_mode(p);
  GalleryView t;
  t.layers = c.take<float>(L * n * d);
  t.deg = c.take<float>((size_t)(p->T > 0 ? p->T : 1) * n);
  t.n64 = c.take<double>(L * n);
  t.n32 = c.take<float>(L * n);
  t.xr = bf ? c.take<char>(L * n * d * elt_size(p)) : nullptr;
  t.enrm = bf ? c.take<float>(L * n) : nullptr;
  t.anrm = bf ? c.take<float>(L * n) : nullptr;
  t.sc = c.take<RowScalars>(L);
  t.nbr = c.take<int32_t>(n * std::max(p->k, 1));
  if (v) *v = t;
  return c.off;
}

struct GalleryBuildWs {
  gcr_graph g;
  char* inner;
  size_t inner_bytes;
};

size_t carve_gallery_build(Carve& c, int64_t ng, int32_t d, const gcr_params* p, const Resolved& r,
                           GalleryBuildWs* w) {
  const size_t n = (size_t)ng;
  GalleryBuildWs t;
  std::memset(&t, 0, sizeof(t));
  t.g.nbr = c.take<int32_t>(n * p->k);
  t.g.nbr_d2 = c.take<float>(n * p->k);
  t.g.deg_r = c.take<float>(n);
  t.g.deg_c = c.take<float>(n);
  t.g.op_rowptr = c.take<int32_t>(n + 1);
  t.g.op_len = c.take<int32_t>(n);
  const size_t cap = op_capacity(ng, p, 1);
  t.g.op_col = c.take<int32_t>(cap);
  t.g.op_val = c.take<float>(cap);
  t.g.row_order = c.take<int32_t>(n);
  Carve cb(nullptr, 0);
  t.inner_bytes = carve_build(cb, ng, d, p, r, nullptr);
  t.inner = c.take<char>(t.inner_bytes);
  if (w) *w = t;
  return c.off;
}

struct ServeWs {
  float* xq[2];
  double* n64;
  float* n32;
  void* qr;            // rounded query rows (tensor-core modes)
  float* enrm;
  float* anrm;
  RowScalars* sc;
  float* part_v;
  int* part_i;
  float* pool_v;
  int* pool_i;
  int* unc_count;
  int* unc_row;
  int* unc_kind;
  float* unc_thr;
  float* unc_dk;
  int* bq_count;       // pairs the ball search hands on to the band rescan
  int* bq_row;
  int* bq_kind;
  float* bq_thr;
  int* bq_flag;
  int* bq_pos;
  int* err;
  int* band_cnt;
  float* band_v;
  int* band_i;
  void* band_a;
  int32_t* nbr;
  float* d2;
  unsigned long long* stats;
  float* seed;         // per query: the admission floor of this search's split pools
};

constexpr int kServeMaxSplits = 152;

// Column splits the pool launchers actually use for `want` splits of `ntiles` tiles.
int split_count(int want, int ntiles) {
  want = std::max(1, std::min(want, ntiles));
  const int tps = (ntiles + want - 1) / want;
  return (ntiles + tps - 1) / tps;
}

int serve_kp_final(const gcr_params* p) {
  const int K = p->topk_out;
  if (p->precision != GCR_PREC_BF16 && K < 32) return 32;
  return K < 64 ? 64 : 128;
}

size_t carve_serve(Carve& c, int64_t b, int32_t d, const gcr_params* p, const Resolved& r, ServeWs* w) {
  const size_t nb = (size_t)b;
  const bool bf = tensor_mode(p);
  const size_t es = elt_size(p);
  const int kpmax = std::max(r.kp, serve_kp_final(p));
  ServeWs t;
  t.xq[0] = c.take<float>(nb * d);
  t.xq[1] = c.take<float>(nb * d);
  t.n64 = c.take<double>(nb);
  t.n32 = c.take<float>(nb);
  t.qr = bf ? c.take<char>(nb * d * es) : nullptr;
  t.enrm = bf ? c.take<float>(nb) : nullptr;
  t.anrm = bf ? c.take<float>(nb) : nullptr;
  t.sc = c.take<RowScalars>(1);
  t.part_v = c.take<float>((size_t)kServeMaxSplits * nb * kpmax);
  t.part_i = c.take<int>((size_t)kServeMaxSplits * nb * kpmax);
  t.pool_v = c.take<float>(nb * kpmax);
  t.pool_i = c.take<int>(nb * kpmax);
  t.unc_count = c.take<int>(4);
  t.unc_row = c.take<int>(nb);
  t.unc_kind = c.take<int>(nb);
  t.unc_thr = c.take<float>(nb);
  t.unc_dk = c.take<float>(nb);
  t.bq_count = c.take<int>(4);
  t.bq_row = c.take<int>(nb);
  t.bq_kind = c.take<int>(nb);
  t.bq_thr = c.take<float>(nb);
  t.bq_flag = c.take<int>(nb);
  t.bq_pos = c.take<int>(nb + 1);
  t.err = c.take<int>(4);
  t.band_cnt = c.take<int>(nb);
  t.band_v = c.take<float>(nb * kBandCap);
  t.band_i = c.take<int>(nb * kBandCap);
  t.band_a = bf ? c.take<char>(nb * d * es) : nullptr;
  t.nbr = c.take<int32_t>(nb * std::max(p->k, 1));
  t.d2 = c.take<float>(nb * std::max(p->k, 1));
  t.stats = c.take<unsigned long long>(GCR_STATS_LEN);
  t.seed = c.take<float>(nb);
  if (w) *w = t;
  return c.off;
}

// The gallery side of a certified top-k search: FP32 rows, their rounded operand copy
// (tensor-core modes), squared norms and maxima.
struct GallerySide {
  const float* G;
  const void* Gr;
  const double* n64;
  const RowScalars* sc;
  const float* enrm;  // rounding statistics of the rows (tensor-core modes)
  const float* anrm;
};

GallerySide gallery_layer(const GalleryView& g, int layer, int ng, int d, size_t es) {
  return GallerySide{g.layers + (size_t)layer * ng * d, g.xr ? g.xr + (size_t)layer * ng * d * es : nullptr,
                     g.n64 + (size_t)layer * ng, g.sc + layer,
                     g.enrm ? g.enrm + (size_t)layer * ng : nullptr, g.anrm ? g.anrm + (size_t)layer * ng : nullptr};
}

// Where the seeds of a search's split pools come from: the previous search's merged pool
// (prev_kp per query, still in the workspace) and optionally the gallery lists hop (hop_k per row).
// Both searches run on the same query rows (at different layers).
struct SeedSource {
  int prev_kp = 0;          // 0: no seed
  const int32_t* hop = nullptr;
  int hop_k = 0;
  int sample = 0;           // evenly spaced gallery rows added to the candidates
};

// Certified k nearest gallery rows for the b query rows xq: pool, merge, refine, band.
// ball (may be NULL; tensor-core modes): workspace of the ball search of the rows the pools
// cannot certify (without it, pools saturated with near-ties keep the 2 delta bound).
int serve_knn(const float* xq, int b, int d, const gcr_params* p, int k, int kp, const GallerySide& gs, int ng,
              const ServeWs& w, unsigned long long* stats, int32_t* nbr, float* d2, cudaStream_t st,
              const SeedSource& seed_src = SeedSource(), const BallArgs* ball = nullptr) {
  const bool bf = tensor_mode(p);
  const Elt elt = elt_of(p);
  const float* G = gs.G;
  const int rblocks = (b + 127) / 128;
  const int splits = std::max(1, std::min(kServeMaxSplits, (152 + rblocks - 1) / rblocks));
  {
    StageScope sc_(GCR_STAGE_PREP, st, bf ? 2 : 2);
    GCR_CUDA_TRY(launch_row_stats(xq, b, d, w.n64, w.n32, bf ? w.qr : nullptr, elt, w.enrm, w.anrm, w.sc, st));
  }
  GCR_CUDA_TRY(cudaMemsetAsync(w.unc_count, 0, sizeof(int) * 4, st));
  GCR_CUDA_TRY(cudaMemsetAsync(w.band_cnt, 0, sizeof(int) * b, st));
  int used_splits;
  // the split pools' admission floors (tensor-core modes), from the previous search's merged
  // pool, when given its rows' gallery lists, and a sample of the gallery
  const bool seeded = bf && (seed_src.prev_kp > 0 || seed_src.sample > 0) &&
                      (long)seed_src.prev_kp * (1 + seed_src.hop_k) + seed_src.sample <= kSeedCandidates;
  if (seeded) {
    SeedArgs sa;
    sa.xq = xq; sa.G = G; sa.b = b; sa.ng = ng; sa.d = d; sa.precision = p->precision;
    sa.n64q = w.n64; sa.enrm = w.enrm; sa.anrm = w.anrm; sa.gsc = gs.sc;
    sa.pool_i = seed_src.prev_kp > 0 ? w.pool_i : nullptr; sa.prev_kp = seed_src.prev_kp; sa.hop = seed_src.hop; sa.hop_k = seed_src.hop ? seed_src.hop_k : 0;
    sa.sample = seed_src.sample; sa.k = k; sa.kp = kp; sa.seed = w.seed;
    StageScope sc_(GCR_STAGE_PREP, st);
    GCR_CUDA_TRY(launch_serve_seed(sa, st));
  }
  {
    StageScope sc_(GCR_STAGE_SIM_GEMM, st, 2);
    if (bf) {
      const int ntiles = (ng + 255) / 256;
      used_splits = split_count(splits, ntiles);
      GCR_CUDA_TRY(launch_umma_pool(w.qr, b, gs.Gr, ng, d, elt, nullptr, false, 0, kp, used_splits, w.part_v,
                                    w.part_i, st, seeded ? w.seed : nullptr));
    } else {
      const int ntiles = (ng + 127) / 128;
      used_splits = split_count(splits, ntiles);
      GCR_CUDA_TRY(launch_sgemm_pool(xq, b, G, ng, d, nullptr, kp, false, 0, used_splits, w.part_v, w.part_i, st));
    }
    GCR_CUDA_TRY(launch_merge_splits(w.part_v, w.part_i, used_splits, 1, b, kp, w.pool_v, w.pool_i, st));
  }
  RefineArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  ra.X = xq; ra.XB = G; ra.n = b; ra.d = d; ra.k = k; ra.kinds = 1; ra.precision = p->precision;
  ra.n64 = w.n64; ra.n64B = gs.n64;
  ra.enrm = w.enrm; ra.anrm = w.anrm; ra.sc = gs.sc;
  ra.pool_v = w.pool_v; ra.pool_i = w.pool_i; ra.kp = kp;
  ra.nbr[0] = ra.nbr[1] = nbr;
  ra.d2[0] = ra.d2[1] = d2;
  ra.unc_count = w.unc_count; ra.unc_row = w.unc_row; ra.unc_kind = w.unc_kind; ra.unc_thr = w.unc_thr;
  ra.stats = stats;
  ra.band_cnt = w.band_cnt; ra.band_v = w.band_v; ra.band_i = w.band_i; ra.bcap = kBandCap; ra.band_rows = b;
  ra.floor = seeded ? w.seed : nullptr;
  const bool use_ball = bf && ball != nullptr && !seeded;
  ra.skip_saturated = use_ball ? 0 : 1;
  ra.unc_dk = w.unc_dk;
  {
    StageScope sc_(GCR_STAGE_REFINE, st);
    GCR_CUDA_TRY(launch_refine_pool(ra, st));
  }
  RefineArgs rb = ra;
  if (use_ball) {
    StageScope sc_(GCR_STAGE_BALL, st, 20);
    BallArgs bl = *ball;
    bl.two = 1; bl.XA = xq; bl.XB = G; bl.xrA = w.qr; bl.xrB = gs.Gr; bl.elt = elt; bl.na = b; bl.nb = ng;
    bl.d = d; bl.k = k; bl.kp = kp; bl.kinds = 1; bl.precision = p->precision; bl.n64A = w.n64; bl.n64B = gs.n64;
    bl.enrmA = w.enrm; bl.anrmA = w.anrm; bl.enrmB = gs.enrm; bl.anrmB = gs.anrm; bl.scB = gs.sc; bl.cam = nullptr;
    bl.pool_i = w.pool_i; bl.pool_v = w.pool_v; bl.unc_count = w.unc_count; bl.unc_row = w.unc_row;
    bl.unc_kind = w.unc_kind; bl.unc_dk = w.unc_dk; bl.dk_all = nullptr; bl.unc_cap = b; bl.cent = w.band_a;
    bl.cent_rows = b; bl.err = w.err; bl.stats = stats;
    GCR_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int) * 4, st));
    GCR_CUDA_TRY(launch_ball_prepare(bl, st));
    GCR_CUDA_TRY(launch_umma_gpool(bl.Yr, bl.cap_rows, d, elt, nullptr, false, 0, kp, bl.items, bl.ioff + b + ng,
                                   bl.max_items, bl.hy, bl.gpool_v, bl.gpool_i, st));
    ra.bq_count = w.bq_count; ra.bq_row = w.bq_row; ra.bq_kind = w.bq_kind; ra.bq_thr = w.bq_thr;
    ra.bq_flag = w.bq_flag; ra.bq_pos = w.bq_pos;
    GCR_CUDA_TRY(launch_refine_ball(ra, bl, st));
    rb.unc_count = w.bq_count; rb.unc_row = w.bq_row; rb.unc_kind = w.bq_kind; rb.unc_thr = w.bq_thr;
  }
  {
    StageScope sc_(GCR_STAGE_BAND, st, bf ? 3 : 2);
    if (bf) {
      GCR_CUDA_TRY(launch_gather_rows(w.qr, (size_t)d * elt_bytes(elt), rb.unc_count, rb.unc_row, b, w.band_a, st));
      GCR_CUDA_TRY(launch_umma_band(gs.Gr, ng, d, elt, nullptr, 0, w.band_a, rb.unc_count, b, rb.unc_row,
                                    rb.unc_kind, rb.unc_thr, kBandCap, w.band_cnt, w.band_v, w.band_i, st));
    } else {
      GCR_CUDA_TRY(launch_sgemm_band(xq, G, ng, d, nullptr, 0, rb.unc_count, b, rb.unc_row, rb.unc_kind, rb.unc_thr,
                                     kBandCap, w.band_cnt, w.band_v, w.band_i, st));
    }
    GCR_CUDA_TRY(launch_refine_band(rb, st));
  }
  return GCR_OK;
}

struct TopkRerankWs {
  ServeWs sw;
  double* n64g;
  float* n32g;
  void* gr;            // rounded gallery rows (tensor-core modes)
  float* genrm;
  float* ganrm;
  RowScalars* scg;
  BallArgs ball;       // ball search of the queries the pools cannot certify (tensor-core modes)
};

size_t carve_topk_rerank(Carve& c, int64_t nq, int64_t ng, int32_t d, const gcr_params* p, TopkRerankWs* w) {
  const bool bf = tensor_mode(p);
  Resolved r;
  r.kp = serve_kp_final(p);
  r.kinds = 1;
  TopkRerankWs t;
  carve_serve(c, nq, d, p, r, &t.sw);
  t.n64g = c.take<double>(ng);
  t.n32g = c.take<float>(ng);
  t.gr = bf ? c.take<char>((size_t)ng * d * elt_size(p)) : nullptr;
  t.genrm = c.take<float>(ng);
  t.ganrm = c.take<float>(ng);
  t.scg = c.take<RowScalars>(1);
  std::memset(&t.ball, 0, sizeof(t.ball));
  // gathered positions: each group's queries and its ball of gallery rows (balls may overlap)
  if (bf) carve_ball(c, (int)(nq + ng), d, 1, r.kp, elt_of(p), (int)std::min<int64_t>(nq + 2 * ng, INT32_MAX / 2),
                     &t.ball, (int)ng);
  if (w) *w = t;
  return c.off;
}

int topk_rerank_impl(const float* Xq, int64_t nq, const float* Xg, int64_t ng, int32_t d, const gcr_params* p,
                     int32_t* idx_out, float* dist_out, const TopkRerankWs& w, cudaStream_t st) {
  const bool bf = tensor_mode(p);
  {
    StageScope sc_(GCR_STAGE_PREP, st, 2);
    GCR_CUDA_TRY(launch_row_stats(Xg, (int)ng, d, w.n64g, w.n32g, bf ? w.gr : nullptr, elt_of(p), w.genrm, w.ganrm,
                                  w.scg, st));
  }
  GCR_CUDA_TRY(cudaMemsetAsync(w.sw.stats, 0, sizeof(unsigned long long) * GCR_STATS_LEN, st));
  const GallerySide gs{Xg, w.gr, w.n64g, w.scg, w.genrm, w.ganrm};
  return serve_knn(Xq, (int)nq, d, p, p->topk_out, serve_kp_final(p), gs, (int)ng, w.sw, w.sw.stats, idx_out,
                   dist_out, st, SeedSource(), bf ? &w.ball : nullptr);
}

// The whole re-ranking on device buffers (gcr_pipeline); hd (may be NULL) delivers the
// ranking of the full-sort path to host memory chunk by chunk.
int pipeline_impl(const float* X, int64_t n, int64_t nq, int32_t d, const int32_t* cam, const gcr_params* p,
                  const Resolved& r, float* X_final, int32_t* idx_out, float* dist_out, int64_t* stats,
                  PipeWs& w, cudaStream_t st, const HostDelivery* hd) {
  int s = GCR_OK;
  w.g.stats = stats;
  {
    StageScope sc_(GCR_STAGE_NORMALIZE, st);
    GCR_CUDA_TRY(launch_normalize(X, w.Xa, n, d, st));
  }
  float* cur = w.Xa;
  float* nxt = w.Xb;
  for (int t = 0; t < p->T; ++t) {
    Carve cb(w.inner, w.inner_bytes);
    BuildWs bw;
    carve_build(cb, n, d, p, r, &bw);
    s = build_graph_impl(cur, n, d, cam, p, r, &w.g, bw, st);
    if (s != GCR_OK) return s;
    {
      StageScope sc_(GCR_STAGE_PROPAGATE, st);
      GCR_CUDA_TRY(launch_propagate(w.g.op_rowptr, w.g.op_len, w.g.op_col, w.g.op_val, cur, nxt, (int)n, d,
                                    p->k > 0 ? w.g.row_order : nullptr, st));
    }
    float* tmp = cur; cur = nxt; nxt = tmp;
  }
  Carve cr(w.inner, w.inner_bytes);
  if (rerank_uses_pool(p, n - nq)) {
    TopkRerankWs tw;
    carve_topk_rerank(cr, nq, n - nq, d, p, &tw);
    s = topk_rerank_impl(cur, nq, cur + (size_t)nq * d, n - nq, d, p, idx_out, dist_out, tw, st);
  } else {
    RerankWs rw;
    carve_rerank(cr, nq, n - nq, d, tensor_mode(p), &rw);
    s = rerank_impl(cur, nq, cur + (size_t)nq * d, n - nq, d, p, idx_out, dist_out, rw, st, hd);
  }
  if (s != GCR_OK) return s;
  if (X_final) GCR_CUDA_TRY(cudaMemcpyAsync(X_final, cur, sizeof(float) * n * d, cudaMemcpyDeviceToDevice, st));
  return GCR_OK;
}

// Device staging of gcr_pipeline_host: camera ids and the ranking.
struct HostStaging {
  int32_t* cam;
  int32_t* idx;
  float* dist;
};
size_t carve_host_staging(Carve& c, int64_t n, int64_t nq, const gcr_params* p, HostStaging* h) {
  const int64_t ng = n - nq;
  const int64_t K = p->topk_out > 0 ? std::min<int64_t>(p->topk_out, ng) : ng;
  HostStaging t;
  t.cam = c.take<int32_t>((size_t)n);
  t.idx = c.take<int32_t>((size_t)nq * K);
  t.dist = c.take<float>((size_t)nq * K);
  if (h) *h = t;
  return c.off;
}

// Per-device copy stream and events of gcr_pipeline_host, created on first use and kept.
constexpr int kHostChunks = 8;
constexpr int kMaxDevices = 64;
struct HostCopyState {
  bool ready = false;
  cudaStream_t copy = nullptr;
  cudaEvent_t ev[kHostChunks + 1];
};
std::mutex g_copy_mu;
HostCopyState g_copy[kMaxDevices];

// Workspace of gcr_dsfp: the normalised input, the kNN lists and the kNN search's own.
struct DsfpWs {
  float* Xn;
  int32_t* nbr;
  float* d2;
  BuildWs bw;
};

size_t carve_dsfp(Carve& c, int64_t n, int32_t d, const gcr_params* p, const Resolved& r, DsfpWs* w) {
  DsfpWs t;
  t.Xn = c.take<float>((size_t)n * d);
  t.nbr = c.take<int32_t>((size_t)n * p->k);
  t.d2 = c.take<float>((size_t)n * p->k);
  carve_build(c, n, d, p, r, &t.bw);
  if (w) *w = t;
  return c.off;
}

int check_dsfp(const gcr_params* p, int64_t n, int32_t d, Resolved* r) {
  const int s = check_params(p, n, d, r);
  if (s != GCR_OK) return s;
  if (p->cross_camera || p->T < 0) return GCR_E_INVALID;
  if (p->k > kDsfpMaxK) return GCR_E_UNSUPPORTED;
  return GCR_OK;
}

}  // namespace

extern "C" {

const char* gcr_status_string(int s) {
  switch (s) {
    case GCR_OK: return "ok";
    case GCR_E_INVALID: return "invalid argument";
    case GCR_E_WORKSPACE: return "workspace too small";
    case GCR_E_CUDA: return "CUDA error";
    case GCR_E_TIMEOUT: return "device wait timed out";
    case GCR_E_UNSUPPORTED: return "unsupported shape or mode";
    default: return "unknown status";
  }
}

int gcr_version(void) { return 100; }

int gcr_profile_enable(int on) {
  if (on && !g_prof.created) {
    for (int i = 0; i < StageProfiler::kMaxRec; ++i)
      for (int j = 0; j < 2; ++j)
        if (cudaEventCreate(&g_prof.ev[i][j]) != cudaSuccess) return GCR_E_CUDA;
    g_prof.created = true;
  }
  g_prof.on = on != 0;
  g_prof.used = 0;
  return GCR_OK;
}

int gcr_profile_read(double* ms, int64_t* launches, int64_t* calls, int n_stages) {
  if (!ms || !launches || !calls || n_stages < 1) return GCR_E_INVALID;
  for (int s = 0; s < n_stages; ++s) { ms[s] = 0.0; launches[s] = 0; calls[s] = 0; }
  for (int i = 0; i < g_prof.used; ++i) {
    if (cudaEventSynchronize(g_prof.ev[i][1]) != cudaSuccess) return GCR_E_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, g_prof.ev[i][0], g_prof.ev[i][1]) != cudaSuccess) return GCR_E_CUDA;
    const int s = g_prof.stage[i];
    if (s < n_stages) { ms[s] += t; launches[s] += g_prof.launches[i]; calls[s] += 1; }
  }
  g_prof.used = 0;
  return GCR_OK;
}

void gcr_default_params(gcr_params* p) {
  if (!p) return;
  p->k = 15;
  p->gamma = 0.2f;
  p->alpha = 0.7f;
  p->symmetric = 1;
  p->cross_camera = 0;
  p->precision = GCR_PREC_FP32;
  p->pool = 0;
  p->topk_out = 0;
  p->T = 3;
}

int gcr_device_supported(int device) {
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) return 0;
  return (major == 10 && minor == 3) ? 1 : 0;
}

int gcr_sync(gcr_stream_t stream) {
  GCR_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  GCR_CUDA_TRY(cudaGetLastError());
  const int t = umma_read_and_clear_timeouts();
  if (t < 0) return GCR_E_CUDA;
  if (t > 0) return GCR_E_TIMEOUT;
  return GCR_OK;
}

int gcr_selftest_wait_timeout(int64_t limit_us, gcr_stream_t stream) {
  if (limit_us < 1 || limit_us > 1000000) return GCR_E_INVALID;
  GCR_CUDA_TRY(launch_wait_probe((unsigned long long)limit_us * 1000ull, (cudaStream_t)stream));
  return GCR_OK;
}

int gcr_normalize(const float* X_in, float* X_out, int64_t n, int32_t d, gcr_stream_t stream) {
  if (!X_in || !X_out || n < 1 || d < 4 || d > kMaxD || misaligned(X_in) || misaligned(X_out)) return GCR_E_INVALID;
  if (d % 4 != 0) return GCR_E_UNSUPPORTED;
  StageScope sc_(GCR_STAGE_NORMALIZE, (cudaStream_t)stream);
  GCR_CUDA_TRY(launch_normalize(X_in, X_out, n, d, (cudaStream_t)stream));
  return GCR_OK;
}

size_t gcr_graph_op_capacity(int64_t n, const gcr_params* p) {
  if (!p || n < 1) return 0;
  return op_capacity(n, p, p->cross_camera ? 2 : 1);
}

size_t gcr_build_graph_workspace_size(int64_t n, int32_t d, const gcr_params* p) {
  Resolved r;
  if (check_params(p, n, d, &r) != GCR_OK) return 0;
  Carve c(nullptr, 0);
  return carve_build(c, n, d, p, r, nullptr) + 256;
}

int gcr_build_graph(const float* X, int64_t n, int32_t d, const int32_t* cam, const gcr_params* p,
                    gcr_graph* g, void* ws, size_t ws_bytes, gcr_stream_t stream) {
  Resolved r;
  int s = check_params(p, n, d, &r);
  if (s != GCR_OK) return s;
  if (!X || misaligned(X) || (p->cross_camera && !cam)) return GCR_E_INVALID;
  s = check_graph(g, r.kinds, p->k);
  if (s != GCR_OK) return s;
  if (!ws) return GCR_E_WORKSPACE;
  Carve c(ws, ws_bytes);
  BuildWs w;
  if (carve_build(c, n, d, p, r, &w) > ws_bytes) return GCR_E_WORKSPACE;
  return build_graph_impl(X, n, d, cam, p, r, g, w, (cudaStream_t)stream);
}

int gcr_propagate(const gcr_graph* g, const float* X_in, float* X_out, int64_t n, int32_t d, gcr_stream_t stream) {
  if (!g || !g->op_rowptr || !g->op_len || !g->op_col || !g->op_val || !X_in || !X_out) return GCR_E_INVALID;
  if (X_in == X_out || n < 1 || n > (1 << 24) || d < 4 || d > kMaxD) return GCR_E_INVALID;
  if (misaligned(X_in) || misaligned(X_out)) return GCR_E_INVALID;
  if (d % 4 != 0) return GCR_E_UNSUPPORTED;
  StageScope sc_(GCR_STAGE_PROPAGATE, (cudaStream_t)stream);
  GCR_CUDA_TRY(launch_propagate(g->op_rowptr, g->op_len, g->op_col, g->op_val, X_in, X_out, (int)n, d,
                                g->row_order, (cudaStream_t)stream));
  return GCR_OK;
}

size_t gcr_rerank_workspace_size(int64_t nq, int64_t ng, int32_t d, const gcr_params* p) {
  if (check_rerank(nq, ng, d, p) != GCR_OK) return 0;
  Carve c(nullptr, 0);
  if (rerank_uses_pool(p, ng)) return carve_topk_rerank(c, nq, ng, d, p, nullptr) + 256;
  return carve_rerank(c, nq, ng, d, tensor_mode(p), nullptr) + 256;
}

int gcr_rerank(const float* Xq, int64_t nq, const float* Xg, int64_t ng, int32_t d, const gcr_params* p,
               int32_t* idx_out, float* dist_out, void* ws, size_t ws_bytes, gcr_stream_t stream) {
  int s = check_rerank(nq, ng, d, p);
  if (s != GCR_OK) return s;
  if (!Xq || !Xg || !idx_out || !dist_out || misaligned(Xq) || misaligned(Xg)) return GCR_E_INVALID;
  if (!ws) return GCR_E_WORKSPACE;
  Carve c(ws, ws_bytes);
  if (rerank_uses_pool(p, ng)) {
    TopkRerankWs tw;
    if (carve_topk_rerank(c, nq, ng, d, p, &tw) > ws_bytes) return GCR_E_WORKSPACE;
    return topk_rerank_impl(Xq, nq, Xg, ng, d, p, idx_out, dist_out, tw, (cudaStream_t)stream);
  }
  RerankWs w;
  if (carve_rerank(c, nq, ng, d, tensor_mode(p), &w) > ws_bytes) return GCR_E_WORKSPACE;
  return rerank_impl(Xq, nq, Xg, ng, d, p, idx_out, dist_out, w, (cudaStream_t)stream);
}

size_t gcrv_profiles_workspace_size(int64_t F, int32_t d, int32_t C, int32_t n_cams) {
  if (F < 1 || C < 1 || d < 4 || d > kMaxD || d % 4 || n_cams < 1 || n_cams > 64 || F > (int64_t)INT32_MAX) return 0;
  Carve c(nullptr, 0);
  return gcrv_carve(c, F, d, C, n_cams, nullptr) + 256;
}

int gcrv_profiles(const float* frames, int64_t F, int32_t d, const int64_t* trk_off, const int32_t* trk_cam,
                  int32_t C, int32_t n_cams, float lambda, float* W_out, void* ws, size_t ws_bytes,
                  gcr_stream_t stream) {
  if (!frames || !trk_off || !trk_cam || !W_out || misaligned(frames) || misaligned(W_out)) return GCR_E_INVALID;
  if (F < 1 || C < 1 || n_cams < 1 || n_cams > 64 || F > (int64_t)INT32_MAX) return GCR_E_INVALID;
  if (d < 4 || d > kMaxD) return GCR_E_INVALID;
  if (d % 4 != 0) return GCR_E_UNSUPPORTED;
  if (!(lambda > 0.f) || !std::isfinite(lambda)) return GCR_E_INVALID;
  if (!ws) return GCR_E_WORKSPACE;
  Carve c(ws, ws_bytes);
  GcrvWs w;
  if (gcrv_carve(c, F, d, C, n_cams, &w) > ws_bytes) return GCR_E_WORKSPACE;
  StageScope sc_(GCR_STAGE_GCRV, (cudaStream_t)stream);
  GCR_CUDA_TRY(launch_gcrv(frames, F, d, trk_off, trk_cam, C, n_cams, lambda, W_out, w, (cudaStream_t)stream));
  return GCR_OK;
}

size_t gcrv_mean_profiles_workspace_size(int64_t F, int32_t d, int32_t C) {
  if (F < 1 || C < 1 || F > (int64_t)INT32_MAX || d < 4 || d > kMaxD || d % 4) return 0;
  return sizeof(float) * (size_t)F + 256;
}

int gcrv_mean_profiles(const float* frames, int64_t F, int32_t d, const int64_t* trk_off, int32_t C, float* W_out,
                       void* ws, size_t ws_bytes, gcr_stream_t stream) {
  if (!frames || !trk_off || !W_out || misaligned(frames) || misaligned(W_out)) return GCR_E_INVALID;
  if (F < 1 || C < 1 || F > (int64_t)INT32_MAX || d < 4 || d > kMaxD) return GCR_E_INVALID;
  if (d % 4 != 0) return GCR_E_UNSUPPORTED;
  if (!ws) return GCR_E_WORKSPACE;
  Carve c(ws, ws_bytes);
  float* inv = c.take<float>((size_t)F);
  if (c.off > ws_bytes) return GCR_E_WORKSPACE;
  StageScope sc_(GCR_STAGE_GCRV, (cudaStream_t)stream);
  GCR_CUDA_TRY(launch_gcrv_means(frames, F, d, trk_off, C, inv, W_out, (cudaStream_t)stream));
  return GCR_OK;
}

size_t gcr_gallery_bytes(int64_t ng, int32_t d, const gcr_params* p) {
  Resolved r;
  if (check_serve_params(p, ng, d, &r) != GCR_OK) return 0;
  Carve c(nullptr, 0);
  return carve_gallery(c, ng, d, p, nullptr) + 256;
}

size_t gcr_gallery_build_workspace_size(int64_t ng, int32_t d, const gcr_params* p) {
  Resolved r;
  if (check_serve_params(p, ng, d, &r) != GCR_OK) return 0;
  Carve c(nullptr, 0);
  return carve_gallery_build(c, ng, d, p, r, nullptr) + 256;
}

int gcr_gallery_build(const float* Xg, int64_t ng, int32_t d, const gcr_params* p, void* state, size_t state_bytes,
                      void* ws, size_t ws_bytes, gcr_stream_t stream) {
  Resolved r;
  int s = check_serve_params(p, ng, d, &r);
  if (s != GCR_OK) return s;
  if (!Xg || !state || misaligned(Xg)) return GCR_E_INVALID;
  if (!ws) return GCR_E_WORKSPACE;
  Carve cs(state, state_bytes);
  GalleryView g;
  if (carve_gallery(cs, ng, d, p, &g) > state_bytes) return GCR_E_WORKSPACE;
  Carve cw(ws, ws_bytes);
  GalleryBuildWs w;
  if (carve_gallery_build(cw, ng, d, p, r, &w) > ws_bytes) return GCR_E_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = (int)ng;
  const bool bf = tensor_mode(p);
  const size_t es = elt_size(p);
  GCR_CUDA_TRY(launch_normalize(Xg, g.layers, ng, d, st));
  for (int t = 0; t < p->T; ++t) {
    float* cur = g.layers + (size_t)t * n * d;
    float* nxt = g.layers + (size_t)(t + 1) * n * d;
    Carve cb(w.inner, w.inner_bytes);
    BuildWs bw;
    carve_build(cb, ng, d, p, r, &bw);
    s = build_graph_impl(cur, ng, d, nullptr, p, r, &w.g, bw, st);
    if (s != GCR_OK) return s;
    GCR_CUDA_TRY(launch_layer_degree(w.g.deg_r, w.g.deg_c, n, p->symmetric, g.deg + (size_t)t * n, st));
    GCR_CUDA_TRY(launch_propagate(w.g.op_rowptr, w.g.op_len, w.g.op_col, w.g.op_val, cur, nxt, n, d,
                                  p->k > 0 ? w.g.row_order : nullptr, st));
  }
  if (p->T >= 1 && p->k > 0)
    GCR_CUDA_TRY(cudaMemcpyAsync(g.nbr, w.g.nbr, sizeof(int32_t) * (size_t)n * p->k, cudaMemcpyDeviceToDevice, st));
  for (int t = 0; t <= p->T; ++t) {
    GCR_CUDA_TRY(launch_row_stats(g.layers + (size_t)t * n * d, n, d, g.n64 + (size_t)t * n, g.n32 + (size_t)t * n,
                                  bf ? g.xr + (size_t)t * n * d * es : nullptr, elt_of(p),
                                  bf ? g.enrm + (size_t)t * n : nullptr,
                                  bf ? g.anrm + (size_t)t * n : nullptr, g.sc + t, st));
  }
  return GCR_OK;
}

size_t gcr_serve_workspace_size(int64_t b, int64_t ng, int32_t d, const gcr_params* p) {
  Resolved r;
  if (b < 1 || check_serve_params(p, ng, d, &r) != GCR_OK) return 0;
  Carve c(nullptr, 0);
  return carve_serve(c, b, d, p, r, nullptr) + 256;
}

int gcr_serve(const void* state, size_t state_bytes, int64_t ng, const float* Xq, int64_t b, int32_t d,
              const gcr_params* p, int32_t* idx_out, float* dist_out, int64_t* stats, void* ws, size_t ws_bytes,
              gcr_stream_t stream) {
  Resolved r;
  int s = check_serve_params(p, ng, d, &r);
  if (s != GCR_OK) return s;
  if (!state || !Xq || !idx_out || !dist_out || b < 1 || b > (1 << 20) || misaligned(Xq)) return GCR_E_INVALID;
  Carve cs(const_cast<void*>(state), state_bytes);
  GalleryView g;
  if (carve_gallery(cs, ng, d, p, &g) > state_bytes) return GCR_E_WORKSPACE;
  if (!ws) return GCR_E_WORKSPACE;
  Carve cw(ws, ws_bytes);
  ServeWs w;
  if (carve_serve(cw, b, d, p, r, &w) > ws_bytes) return GCR_E_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* stp = stats ? reinterpret_cast<unsigned long long*>(stats) : w.stats;
  const int nq = (int)b, n = (int)ng;
  {
    StageScope sc_(GCR_STAGE_NORMALIZE, st);
    GCR_CUDA_TRY(launch_normalize(Xq, w.xq[0], b, d, st));
  }
  int cur = 0;
  for (int t = 0; t < p->T; ++t) {
    if (p->k > 0) {
      // every search after the first starts from the previous search's pool; the first one, for
      // 32 queries or more, from a sample of the gallery (the seed kernel, one latency-bound CTA
      // per query, costs more than it saves for fewer: measured 1.63 -> 1.76 ms per call at b = 1,
      // 2.75 -> 2.37 ms at b = 64 on a 500,000 x 256 gallery)
      SeedSource src;
      if (t > 0)
        src.prev_kp = r.kp;
      else if (nq >= 32)
        src.sample = (int)std::min<int64_t>(ng, kSeedCandidates);
      s = serve_knn(w.xq[cur], nq, d, p, p->k, r.kp, gallery_layer(g, t, n, d, elt_size(p)), n, w, stp, w.nbr, w.d2,
                    st, src);
      if (s != GCR_OK) return s;
    }
    StageScope sc_(GCR_STAGE_PROPAGATE, st);
    GCR_CUDA_TRY(launch_query_step(w.xq[cur], nq, d, g.layers + (size_t)t * n * d, g.deg + (size_t)t * n, w.nbr,
                                   w.d2, p->k, p->gamma, p->symmetric, w.xq[cur ^ 1], st));
    cur ^= 1;
  }
  // the final search starts from the last layer search's pool, those rows' gallery lists and,
  // when it must certify more rows than that pool holds, a sample of the gallery (the lists
  // mostly lead back into the pool's own clusters)
  SeedSource src;
  if (p->T >= 1 && p->k > 0) {
    src.prev_kp = r.kp;
    if (r.kp * (1 + p->k) <= kSeedCandidates) {
      src.hop = g.nbr;
      src.hop_k = p->k;
    }
    if (p->topk_out > r.kp)
      src.sample = (int)std::min<int64_t>(ng, kSeedCandidates - (int64_t)r.kp * (1 + src.hop_k));
  }
  return serve_knn(w.xq[cur], nq, d, p, p->topk_out, serve_kp_final(p), gallery_layer(g, p->T, n, d, elt_size(p)), n, w, stp,
                   idx_out, dist_out, st, src);
}

size_t gcr_pipeline_workspace_size(int64_t n, int64_t nq, int32_t d, const gcr_params* p) {
  Resolved r;
  if (check_params(p, n, d, &r) != GCR_OK) return 0;
  if (nq < 1 || nq >= n || check_rerank(nq, n - nq, d, p) != GCR_OK) return 0;
  Carve c(nullptr, 0);
  return carve_pipe(c, n, nq, d, p, r, nullptr) + 256;
}

int gcr_pipeline(const float* X, int64_t n, int64_t nq, int32_t d, const int32_t* cam, const gcr_params* p,
                 float* X_final, int32_t* idx_out, float* dist_out, int64_t* stats, void* ws, size_t ws_bytes,
                 gcr_stream_t stream) {
  Resolved r;
  int s = check_params(p, n, d, &r);
  if (s != GCR_OK) return s;
  if (nq < 1 || nq >= n) return GCR_E_INVALID;
  s = check_rerank(nq, n - nq, d, p);
  if (s != GCR_OK) return s;
  if (!X || !idx_out || !dist_out || (p->cross_camera && !cam) || p->T < 0) return GCR_E_INVALID;
  if (misaligned(X) || misaligned(X_final)) return GCR_E_INVALID;
  if (!ws) return GCR_E_WORKSPACE;
  Carve c(ws, ws_bytes);
  PipeWs w;
  if (carve_pipe(c, n, nq, d, p, r, &w) > ws_bytes) return GCR_E_WORKSPACE;
  return pipeline_impl(X, n, nq, d, cam, p, r, X_final, idx_out, dist_out, stats, w, (cudaStream_t)stream, nullptr);
}

size_t gcr_pipeline_host_workspace_size(int64_t n, int64_t nq, int32_t d, const gcr_params* p) {
  Resolved r;
  if (check_params(p, n, d, &r) != GCR_OK) return 0;
  if (nq < 1 || nq >= n || check_rerank(nq, n - nq, d, p) != GCR_OK) return 0;
  Carve c(nullptr, 0);
  carve_pipe(c, n, nq, d, p, r, nullptr);
  HostStaging h;
  return carve_host_staging(c, n, nq, p, &h) + 256;
}

int gcr_pipeline_host(const float* X_host, int64_t n, int64_t nq, int32_t d, const int32_t* cam_host,
                      const gcr_params* p, int32_t* idx_host, float* dist_host, int64_t* stats, void* ws,
                      size_t ws_bytes, gcr_stream_t stream) {
  Resolved r;
  int s = check_params(p, n, d, &r);
  if (s != GCR_OK) return s;
  if (nq < 1 || nq >= n) return GCR_E_INVALID;
  s = check_rerank(nq, n - nq, d, p);
  if (s != GCR_OK) return s;
  if (!X_host || !idx_host || !dist_host || (p->cross_camera && !cam_host) || p->T < 0) return GCR_E_INVALID;
  if (!ws) return GCR_E_WORKSPACE;
  Carve c(ws, ws_bytes);
  PipeWs w;
  carve_pipe(c, n, nq, d, p, r, &w);
  HostStaging h;
  if (carve_host_staging(c, n, nq, p, &h) > ws_bytes) return GCR_E_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  GCR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return GCR_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_copy_mu);
  HostCopyState& cs = g_copy[dev];
  if (!cs.ready) {
    GCR_CUDA_TRY(cudaStreamCreateWithFlags(&cs.copy, cudaStreamNonBlocking));
    for (int e = 0; e <= kHostChunks; ++e) GCR_CUDA_TRY(cudaEventCreateWithFlags(&cs.ev[e], cudaEventDisableTiming));
    cs.ready = true;
  }
  // the input rows land in the second feature buffer, which the pipeline only overwrites
  // after normalising them into the first
  GCR_CUDA_TRY(cudaMemcpyAsync(w.Xb, X_host, sizeof(float) * n * d, cudaMemcpyHostToDevice, st));
  if (p->cross_camera) GCR_CUDA_TRY(cudaMemcpyAsync(h.cam, cam_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
  const int64_t ng = n - nq;
  const int64_t K = p->topk_out > 0 ? std::min<int64_t>(p->topk_out, ng) : ng;
  HostDelivery hd;
  hd.idx_host = idx_host;
  hd.dist_host = dist_host;
  const int64_t tiles = (nq + 127) / 128;
  const int64_t per = (tiles + kHostChunks - 1) / kHostChunks;
  hd.chunk_rows = (int)(per * 128);
  hd.copy = cs.copy;
  hd.ready = cs.ev;
  hd.n_events = kHostChunks;
  s = pipeline_impl(w.Xb, n, nq, d, p->cross_camera ? h.cam : nullptr, p, r, nullptr, h.idx, h.dist, stats, w, st,
                    &hd);
  if (s != GCR_OK) return s;
  if (rerank_uses_pool(p, ng)) {
    // the certified top-K search returns all rows at once: copy them after it
    GCR_CUDA_TRY(cudaEventRecord(cs.ev[0], st));
    GCR_CUDA_TRY(cudaStreamWaitEvent(cs.copy, cs.ev[0], 0));
    GCR_CUDA_TRY(cudaMemcpyAsync(idx_host, h.idx, sizeof(int32_t) * nq * K, cudaMemcpyDeviceToHost, cs.copy));
    GCR_CUDA_TRY(cudaMemcpyAsync(dist_host, h.dist, sizeof(float) * nq * K, cudaMemcpyDeviceToHost, cs.copy));
  }
  // the caller's stream completes only after the last copy
  GCR_CUDA_TRY(cudaEventRecord(cs.ev[kHostChunks], cs.copy));
  GCR_CUDA_TRY(cudaStreamWaitEvent(st, cs.ev[kHostChunks], 0));
  return GCR_OK;
}

// ---------------------------------------------------------------- DSFP (Algorithm 1)
size_t gcr_dsfp_workspace_size(int64_t n, int32_t d, const gcr_params* p) {
  Resolved r;
  if (check_dsfp(p, n, d, &r) != GCR_OK) return 0;
  Carve c(nullptr, 0);
  return carve_dsfp(c, n, d, p, r, nullptr) + 256;
}

int gcr_dsfp(const float* X, int64_t n, int32_t d, const gcr_params* p, float* X_out, int32_t* nbr_out,
             int64_t* stats, void* ws, size_t ws_bytes, gcr_stream_t stream) {
  Resolved r;
  int s = check_dsfp(p, n, d, &r);
  if (s != GCR_OK) return s;
  if (!X || !X_out || X == X_out || misaligned(X) || misaligned(X_out)) return GCR_E_INVALID;
  if (!ws) return GCR_E_WORKSPACE;
  Carve c(ws, ws_bytes);
  DsfpWs w;
  if (carve_dsfp(c, n, d, p, r, &w) > ws_bytes) return GCR_E_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  {
    StageScope sc_(GCR_STAGE_NORMALIZE, st);
    GCR_CUDA_TRY(launch_normalize(X, w.Xn, n, d, st));
  }
  int32_t* nbr = nbr_out ? nbr_out : w.nbr;
  if (p->k > 0) {
    // step 1 of Algorithm 1: the certified kNN search on the normalised input
    gcr_graph g;
    std::memset(&g, 0, sizeof(g));
    g.nbr = nbr;
    g.nbr_d2 = w.d2;
    g.stats = stats;
    s = knn_impl(w.Xn, n, d, nullptr, p, r, &g, w.bw, st);
    if (s != GCR_OK) return s;
  }
  StageScope sc_(GCR_STAGE_PROPAGATE, st);
  GCR_CUDA_TRY(launch_dsfp(w.Xn, (int)n, d, nbr, p->k, p->gamma, p->T, X_out, st));
  return GCR_OK;
}

int gcr_dsfp_propagate(const float* X, int64_t n, int32_t d, const int32_t* nbr, int32_t k, float gamma,
                       int32_t T, float* X_out, gcr_stream_t stream) {
  if (!X || !X_out || X == X_out || n < 1 || n > (1 << 24) || d < 4 || d > kMaxD || k < 0 || T < 0)
    return GCR_E_INVALID;
  if (!(gamma > 0.f) || !std::isfinite(gamma)) return GCR_E_INVALID;
  if (k > 0 && !nbr) return GCR_E_INVALID;
  if (misaligned(X) || misaligned(X_out)) return GCR_E_INVALID;
  if (k > kDsfpMaxK || d % 4) return GCR_E_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  StageScope sc_(GCR_STAGE_PROPAGATE, st);
  GCR_CUDA_TRY(launch_dsfp(X, (int)n, d, nbr, k, gamma, T, X_out, st));
  return GCR_OK;
}

int gcr_eval_retrieval(const int32_t* idx, int64_t nq, int64_t K, const int32_t* q_label, const int32_t* q_cam,
                       const int32_t* g_label, const int32_t* g_cam, int64_t ng, int32_t protocol, double* ap_out,
                       int32_t* first_out, gcr_stream_t stream) {
  if (!idx || !q_label || !g_label || !ap_out || !first_out) return GCR_E_INVALID;
  if (nq < 1 || nq > INT32_MAX || K < 1 || ng < 1 || ng > INT32_MAX || K > ((int64_t)1 << 40) / nq)
    return GCR_E_INVALID;
  if (protocol != 0 && protocol != 1) return GCR_E_INVALID;
  if (protocol == 1 && (!q_cam || !g_cam)) return GCR_E_INVALID;
  GCR_CUDA_TRY(launch_eval(idx, (int)nq, (long)K, q_label, q_cam, g_label, g_cam, (int)ng, protocol, ap_out,
                           first_out, (cudaStream_t)stream));
  return GCR_OK;
}

}  // extern "C"
