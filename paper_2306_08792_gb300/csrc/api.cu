// Host entry points of the C ABI declared in include/gcr.h.
//
// Every entry point validates its arguments on the host, carves its scratch from the
// caller's workspace and enqueues kernels on the caller's stream. Nothing here allocates
// device memory or synchronises (except gcr_sync).
#include <cmath>
#include <cstring>

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
constexpr int kBandRowsMax = 32768;  // (row, graph) pairs a band rescan can hold
constexpr int kMaxD = 4096;

struct Resolved {
  int kp;
  int kinds;
};

int check_params(const gcr_params* p, int64_t n, int32_t d, Resolved* r) {
  if (!p || n < 1 || n > (1 << 24)) return GCR_E_INVALID;
  if (d < 4 || d > kMaxD) return GCR_E_INVALID;
  if (d % 4 != 0) return GCR_E_UNSUPPORTED;
  if (p->precision != GCR_PREC_FP32 && p->precision != GCR_PREC_BF16) return GCR_E_INVALID;
  if (p->precision == GCR_PREC_BF16 && d % 8 != 0) return GCR_E_UNSUPPORTED;
  if (!(p->gamma > 0.f) || !std::isfinite(p->gamma)) return GCR_E_INVALID;
  if (p->symmetric != 0 && p->symmetric != 1) return GCR_E_INVALID;
  if (p->cross_camera != 0 && p->cross_camera != 1) return GCR_E_INVALID;
  if (p->cross_camera && !(p->alpha >= 0.f && p->alpha <= 1.f)) return GCR_E_INVALID;
  int kp = p->pool ? p->pool : (p->precision == GCR_PREC_BF16 ? 64 : 32);
  if (kp != 32 && kp != 64) return GCR_E_INVALID;
  if (p->k < 0 || p->k >= kp) return GCR_E_INVALID;
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
  __nv_bfloat16* xb;
  float* enrm;
  float* anrm;
  float* pool_v;
  int* pool_i;
  int* unc_count;
  int* unc_row;
  int* unc_kind;
  float* unc_thr;
  int* band_cnt;
  float* band_v;
  int* band_i;
  __nv_bfloat16* band_a;
  float* w;
  int* cnt;
  int* fill;
  int* t_src;
  float* t_w;
  int* raw_col;
  float* raw_val;
  int* op_cnt;
  int* scan_tmp;
  unsigned long long* stats;
  int* err;
  int band_rows;
};

size_t carve_build(Carve& c, int64_t n, int32_t d, const gcr_params* p, const Resolved& r, BuildWs* w) {
  const size_t nn = (size_t)n;
  const int kinds = r.kinds;
  const bool bf = p->precision == GCR_PREC_BF16;
  const int band_rows = (int)std::min<int64_t>((int64_t)kinds * n, kBandRowsMax);
  const size_t cap = op_capacity(n, p, kinds);
  BuildWs t;
  t.n64 = c.take<double>(nn);
  t.n32 = c.take<float>(nn);
  t.sc = c.take<RowScalars>(1);
  t.xb = bf ? c.take<__nv_bfloat16>(nn * d) : nullptr;
  t.enrm = bf ? c.take<float>(nn) : nullptr;
  t.anrm = bf ? c.take<float>(nn) : nullptr;
  t.pool_v = c.take<float>((size_t)kinds * nn * r.kp);
  t.pool_i = c.take<int>((size_t)kinds * nn * r.kp);
  t.unc_count = c.take<int>(4);
  t.unc_row = c.take<int>((size_t)kinds * nn);
  t.unc_kind = c.take<int>((size_t)kinds * nn);
  t.unc_thr = c.take<float>((size_t)kinds * nn);
  t.band_cnt = c.take<int>(band_rows);
  t.band_v = c.take<float>((size_t)band_rows * kBandCap);
  t.band_i = c.take<int>((size_t)band_rows * kBandCap);
  t.band_a = bf ? c.take<__nv_bfloat16>((size_t)band_rows * d) : nullptr;
  t.w = c.take<float>((size_t)kinds * nn * p->k);
  t.cnt = c.take<int>((size_t)kinds * (nn + 1));
  t.fill = c.take<int>((size_t)kinds * nn);
  t.t_src = c.take<int>((size_t)kinds * nn * p->k);
  t.t_w = c.take<float>((size_t)kinds * nn * p->k);
  t.raw_col = c.take<int>(cap);
  t.raw_val = c.take<float>(cap);
  t.op_cnt = c.take<int>(nn);
  t.scan_tmp = c.take<int>(nn + 1);
  t.stats = c.take<unsigned long long>(GCR_STATS_LEN);
  t.err = c.take<int>(4);
  t.band_rows = band_rows;
  if (w) *w = t;
  return c.off;
}

int build_graph_impl(const float* X, int64_t n64_, int32_t d, const int32_t* cam, const gcr_params* p,
                     const Resolved& r, gcr_graph* g, const BuildWs& w, cudaStream_t st) {
  const int n = (int)n64_;
  const int kinds = r.kinds;
  const bool bf = p->precision == GCR_PREC_BF16;
  unsigned long long* stats = g->stats ? reinterpret_cast<unsigned long long*>(g->stats) : w.stats;
  if (!g->stats) GCR_CUDA_TRY(cudaMemsetAsync(w.stats, 0, sizeof(unsigned long long) * GCR_STATS_LEN, st));

  {
    StageScope sc_(GCR_STAGE_PREP, st, 2);
    GCR_CUDA_TRY(launch_row_stats(X, n, d, w.n64, w.n32, bf ? w.xb : nullptr, w.enrm, w.anrm, w.sc, st));
  }
  GCR_CUDA_TRY(cudaMemsetAsync(w.unc_count, 0, sizeof(int) * 4, st));
  GCR_CUDA_TRY(cudaMemsetAsync(w.band_cnt, 0, sizeof(int) * w.band_rows, st));
  GCR_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int) * 4, st));
  const int* camp = p->cross_camera ? cam : nullptr;

  if (p->k > 0) {
    StageScope sc_(GCR_STAGE_SIM_GEMM, st);
    if (bf) {
      GCR_CUDA_TRY(launch_umma_pool(w.xb, n, d, camp, p->cross_camera != 0, w.pool_v, w.pool_i, w.err, st));
    } else {
      GCR_CUDA_TRY(launch_sgemm_pool(X, n, d, camp, r.kp, p->cross_camera != 0, w.pool_v, w.pool_i, st));
    }
  }

  RefineArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  ra.X = X; ra.n = n; ra.d = d; ra.k = p->k; ra.kinds = kinds; ra.precision = p->precision;
  ra.n64 = w.n64; ra.enrm = w.enrm; ra.anrm = w.anrm; ra.sc = w.sc;
  ra.pool_v = w.pool_v; ra.pool_i = w.pool_i; ra.kp = r.kp;
  ra.nbr[0] = g->nbr; ra.d2[0] = g->nbr_d2;
  ra.nbr[1] = kinds == 2 ? g->nbr_cr : g->nbr;
  ra.d2[1] = kinds == 2 ? g->nbr_cr_d2 : g->nbr_d2;
  ra.unc_count = w.unc_count; ra.unc_row = w.unc_row; ra.unc_kind = w.unc_kind; ra.unc_thr = w.unc_thr;
  ra.stats = stats;
  ra.band_cnt = w.band_cnt; ra.band_v = w.band_v; ra.band_i = w.band_i; ra.bcap = kBandCap;
  ra.band_rows = w.band_rows;
  if (p->k > 0) {
    {
      StageScope sc_(GCR_STAGE_REFINE, st);
      GCR_CUDA_TRY(launch_refine_pool(ra, st));
    }
    // threshold rescan of the rows whose pool could not certify the k-th neighbour
    StageScope sc_(GCR_STAGE_BAND, st, bf ? 3 : 2);
    if (bf) {
      GCR_CUDA_TRY(launch_gather_bf16(w.xb, d, w.unc_count, w.unc_row, w.band_rows, w.band_a, st));
      GCR_CUDA_TRY(launch_umma_band(w.xb, n, d, camp, w.band_a, w.unc_count, w.band_rows, w.unc_row,
                                    w.unc_kind, w.unc_thr, kBandCap, w.band_cnt, w.band_v, w.band_i, w.err, st));
    } else {
      GCR_CUDA_TRY(launch_sgemm_band(X, n, d, camp, w.unc_count, w.band_rows, w.unc_row, w.unc_kind,
                                     w.unc_thr, kBandCap, w.band_cnt, w.band_v, w.band_i, st));
    }
    GCR_CUDA_TRY(launch_refine_band(ra, st));
  }

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
  {
    StageScope sc_(GCR_STAGE_GRAPH, st, 4 * kinds + 3);
    GCR_CUDA_TRY(launch_build_operator(ga, st));
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

size_t carve_rerank(Carve& c, int64_t nq, int64_t ng, int32_t d, bool bf, RerankWs* w) {
  RerankWs t;
  t.D = c.take<float>((size_t)nq * ng);
  t.n64q = c.take<double>(nq);
  t.n64g = c.take<double>(ng);
  t.nq = c.take<float>(nq);
  t.ng = c.take<float>(ng);
  t.sc = c.take<RowScalars>(2);
  t.qb = bf ? c.take<__nv_bfloat16>((size_t)nq * d) : nullptr;
  t.gb = bf ? c.take<__nv_bfloat16>((size_t)ng * d) : nullptr;
  t.dummy = c.take<float>(2 * (size_t)std::max(nq, ng));
  t.err = c.take<int>(4);
  if (w) *w = t;
  return c.off;
}

int rerank_impl(const float* Xq, int64_t nq, const float* Xg, int64_t ng, int32_t d, const gcr_params* p,
                int32_t* idx_out, float* dist_out, const RerankWs& w, cudaStream_t st) {
  const bool bf = p->precision == GCR_PREC_BF16;
  const int K = p->topk_out > 0 ? (int)std::min<int64_t>(p->topk_out, ng) : (int)ng;
  const size_t mx = (size_t)std::max(nq, ng);
  {
    StageScope sc_(GCR_STAGE_PREP, st, 4);
    GCR_CUDA_TRY(launch_row_stats(Xq, (int)nq, d, w.n64q, w.nq, bf ? w.qb : nullptr, w.dummy, w.dummy + mx, w.sc, st));
    GCR_CUDA_TRY(launch_row_stats(Xg, (int)ng, d, w.n64g, w.ng, bf ? w.gb : nullptr, w.dummy, w.dummy + mx, w.sc + 1, st));
  }
  if (bf) GCR_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int) * 4, st));
  {
    StageScope sc_(GCR_STAGE_DIST_GEMM, st);
    if (bf) {
    GCR_CUDA_TRY(launch_umma_dist(w.qb, (int)nq, w.gb, (int)ng, d, w.nq, w.ng, w.D, w.err, st));
  } else {
    GCR_CUDA_TRY(launch_sgemm_dist(Xq, (int)nq, Xg, (int)ng, d, w.nq, w.ng, w.D, st));
  }
  }
  {
    StageScope sc_(GCR_STAGE_SORT, st);
    GCR_CUDA_TRY(launch_rank_rows(w.D, (int)nq, (int)ng, K, idx_out, dist_out, st));
  }
  return GCR_OK;
}

int check_rerank(int64_t nq, int64_t ng, int32_t d, const gcr_params* p) {
  if (!p || nq < 1 || ng < 1 || ng > (1 << 24) || nq > (1 << 24)) return GCR_E_INVALID;
  if (d < 4 || d > kMaxD) return GCR_E_INVALID;
  if (d % 4 != 0) return GCR_E_UNSUPPORTED;
  if (p->precision != GCR_PREC_FP32 && p->precision != GCR_PREC_BF16) return GCR_E_INVALID;
  if (p->precision == GCR_PREC_BF16 && d % 8 != 0) return GCR_E_UNSUPPORTED;
  if (p->topk_out < 0) return GCR_E_INVALID;
  if (ng > 16384) return GCR_E_UNSUPPORTED;
  return GCR_OK;
}

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
  t.g.stats = nullptr;
  // the build and re-rank scratch run one after the other: they share one region
  Carve cb(nullptr, 0);
  const size_t b = carve_build(cb, n, d, p, r, nullptr);
  Carve cr(nullptr, 0);
  const size_t rr = carve_rerank(cr, nq, n - nq, d, p->precision == GCR_PREC_BF16, nullptr);
  t.inner_bytes = std::max(b, rr);
  t.inner = c.take<char>(t.inner_bytes);
  if (w) *w = t;
  return c.off;
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
  return GCR_OK;
}

int gcr_normalize(const float* X_in, float* X_out, int64_t n, int32_t d, gcr_stream_t stream) {
  if (!X_in || !X_out || n < 1 || d < 4 || d > kMaxD) return GCR_E_INVALID;
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
  if (!X || (p->cross_camera && !cam)) return GCR_E_INVALID;
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
  if (d % 4 != 0) return GCR_E_UNSUPPORTED;
  StageScope sc_(GCR_STAGE_PROPAGATE, (cudaStream_t)stream);
  GCR_CUDA_TRY(launch_propagate(g->op_rowptr, g->op_len, g->op_col, g->op_val, X_in, X_out, (int)n, d,
                                (cudaStream_t)stream));
  return GCR_OK;
}

size_t gcr_rerank_workspace_size(int64_t nq, int64_t ng, int32_t d, const gcr_params* p) {
  if (check_rerank(nq, ng, d, p) != GCR_OK) return 0;
  Carve c(nullptr, 0);
  return carve_rerank(c, nq, ng, d, p->precision == GCR_PREC_BF16, nullptr) + 256;
}

int gcr_rerank(const float* Xq, int64_t nq, const float* Xg, int64_t ng, int32_t d, const gcr_params* p,
               int32_t* idx_out, float* dist_out, void* ws, size_t ws_bytes, gcr_stream_t stream) {
  int s = check_rerank(nq, ng, d, p);
  if (s != GCR_OK) return s;
  if (!Xq || !Xg || !idx_out || !dist_out) return GCR_E_INVALID;
  if (!ws) return GCR_E_WORKSPACE;
  Carve c(ws, ws_bytes);
  RerankWs w;
  if (carve_rerank(c, nq, ng, d, p->precision == GCR_PREC_BF16, &w) > ws_bytes) return GCR_E_WORKSPACE;
  return rerank_impl(Xq, nq, Xg, ng, d, p, idx_out, dist_out, w, (cudaStream_t)stream);
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
  if (!ws) return GCR_E_WORKSPACE;
  Carve c(ws, ws_bytes);
  PipeWs w;
  if (carve_pipe(c, n, nq, d, p, r, &w) > ws_bytes) return GCR_E_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
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
      GCR_CUDA_TRY(launch_propagate(w.g.op_rowptr, w.g.op_len, w.g.op_col, w.g.op_val, cur, nxt, (int)n, d, st));
    }
    float* tmp = cur; cur = nxt; nxt = tmp;
  }
  Carve cr(w.inner, w.inner_bytes);
  RerankWs rw;
  carve_rerank(cr, nq, n - nq, d, p->precision == GCR_PREC_BF16, &rw);
  s = rerank_impl(cur, nq, cur + (size_t)nq * d, n - nq, d, p, idx_out, dist_out, rw, st);
  if (s != GCR_OK) return s;
  if (X_final) GCR_CUDA_TRY(cudaMemcpyAsync(X_final, cur, sizeof(float) * n * d, cudaMemcpyDeviceToDevice, st));
  return GCR_OK;
}

}  // extern "C"
