/*
 * gcr.h -- C ABI of the GB300 (sm_103a) implementation of Graph Convolution based
 * Re-ranking (GCR) and its video extension (GCRV), arXiv 2306.08792.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers to feature matrices, graphs, outputs and workspaces are DEVICE pointers
 *   (global memory of the current CUDA device) unless a comment says "host". The
 *   caller owns every buffer; the library never allocates, frees or retains memory.
 * - Feature matrices are row-major float32, one sample per row: X[i*d + c].
 *   d must be a multiple of 4 (16-byte rows) and at most 4096; the BF16 tensor-core
 *   path additionally needs d % 8 == 0. Device feature matrices must start on a 16-byte
 *   boundary (every cudaMalloc or PyTorch allocation does; so does any row of one):
 *   a misaligned one is GCR_E_INVALID.
 * - Every call is asynchronous on the caller's stream (a cudaStream_t passed as
 *   gcr_stream_t; NULL is the legacy default stream) and returns a gcr_status code.
 *   Arguments are validated on the host before anything is launched; on a non-zero
 *   status nothing has been launched. CUDA errors raised by earlier asynchronous work
 *   surface as GCR_E_CUDA at a later call or at gcr_sync().
 * - A call that needs scratch memory takes (void* ws, size_t ws_bytes); the needed
 *   size comes from the matching *_workspace_size() query. Scratch contents need no
 *   initialisation and are meaningless after the call. Distinct workspaces make calls
 *   independent, so they may run concurrently on different streams.
 * - Nothing in this file synchronises the device except gcr_sync().
 *
 * Notation follows the paper: X (features), N_i (the k nearest neighbours of sample i,
 * i excluded), A~ (Eq. 4 affinity), D_r / D_c (Eq. 5 degrees), gamma (temperature),
 * alpha (Eq. 9 mix), lambda (Eq. 17 regularisation), T (iterations, Eq. 3).
 */
#ifndef GCR_H
#define GCR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* gcr_stream_t; /* a cudaStream_t */

typedef enum {
  GCR_OK = 0,
  GCR_E_INVALID = 1,     /* bad argument: null pointer, size or parameter out of range */
  GCR_E_WORKSPACE = 2,   /* ws_bytes below the *_workspace_size() requirement */
  GCR_E_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  GCR_E_TIMEOUT = 4,     /* a bounded device-side wait ran out (serving loop) */
  GCR_E_UNSUPPORTED = 5  /* shape or mode not supported by this build or device */
} gcr_status;

typedef enum {
  GCR_PREC_FP32 = 0, /* similarity GEMM on CUDA cores in FP32 (the reference path) */
  GCR_PREC_BF16 = 1, /* similarity GEMM on tcgen05 tensor cores, BF16 x BF16 -> FP32,
                        then boundary candidates re-scored in FP32 (FP64 for ties) */
  GCR_PREC_TF32 = 2  /* as BF16 with the rows rounded to TF32 (kind::tf32): a rounding
                        bound 8x tighter, so fewer candidates need the FP32 re-score.
                        Both tensor-core modes need d % 8 == 0 (BF16 also pool >= 64);
                        their certified re-score returns the neighbour sets of the exact
                        search */
} gcr_precision;

/* Hyper-parameters of one GCR run. gcr_default_params() fills the paper's defaults:
 * k = 15, gamma = 0.2, T = 3 (Sec. IV-B), alpha = 0.7 (Sec. IV-D). */
typedef struct {
  int32_t k;            /* neighbours per sample, |N_i| (Eq. 4); 0 <= k < pool          */
  float   gamma;        /* temperature of Eq. 4 / Eq. 8; > 0                             */
  float   alpha;        /* weight of the global graph in Eq. 9; in [0, 1]; used only
                           with cross_camera = 1                                          */
  int32_t symmetric;    /* 1: A = (A~ + A~^T)/2 and D^{-1/2} A D^{-1/2} (Eq. 7, Eq. 2);
                           0: D_r^{-1/2} A~ D_c^{-1/2} (Eq. 6)                            */
  int32_t cross_camera; /* 1: add the cross-camera graph (Eq. 8) and mix by Eq. 9         */
  int32_t precision;    /* gcr_precision                                                  */
  int32_t pool;         /* per-row candidate pool of the streaming kNN search: 32, 64 or
                           128; 0 picks the smallest of these that holds k plus a
                           margin of max(12, k/2) (32 for k <= 20), at least 64 under
                           BF16 (which needs >= 64);
                           must exceed k. A larger pool certifies more rows without the
                           threshold rescan at the cost of a busier GEMM epilogue.        */
  int32_t topk_out;     /* gcr_rerank: results per query; 0 = the whole gallery           */
  int32_t T;            /* iterations of Eq. 3, used by gcr_pipeline                      */
} gcr_params;

/* Counters written by gcr_build_graph (added to, never cleared by the library). */
enum {
  GCR_STAT_ROWS = 0,          /* (row, graph) pairs searched                               */
  GCR_STAT_UNCERTIFIED = 1,   /* pairs whose candidate pool could not certify the k-th
                                 neighbour: they go through the ball search (tensor-core
                                 modes of gcr_build_graph) and, where that does not
                                 certify them, the threshold (band) rescan               */
  GCR_STAT_BAND_FAILED = 2,   /* pairs whose band rescan found more than 512 columns
                                 within the certified margin of the k-th (a dense
                                 boundary the ball search did not take): they keep the
                                 pool's exact top k, whose exact scores are within
                                 2*delta of the exact k-th score (delta = the certified
                                 bound of the GEMM)                                       */
  GCR_STAT_FP64_ROWS = 3,     /* pairs whose k-th / (k+1)-th boundary needed FP64          */
  GCR_STAT_FP64_DOTS = 4,     /* FP64 dot products computed for those boundaries           */
  GCR_STAT_CLAMPED = 5,       /* pairs with fewer than k eligible samples                  */
  GCR_STAT_RESCORED = 6,      /* FP32 re-scored candidates                                 */
  GCR_STAT_SATURATED = 7,     /* searches against a gallery (gcr_rerank top-K, gcr_serve):
                                 uncertified pairs whose pool is saturated with near-ties
                                 (its lower half's density predicts more than 512 band
                                 entries), so the rescan is skipped; the same 2*delta
                                 guarantee as GCR_STAT_BAND_FAILED                        */
  GCR_STAT_BALL = 8,          /* uncertified pairs certified by the ball search: the exact
                                 search, in coordinates centred on a shared ball, of every
                                 sample that can be among their k nearest                 */
  GCR_STAT_BALL_PAIRS = 9,    /* uncertified pairs that took part in the ball search (it
                                 runs when a pair is predicted dense or 1,024 take part)  */
  GCR_STAT_BALL_GROUPS = 10,  /* balls searched                                            */
  GCR_STAT_BALL_ROWS = 11,    /* rows gathered into the searched balls                     */
  GCR_STATS_LEN = 12
};

/* The graph produced by gcr_build_graph and consumed by gcr_propagate. All arrays are
 * device arrays owned by the caller and sized by gcr_graph_op_capacity() and n, k.
 * Rows of nbr / nbr_cr list N_i (resp. N_i^cr) by ascending distance; a row with
 * fewer than k eligible samples is padded with index -1 and distance +inf.
 * The operator arrays hold, in CSR form, the matrix applied by one propagation layer:
 *   symmetric:  alpha * D^{-1/2} A D^{-1/2} + (1 - alpha) * (same for the cross graph)
 *   otherwise:  alpha * D_r^{-1/2} A~ D_c^{-1/2} + (1 - alpha) * (same for cross)
 * (alpha = 1 when cross_camera = 0). Row i occupies op_col/op_val[op_rowptr[i] ..
 * op_rowptr[i] + op_len[i]), sorted by column, one entry per column.              */
typedef struct {
  int32_t* nbr;       /* [n*k]  N_i (Eq. 4)                                        */
  float*   nbr_d2;    /* [n*k]  ||x_i - x_j||^2 of those edges                      */
  int32_t* nbr_cr;    /* [n*k]  N_i^cr (Eq. 8); may be NULL when cross_camera = 0   */
  float*   nbr_cr_d2; /* [n*k]  may be NULL when cross_camera = 0                   */
  float*   deg_r;     /* [n]    D_r of Eq. 5 (global graph)                         */
  float*   deg_c;     /* [n]    D_c of Eq. 5 (global graph)                         */
  float*   deg_r_cr;  /* [n]    D_r^cr (may be NULL when cross_camera = 0)          */
  float*   deg_c_cr;  /* [n]    D_c^cr (may be NULL when cross_camera = 0)          */
  int32_t* op_rowptr; /* [n+1]                                                      */
  int32_t* op_len;    /* [n]                                                        */
  int32_t* op_col;    /* [op_capacity]                                              */
  float*   op_val;    /* [op_capacity]                                              */
  int64_t* stats;     /* [GCR_STATS_LEN] device counters (may be NULL)              */
  int32_t* row_order; /* [n] optional (may be NULL): filled by gcr_build_graph with a
                         cluster-local order of the rows (rows sharing their nearest
                         candidates end up adjacent), used by gcr_propagate to walk the
                         rows in that order. Results do not depend on it.             */
} gcr_graph;

/* ------------------------------------------------------------------ utilities */
const char* gcr_status_string(int status);
int gcr_version(void);
/* Paper defaults (Sec. IV-B, IV-D): k=15, gamma=0.2, T=3, alpha=0.7, symmetric=1,
 * cross_camera=0, precision=FP32, pool=0, topk_out=0. Host pointer. */
void gcr_default_params(gcr_params* p);
/* 1 if `device` is an sm_103 GPU this library was built for, else 0. */
int gcr_device_supported(int device);
/* cudaStreamSynchronize(stream) and report any pending CUDA error; GCR_E_TIMEOUT if a
 * bounded device-side wait of a tensor-core kernel ran out since the last gcr_sync (that
 * kernel aborted and its outputs are incomplete). */
int gcr_sync(gcr_stream_t stream);

/* Failure-path self-test (no counterpart in the paper): launches one warp that waits, with
 * the same bounded wait the tensor-core kernels use, on a barrier that nothing signals. The
 * wait gives up after limit_us microseconds (1..1e6) and the kernel returns, so the next
 * gcr_sync on that stream reports GCR_E_TIMEOUT and the context stays usable. */
int gcr_selftest_wait_timeout(int64_t limit_us, gcr_stream_t stream);

/* ------------------------------------------------------------------ S0: normalise
 * X_out[i] = X_in[i] / ||X_in[i]||_2 (zero rows stay zero). The method works on unit
 * features: the profile derivation of Sec. III-D assumes ||x_i|| = 1, and each
 * propagation layer ends with the same normalisation. X_in may equal X_out. */
int gcr_normalize(const float* X_in, float* X_out, int64_t n, int32_t d, gcr_stream_t stream);

/* ------------------------------------------------------------------ S1-S4: graph
 * Builds, from the current features X (n x d, unit rows), the kNN graph of Eq. 4
 * (and of Eq. 8 when cross_camera = 1, with cam[i] the camera of sample i), its
 * degrees (Eq. 5) and the propagation operator (Eq. 6 or Eq. 7, mixed by Eq. 9).
 * The all-pairs similarity is streamed tile by tile and never stored. kNN sets are
 * exact: every candidate whose score lies within the certified error bound of the
 * k-th is re-scored in FP32 and, where FP32 cannot separate two candidates, in FP64;
 * exact FP64 ties go to the smaller index.
 * Part of the work (the cross-camera graph's transpose, the propagation's row order) runs
 * on helper streams that the call forks from `stream` and joins back into it by events
 * (one set per device, created on the first such call and kept): `stream` still orders
 * the whole call, and once a first call on the device has created them, later calls can
 * be captured in a CUDA graph (the fork and join become graph dependencies).
 * cam: device int32[n], required when cross_camera = 1, else may be NULL.
 * Errors: GCR_E_INVALID (n < 1, k out of range, gamma <= 0, alpha outside [0,1],
 * pool <= k, missing arrays), GCR_E_UNSUPPORTED (d % 4, d % 8 with BF16 or TF32,
 * pool 32 with BF16),
 * GCR_E_WORKSPACE. */
size_t gcr_graph_op_capacity(int64_t n, const gcr_params* p);
size_t gcr_build_graph_workspace_size(int64_t n, int32_t d, const gcr_params* p);
int gcr_build_graph(const float* X, int64_t n, int32_t d, const int32_t* cam,
                    const gcr_params* p, gcr_graph* g, void* ws, size_t ws_bytes,
                    gcr_stream_t stream);

/* ------------------------------------------------------------------ S5: propagate
 * One layer of Eq. 2 / Eq. 9 followed by the row L2 normalisation:
 *   X_out[i] = normalise( sum_j M_ij X_in[j] ),  M = the operator stored in g.
 * X_out must not alias X_in. No workspace. */
int gcr_propagate(const gcr_graph* g, const float* X_in, float* X_out, int64_t n,
                  int32_t d, gcr_stream_t stream);

/* ------------------------------------------------------------------ S7: re-rank
 * Re-ranked retrieval (Sec. III-A: retrieval uses the Euclidean distance of the
 * updated features): for each query q, the gallery sorted by ascending
 * ||x_q - x_g||^2, ties by gallery index. Writes idx_out[q*K + r] (gallery index of
 * rank r) and dist_out[q*K + r], K = topk_out (or ng when topk_out = 0).
 * precision = BF16 computes the distances on tensor cores from compensated operands
 * (x = bf16 hi + bf16 lo; one product of [hi|hi|lo] and [hi|lo|hi] over 3d terms), which
 * refines them to about 1e-5 of the FP64 distance on unit rows.
 * Errors: GCR_E_INVALID, GCR_E_UNSUPPORTED (K = ng above 16384), GCR_E_WORKSPACE. */
size_t gcr_rerank_workspace_size(int64_t nq, int64_t ng, int32_t d, const gcr_params* p);
int gcr_rerank(const float* Xq, int64_t nq, const float* Xg, int64_t ng, int32_t d,
               const gcr_params* p, int32_t* idx_out, float* dist_out, void* ws,
               size_t ws_bytes, gcr_stream_t stream);

/* gcr_rerank without a workspace argument, for callers that cannot allocate device
 * memory: for instance a serving process whose device-memory budget is fixed at start-up
 * and must not allocate per request (allocation can block, synchronise the device or fail
 * once memory is fragmented), or an application that embeds this library without giving
 * it an allocator. The paper has no counterpart; this is an interface convenience.
 * Same arguments, results and errors as gcr_rerank, except that the scratch lives in a
 * fixed device array of GCR_RERANK_NOALLOC_SCRATCH_BYTES compiled into the library. The
 * driver reserves that array on a device when it loads the library's device code there; with
 * CUDA's lazy module loading (the default) that happens during the first call of this entry
 * point with the device current, and it then stays reserved until the process exits. That
 * first call also looks up and caches the array's device address. So make the first call on
 * each device during start-up, before the process fixes its memory budget (a first call with
 * the device already full fails with GCR_E_CUDA) and before any stream capture. The cached
 * address holds until the device is reset (cudaDeviceReset or a new primary context); do not
 * call this entry point on a device after resetting it. The call returns GCR_E_WORKSPACE,
 * launching nothing, when gcr_rerank_workspace_size() of the problem exceeds the array (for
 * FP32 full rankings, roughly nq * ng <= 4 million). Every call shares the one array: calls
 * whose work overlaps on the GPU race and must be serialised by the caller. No call
 * allocates device memory itself. */
#define GCR_RERANK_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int gcr_rerank_noalloc(const float* Xq, int64_t nq, const float* Xg, int64_t ng, int32_t d,
                       const gcr_params* p, int32_t* idx_out, float* dist_out, gcr_stream_t stream);

/* ------------------------------------------------------------------ S0-S7 in one call
 * The whole offline re-ranking of Sec. III (Eq. 3 with T = p->T iterations):
 * X_0 = normalise(X), X_t = normalise(M_t X_{t-1}) with the graph rebuilt from X_{t-1}
 * each iteration, then gcr_rerank(X_T[0:nq], X_T[nq:n]). Queries are rows [0, nq).
 * X_final (may be NULL) receives X_T. stats (may be NULL) receives the counters of
 * every gcr_build_graph call. */
size_t gcr_pipeline_workspace_size(int64_t n, int64_t nq, int32_t d, const gcr_params* p);
int gcr_pipeline(const float* X, int64_t n, int64_t nq, int32_t d, const int32_t* cam,
                 const gcr_params* p, float* X_final, int32_t* idx_out, float* dist_out,
                 int64_t* stats, void* ws, size_t ws_bytes, gcr_stream_t stream);

/* The same re-ranking from and to host memory. X_host (float32 [n][d]) and cam_host
 * (int32 [n], when cross_camera = 1) are copied to the device on `stream`; the ranking
 * (idx_host int32 / dist_host float32, [nq][K] as in gcr_rerank) is copied back in up to 8
 * chunks of queries, each chunk as soon as it is sorted, on a second stream so that the
 * copies overlap the re-ranking of the later chunks; `stream` then waits for the last copy,
 * so a synchronisation of `stream` covers the whole call. Host buffers should be
 * page-locked (cudaHostAlloc / cudaHostRegister) for the copies to run asynchronously. The
 * copy stream and its events are created on the first call per device and kept until the
 * process exits; calls are serialised on them (a host mutex while enqueuing). stats: device
 * pointer or NULL. No counterpart in the paper (its implementation runs on the CPU). */
size_t gcr_pipeline_host_workspace_size(int64_t n, int64_t nq, int32_t d, const gcr_params* p);
int gcr_pipeline_host(const float* X_host, int64_t n, int64_t nq, int32_t d, const int32_t* cam_host,
                      const gcr_params* p, int32_t* idx_host, float* dist_host, int64_t* stats,
                      void* ws, size_t ws_bytes, gcr_stream_t stream);

/* ------------------------------------------------------------------ S8: GCRV profiles
 * Profile vectors of Sec. III-D for video re-ranking (Algorithm 2 step 1):
 *   mu_c = mean of tracklet c's L2-normalised frames                              (Eq. 10)
 *   w_c  = (X_s^T X_s + lambda n_s I)^{-1} (mu_c - mu_s)                           (Eq. 17)
 * X_s stacks the n_s normalised frames of every tracklet of c's camera s, mu_s is their
 * mean (the paper prints X X^T; only the d x d matrix X^T X is dimensionally consistent and
 * matches its "covariance matrix X^T X"). A camera with a single tracklet has mu_c = mu_s,
 * so that tracklet keeps mu_c. W_out (C x d) is not normalised; Algorithm 2 then runs GCR
 * with the global and the cross-camera graph on it (gcr_pipeline with cross_camera = 1 and
 * cam = trk_cam).
 * frames: device float32 [F][d], raw. trk_off: device int64 [C+1], tracklet c owns frames
 * [trk_off[c], trk_off[c+1]) (non-empty, ascending). trk_cam: device int32 [C] in
 * [0, n_cams), n_cams <= 64. The system is solved by conjugate gradients in FP32 with the
 * iteration count fixed by the bound cond <= 1 + 1/lambda (relative error ~1e-7).
 * Errors: GCR_E_INVALID (sizes, lambda <= 0), GCR_E_UNSUPPORTED (d % 4), GCR_E_WORKSPACE.
 * Tracklet offsets and cameras are trusted (not re-validated on the device). */
size_t gcrv_profiles_workspace_size(int64_t F, int32_t d, int32_t C, int32_t n_cams);
int gcrv_profiles(const float* frames, int64_t F, int32_t d, const int64_t* trk_off,
                  const int32_t* trk_cam, int32_t C, int32_t n_cams, float lambda, float* W_out,
                  void* ws, size_t ws_bytes, gcr_stream_t stream);

/* Eq. 10 alone: W_out[c] = the mean of tracklet c's L2-normalised frames (the "mean profile"
 * that Sec. IV's ablation compares with the Eq. 17 profile vectors). frames / trk_off / C as
 * for gcrv_profiles; W_out: device float32 [C][d], not normalised. Workspace: F floats.
 * Errors: GCR_E_INVALID, GCR_E_UNSUPPORTED (d % 4), GCR_E_WORKSPACE. */
size_t gcrv_mean_profiles_workspace_size(int64_t F, int32_t d, int32_t C);
int gcrv_mean_profiles(const float* frames, int64_t F, int32_t d, const int64_t* trk_off, int32_t C,
                       float* W_out, void* ws, size_t ws_bytes, gcr_stream_t stream);

/* ------------------------------------------------------------------ S9: serving
 * Re-ranking against a resident gallery. Sec. IV-F2 notes that with the gallery's graphs
 * computed and stored in advance the cost per query falls to O(N log N); this is that form:
 *  - gcr_gallery_build runs offline GCR (Eq. 3) on the gallery alone and stores, in the
 *    caller's state buffer (gcr_gallery_bytes), the layers G_0..G_T, the degrees of each
 *    layer's graph (D = (D_r + D_c)/2 of Eq. 7, or D_c of Eq. 6), per-row statistics and the
 *    kNN lists of the last layer's graph.
 *  - gcr_serve takes a batch of b raw queries (device float32 [b][d]) and, for t = 1..T,
 *    finds each query's certified k nearest rows of G_{t-1}, forms the query's row of the
 *    operator with the gallery frozen and no query-query edges
 *        symmetric:  y = x/D_q + sum_j (w_qj/2) g_j / sqrt(D_q D_j),  D_q = (2 + sum w)/2
 *        otherwise:  y = x/sqrt(r_q) + sum_j w_qj g_j / sqrt(r_q Dc_j), r_q = 1 + sum w
 *    (w_qj of Eq. 4) and normalises it; then it returns the certified top K = topk_out
 *    (1..127) of the gallery on G_T: idx_out int32 [b][K] by ascending squared distance
 *    (ties to the smaller index) and dist_out float [b][K] (FP32 re-scored distances).
 * In the tensor-core modes the searches give their column-split pools admission floors,
 * from the FP32 scores of the previous search's candidates (for the final search also of
 * their gallery neighbours) and, where those cannot supply enough rows, of an evenly spaced
 * sample of the gallery (the first search, for b >= 32, has only the sample; for b < 32 it
 * runs without a floor): provably below the approximate scores of at least k of the query's
 * gallery rows, so the splits skip most of the pool merging; the certification takes the
 * floor as the bound on every score it left out, and the results are the same certified
 * neighbours as without floors.
 * Every step is per query, so a query's result does not depend on its batch-mates. The
 * state is read-only during gcr_serve: concurrent calls with distinct workspaces may share
 * it. No host synchronisation: a call can be captured in a CUDA graph.
 * cross_camera must be 0 (GCR_E_UNSUPPORTED otherwise). stats: as gcr_graph.stats. */
size_t gcr_gallery_bytes(int64_t ng, int32_t d, const gcr_params* p);
size_t gcr_gallery_build_workspace_size(int64_t ng, int32_t d, const gcr_params* p);
int gcr_gallery_build(const float* Xg, int64_t ng, int32_t d, const gcr_params* p, void* state,
                      size_t state_bytes, void* ws, size_t ws_bytes, gcr_stream_t stream);
size_t gcr_serve_workspace_size(int64_t b, int64_t ng, int32_t d, const gcr_params* p);
int gcr_serve(const void* state, size_t state_bytes, int64_t ng, const float* Xq, int64_t b,
              int32_t d, const gcr_params* p, int32_t* idx_out, float* dist_out, int64_t* stats,
              void* ws, size_t ws_bytes, gcr_stream_t stream);

/* ------------------------------------------------------------------ DSFP (local propagation)
 * Decentralized and synchronous feature propagation, Algorithm 1 (Sec. III-B; "GCR_Local"
 * in Sec. IV-F): every image i is updated from its own local graph only. Its node set is
 * {i} u N_i (N_i its k nearest samples on the input features, i excluded, ties to the
 * smaller index, found by the same certified search as gcr_build_graph); over every pair
 * (u, v) of that set A_uv = exp(-||x_u - x_v||^2 / gamma) (A_uu = 1), D_u = sum_v A_uv, and
 * the (k+1) x d local features run T iterations of X <- normalise(D^{-1/2} A D^{-1/2} X).
 * Row i of X_out is i's own row after the T-th iteration (T = 0: the normalised input).
 * The local graph is built once, from the input (Algorithm 1 has no rebuild step), and the
 * rows are L2-normalised on input and after every iteration, as in the global method.
 *
 * gcr_dsfp: X device float32 [n][d], raw (normalised first). Uses p->k (0..64, < pool),
 * p->gamma, p->precision, p->pool and p->T; p->cross_camera must be 0 (Algorithm 1 is
 * stated for the plain graph); p->symmetric, alpha and topk_out are not used. X_out:
 * device float32 [n][d], must not alias X. nbr_out (may be NULL): device int32 [n][k]
 * receives N_i (-1 where fewer than k samples exist). stats: as gcr_graph.stats.
 * Errors: GCR_E_INVALID (null X / X_out, X_out == X, cross_camera = 1, T < 0, and every
 * gcr_build_graph parameter error), GCR_E_UNSUPPORTED (k > 64, d % 4, the precision rules of
 * gcr_build_graph), GCR_E_WORKSPACE.
 *
 * gcr_dsfp_propagate: the local propagation alone (no kNN search) on given neighbour lists.
 * X: device float32 [n][d], unit rows; nbr: device int32 [n][k], entries in [0, n) or < 0
 * (absent; skipped), trusted (not re-validated on the device); 0 <= k <= 64; gamma > 0;
 * T >= 0; X_out: device float32 [n][d], must not alias X. No workspace.
 * Errors: GCR_E_INVALID, GCR_E_UNSUPPORTED (k > 64, d % 4). */
size_t gcr_dsfp_workspace_size(int64_t n, int32_t d, const gcr_params* p);
int gcr_dsfp(const float* X, int64_t n, int32_t d, const gcr_params* p, float* X_out, int32_t* nbr_out,
             int64_t* stats, void* ws, size_t ws_bytes, gcr_stream_t stream);
int gcr_dsfp_propagate(const float* X, int64_t n, int32_t d, const int32_t* nbr, int32_t k, float gamma,
                       int32_t T, float* X_out, gcr_stream_t stream);

/* ------------------------------------------------------------------ retrieval quality
 * Average precision and first-hit position of ranked lists, from which the mAP and CMC
 * (Rank-k) of the paper's result tables follow, for evaluating re-ranking on labelled data
 * (an evaluation step, not part of the re-ranking). idx: device int32 [nq][K], gallery
 * indices by rank (entries < 0 are skipped, the others must be < ng; trusted). q_label [nq],
 * g_label [ng]: device int32, -1 marks a distractor (relevant to no query). q_cam [nq],
 * g_cam [ng]: device int32, required when protocol = 1, else may be NULL. A gallery item is
 * relevant to a query with the same label (>= 0); protocol 1 (the cross-camera protocol of
 * the re-identification benchmarks) first removes from the list every item with the query's
 * label and camera ("junk"); protocol 0 removes nothing. With the relevant items at 0-based
 * positions p_1 < ... < p_R of the list without junk and R counted over the whole gallery,
 * ap_out[q] = (1/R) sum_i i / (p_i + 1) (device double [nq]; items missing from a truncated
 * list count 0; NaN when R = 0 or the query is a distractor), first_out[q] = p_1 or -1
 * (device int32 [nq]). mAP = mean AP over the queries with R > 0, Rank-k = the fraction of
 * them with 0 <= first < k. Deterministic. No workspace.
 * Errors: GCR_E_INVALID (null arrays, sizes, protocol not 0 or 1, cameras missing). */
int gcr_eval_retrieval(const int32_t* idx, int64_t nq, int64_t K, const int32_t* q_label,
                       const int32_t* q_cam, const int32_t* g_label, const int32_t* g_cam, int64_t ng,
                       int32_t protocol, double* ap_out, int32_t* first_out, gcr_stream_t stream);

/* ------------------------------------------------------------------ stage profiler
 * Process-wide, for measurement only (not thread-safe). While enabled, every entry point
 * records a CUDA event pair on its stream around each stage below. gcr_profile_read()
 * waits for the recorded events, writes per stage the summed milliseconds, kernel launches
 * and timed calls (arrays of n_stages entries, host pointers) and clears the records.
 * At most 4096 stage records are kept between reads. */
enum {
  GCR_STAGE_NORMALIZE = 0, /* S0 row normalisation                         */
  GCR_STAGE_PREP = 1,      /* row norms, BF16 shadow, error bounds          */
  GCR_STAGE_SIM_GEMM = 2,  /* S1+S2 similarity GEMM fused with the top-k    */
  GCR_STAGE_REFINE = 3,    /* S3 certified refinement of the pools          */
  GCR_STAGE_BAND = 4,      /* S3 threshold rescan of uncertified rows       */
  GCR_STAGE_GRAPH = 5,     /* S4 weights, degrees, transpose, operator      */
  GCR_STAGE_PROPAGATE = 6, /* S5 propagation + L2 normalisation             */
  GCR_STAGE_DIST_GEMM = 7, /* S7 re-ranked distance GEMM                    */
  GCR_STAGE_SORT = 8,      /* S7 segmented sort                             */
  GCR_STAGE_GCRV = 9,      /* S8 GCRV profile vectors                       */
  GCR_STAGE_BALL = 10,     /* S3 ball search of the uncertified pairs       */
  GCR_STAGES = 12
};
int gcr_profile_enable(int on);
int gcr_profile_read(double* ms, int64_t* launches, int64_t* calls, int n_stages);

#ifdef __cplusplus
}
#endif
#endif /* GCR_H */
