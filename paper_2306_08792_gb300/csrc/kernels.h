// Internal declarations shared by the GCR translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace gcr {

// Per-call scalars reduced over the rows of X (device memory).
struct RowScalars {
  double nmin, nmax;   // min / max of ||x_j||^2
  double bmax;         // max ||x_j||
  double emax;         // max ||bf16(x_j) - x_j||   (BF16 path)
  double amax;         // max ||bf16(x_j)||         (BF16 path)
};

// ---- prep.cu
cudaError_t launch_normalize(const float* X_in, float* X_out, int64_t n, int d, cudaStream_t st);
cudaError_t launch_row_stats(const float* X, int n, int d, double* n64, float* n32,
                             __nv_bfloat16* xb, float* enrm, float* anrm, RowScalars* sc,
                             cudaStream_t st);

// ---- sgemm.cu
size_t sgemm_pool_smem();
cudaError_t launch_sgemm_pool(const float* X, int n, int d, const int* cam, int kp, bool cross,
                              float* pool_v, int* pool_i, cudaStream_t st);
cudaError_t launch_sgemm_band(const float* X, int n, int d, const int* cam, const int* count,
                              int cap, const int* band_row, const int* band_kind, const float* band_thr,
                              int bcap, int* band_cnt, float* band_v, int* band_i, cudaStream_t st);
cudaError_t launch_sgemm_dist(const float* Xq, int nq, const float* Xg, int ng, int d,
                              const float* nrm_q, const float* nrm_g, float* D, cudaStream_t st);

// ---- umma.cu (tcgen05 BF16 path)
cudaError_t launch_umma_pool(const __nv_bfloat16* Xb, int n, int d, const int* cam, bool cross,
                             float* pool_v, int* pool_i, int* err_flag, cudaStream_t st);
cudaError_t launch_umma_band(const __nv_bfloat16* Xb, int n, int d, const int* cam,
                             const __nv_bfloat16* Ab, const int* count, int cap, const int* band_row,
                             const int* band_kind, const float* band_thr, int bcap, int* band_cnt,
                             float* band_v, int* band_i, int* err_flag, cudaStream_t st);
cudaError_t launch_umma_dist(const __nv_bfloat16* Qb, int nq, const __nv_bfloat16* Gb, int ng,
                             int d, const float* nrm_q, const float* nrm_g, float* D,
                             int* err_flag, cudaStream_t st);

// ---- refine.cu
struct RefineArgs {
  const float* X;
  int n, d, k, kinds;
  int precision;            // GCR_PREC_FP32 / GCR_PREC_BF16
  const double* n64;
  const float* enrm;
  const float* anrm;
  const RowScalars* sc;
  const float* pool_v;      // [kinds][n][kp]
  const int* pool_i;
  int kp;
  int32_t* nbr[2];
  float* d2[2];
  int* unc_count;           // uncertified (row, kind) pairs for the band rescan
  int* unc_row;
  int* unc_kind;
  float* unc_thr;
  unsigned long long* stats;
  // band rescan results
  const int* band_cnt;
  const float* band_v;
  const int* band_i;
  int bcap;
  int band_rows;            // capacity of the band buffers (rows beyond it are not rescanned)
};
cudaError_t launch_refine_pool(const RefineArgs& a, cudaStream_t st);
cudaError_t launch_refine_band(const RefineArgs& a, cudaStream_t st);
cudaError_t launch_gather_bf16(const __nv_bfloat16* Xb, int d, const int* count, const int* rows,
                               int max_rows, __nv_bfloat16* out, cudaStream_t st);

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
};
cudaError_t launch_build_operator(const GraphArgs& g, cudaStream_t st);

// ---- propagate.cu
cudaError_t launch_propagate(const int* rowptr, const int* len, const int* col, const float* val,
                             const float* X_in, float* X_out, int n, int d, cudaStream_t st);

// ---- sort.cu
cudaError_t launch_rank_rows(const float* D, int nq, int ng, int K, int32_t* idx_out,
                             float* dist_out, cudaStream_t st);

}  // namespace gcr
