// Retrieval quality of ranked lists: average precision and first-hit position per query (the
// mAP and CMC / Rank-k of the paper's result tables), for evaluating re-ranking on labelled data.
//
// One warp per query. First the warp counts the relevant gallery items R (same label, label
// >= 0, and under protocol 1 not on the query's camera) over the whole gallery. Then it walks
// the ranked list 32 entries at a time: an entry is junk under protocol 1 when it has the
// query's label and camera (dropped from the list), relevant when it has the query's label.
// Ballots give each lane its position in the list without junk and the number of hits before
// it; every relevant lane adds (hits so far) / (position + 1) to its own FP64 sum, and one
// fixed-order warp reduction at the end gives AP = sum / R. FP64 here costs a few operations
// per relevant item only.
#include <math_constants.h>

#include "common.cuh"
#include "kernels.h"

namespace gcr {
namespace {

__global__ void __launch_bounds__(256) eval_kernel(const int32_t* __restrict__ idx, int nq, long K,
                                                   const int32_t* __restrict__ q_label,
                                                   const int32_t* __restrict__ q_cam,
                                                   const int32_t* __restrict__ g_label,
                                                   const int32_t* __restrict__ g_cam, int ng, int protocol,
                                                   double* __restrict__ ap_out, int32_t* __restrict__ first_out) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= nq) return;
  const int ql = q_label[q];
  const int qc = protocol == 1 ? q_cam[q] : 0;
  if (ql < 0) {
    if (lane == 0) {
      ap_out[q] = CUDART_NAN;
      first_out[q] = -1;
    }
    return;
  }
  int R = 0;
  for (int g = lane; g < ng; g += 32) {
    const bool junk = protocol == 1 && g_cam[g] == qc;
    R += (g_label[g] == ql && !junk) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) R += __shfl_xor_sync(GCR_FULL, R, o);
  if (R == 0) {
    if (lane == 0) {
      ap_out[q] = CUDART_NAN;
      first_out[q] = -1;
    }
    return;
  }
  const unsigned below = (1u << lane) - 1u;
  long pos = 0, hits = 0;
  int first = -1;
  double s = 0.0;
  const int32_t* row = idx + (size_t)q * K;
  for (long r0 = 0; r0 < K; r0 += 32) {
    const long r = r0 + lane;
    const int g = r < K ? row[r] : -1;
    bool keep = false, rel = false;
    if (g >= 0) {
      const bool same = g_label[g] == ql;
      const bool junk = protocol == 1 && same && g_cam[g] == qc;
      keep = !junk;
      rel = same && !junk;
    }
    const unsigned km = __ballot_sync(GCR_FULL, keep);
    const unsigned rm = __ballot_sync(GCR_FULL, rel);
    if (rel) {
      const long p = pos + __popc(km & below);   // position in the list without junk
      const long h = hits + __popc(rm & below) + 1;
      s += (double)h / (double)(p + 1);
    }
    if (first < 0 && rm) {
      const int l = __ffs(rm) - 1;
      first = (int)(pos + __popc(km & ((1u << l) - 1u)));
    }
    pos += __popc(km);
    hits += __popc(rm);
  }
  s = warp_sum_d(s);
  if (lane == 0) {
    ap_out[q] = s / (double)R;
    first_out[q] = first;
  }
}

}  // namespace

cudaError_t launch_eval(const int32_t* idx, int nq, long K, const int32_t* q_label, const int32_t* q_cam,
                        const int32_t* g_label, const int32_t* g_cam, int ng, int protocol, double* ap_out,
                        int32_t* first_out, cudaStream_t st) {
  const int wpb = 8;
  eval_kernel<<<(nq + wpb - 1) / wpb, wpb * 32, 0, st>>>(idx, nq, K, q_label, q_cam, g_label, g_cam, ng, protocol,
                                                         ap_out, first_out);
  return cudaGetLastError();
}

}  // namespace gcr
