// placeholder, replaced by the tcgen05 kernels
#include "common.cuh"
#include "kernels.h"
namespace gcr {
cudaError_t launch_umma_pool(const __nv_bfloat16*, int, int, const int*, bool, float*, int*, int*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_umma_band(const __nv_bfloat16*, int, int, const int*, const __nv_bfloat16*, const int*, int, const int*,
                             const int*, const float*, int, int*, float*, int*, int*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_umma_dist(const __nv_bfloat16*, int, const __nv_bfloat16*, int, int, const float*, const float*, float*, int*, cudaStream_t) { return cudaErrorNotSupported; }
}
