"""GB300 (sm_103a) implementation of Graph Convolution based Re-ranking (GCR / GCRV).

The compute lives in ``libgcr.so`` (CUDA kernels behind the C ABI of ``include/gcr.h``);
this package is its thin Python binding.
"""
from .api import (Dsfp, GcrError, GraphTensors, HostPipeline, Pipeline, alloc_graph, default_params,  # noqa: F401
                  device_supported,
                  gcr_build_graph, gcr_dsfp, gcr_dsfp_propagate, gcr_eval_retrieval, gcr_normalize, gcr_pipeline,
                  gcr_propagate, gcr_rerank, gcr_rerank_noalloc, gcr_sync, gcrv_mean_profiles, gcrv_profiles,
                  retrieval_summary)
from ._lib import GCR_PREC_BF16, GCR_PREC_FP32, GCR_PREC_TF32, STAT_NAMES  # noqa: F401
