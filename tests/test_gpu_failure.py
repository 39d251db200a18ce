"""Failure path on the GPU without a fault: a bounded device wait that runs out.

gcr_selftest_wait_timeout makes one warp wait (with the tensor-core kernels' bounded wait) on
an mbarrier that nothing signals. The wait must give up after the given limit, gcr_sync must
report GCR_E_TIMEOUT exactly once, and the context must stay usable for real work.
"""
import ctypes
import time

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import paper_2306_08792_gb300 as gcr
    from paper_2306_08792_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.gcr_sync(stream) == 0
    t0 = time.perf_counter()
    assert lib.gcr_selftest_wait_timeout(20000, stream) == 0        # 20 ms
    assert lib.gcr_sync(stream) == _lib.GCR_E_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert lib.gcr_sync(stream) == 0                                  # reported once
    assert lib.gcr_selftest_wait_timeout(0, stream) == _lib.GCR_E_INVALID
    # the context still runs the tensor-core path correctly
    X, _ = workloads.random_unit_like(3, 300, 64)
    X0 = gcr.gcr_normalize(torch.from_numpy(X).cuda())
    G = gcr.gcr_build_graph(X0, gcr.default_params(k=5, precision="bf16"))
    assert lib.gcr_sync(stream) == 0
    nbr = G.nbr.cpu().numpy()
    assert np.all((nbr >= 0) & (nbr < 300)) and np.all(nbr != np.arange(300)[:, None])
