"""gcr_rerank_noalloc: re-ranking with the library's fixed scratch array (GPU).

Some callers cannot allocate device memory during a call, e.g. a serving process whose
memory budget is fixed at start-up. gcr_rerank_noalloc serves them with scratch that is
compiled into the library. This test calls it through the C ABI twice in a row, on
different inputs, and checks each result against gcr_rerank (the entry point that takes a
caller-allocated workspace): identical rankings and distances within the FP32 tolerance of
the other re-ranking tests (1e-4). It also checks that a problem too large for the array is
refused with GCR_E_WORKSPACE before anything is launched. This file is collected last so
that, if it fails, a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    from paper_2306_08792_gb300 import build, _lib
    build.build()
    return _lib.load()


def _params(lib, **kw):
    from paper_2306_08792_gb300._lib import Params
    p = Params()
    lib.gcr_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _reference(lib, Xq, Xg, p, stream):
    nq, d = Xq.shape
    ng = Xg.shape[0]
    need = lib.gcr_rerank_workspace_size(nq, ng, d, ctypes.byref(p))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    K = p.topk_out or ng
    idx = torch.empty(nq, K, dtype=torch.int32, device="cuda")
    dist = torch.empty(nq, K, dtype=torch.float32, device="cuda")
    st = lib.gcr_rerank(_p(Xq), nq, _p(Xg), ng, d, ctypes.byref(p), _p(idx), _p(dist), _p(ws), need, stream)
    assert st == 0
    return idx, dist


def test_noalloc_matches_workspace_rerank_twice(lib):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = _params(lib, topk_out=0)
    for seed, (nq, ng, d) in ((0, (500, 2000, 256)), (1, (300, 1500, 128))):
        w = workloads.plain(seed=seed, n_query=nq, n_gallery=ng, d=d)
        X = torch.from_numpy(w.X).cuda()
        X = X / X.norm(dim=1, keepdim=True)
        Xq, Xg = X[:nq].contiguous(), X[nq:].contiguous()
        assert lib.gcr_rerank_workspace_size(nq, ng, d, ctypes.byref(p)) <= (16 << 20)
        idx = torch.full((nq, ng), -7, dtype=torch.int32, device="cuda")
        dist = torch.full((nq, ng), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.gcr_rerank_noalloc(_p(Xq), nq, _p(Xg), ng, d, ctypes.byref(p), _p(idx), _p(dist), stream)
        assert st == 0, lib.gcr_status_string(st)
        ridx, rdist = _reference(lib, Xq, Xg, p, stream)
        torch.cuda.synchronize()
        assert torch.equal(idx, ridx)
        assert float((dist - rdist).abs().max()) <= TOL
        assert np.all(np.diff(dist.cpu().numpy(), axis=1) >= 0)


def test_noalloc_topk_matches_workspace_rerank_twice(lib):
    """Top-K re-ranking (1 <= topk_out <= 127) goes through the certified pool search, whose
    scratch layout differs from the full ranking's; it too must match gcr_rerank."""
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = _params(lib, topk_out=20)
    for seed, (nq, ng, d) in ((2, (300, 1500, 128)), (3, (257, 1100, 64))):
        w = workloads.plain(seed=seed, n_query=nq, n_gallery=ng, d=d)
        X = torch.from_numpy(w.X).cuda()
        X = X / X.norm(dim=1, keepdim=True)
        Xq, Xg = X[:nq].contiguous(), X[nq:].contiguous()
        assert lib.gcr_rerank_workspace_size(nq, ng, d, ctypes.byref(p)) <= (16 << 20)
        idx = torch.full((nq, 20), -7, dtype=torch.int32, device="cuda")
        dist = torch.full((nq, 20), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.gcr_rerank_noalloc(_p(Xq), nq, _p(Xg), ng, d, ctypes.byref(p), _p(idx), _p(dist), stream)
        assert st == 0, lib.gcr_status_string(st)
        ridx, rdist = _reference(lib, Xq, Xg, p, stream)
        torch.cuda.synchronize()
        assert torch.equal(idx, ridx)
        assert float((dist - rdist).abs().max()) <= TOL
        assert np.all(np.diff(dist.cpu().numpy(), axis=1) >= 0)


def test_noalloc_refuses_problems_beyond_its_scratch(lib):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = _params(lib)
    nq, ng, d = 2000, 16000, 64               # 128 MB of distances: far beyond 16 MiB
    assert lib.gcr_rerank_workspace_size(nq, ng, d, ctypes.byref(p)) > (16 << 20)
    Xq = torch.zeros(nq, d, device="cuda")
    Xg = torch.zeros(ng, d, device="cuda")
    idx = torch.full((4,), 5, dtype=torch.int32, device="cuda")
    dist = torch.zeros(4, device="cuda")
    st = lib.gcr_rerank_noalloc(_p(Xq), nq, _p(Xg), ng, d, ctypes.byref(p), _p(idx), _p(dist), stream)
    assert st == 2                            # GCR_E_WORKSPACE, nothing launched
    torch.cuda.synchronize()
    assert torch.equal(idx, torch.full((4,), 5, dtype=torch.int32, device="cuda"))
