"""GPU parity tests for serving against a resident gallery (gcr_gallery_build / gcr_serve)
and for the continuous-batching loop.

Tolerances: gallery layers 1e-4 absolute (exact kNN sets, FP32 sums); the top-K sets must
equal the oracle's except certified ties (FP64 gap < 1e-9); returned distances are FP32
re-scored on both precisions, 1e-4 absolute. Staged: the oracle's query steps run on the
GPU's gallery layers and degrees (upcast to FP64).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

PRECISIONS = ["fp32", "bf16", "tf32"]


@pytest.fixture(scope="module")
def gcr():
    import paper_2306_08792_gb300 as g
    from paper_2306_08792_gb300 import build
    build.build()
    return g


def _gallery_host(G, p, ng, d):
    """Unpack the FP32 layers and degrees from the opaque state (leading regions of the buffer)."""
    raw = G.state
    T = p.T
    L = (T + 1) * ng * d * 4
    layers = raw[:L].view(torch.float32).reshape(T + 1, ng, d).double().cpu().numpy()
    off = (L + 255) // 256 * 256
    degs = raw[off:off + T * ng * 4].view(torch.float32).reshape(T, ng).double().cpu().numpy()
    return layers, degs


def _check_topk(layers_T, xq64, idx, dist, K):
    D = oracle.sq_dist(xq64, layers_T)
    bad = 0
    for i in range(idx.shape[0]):
        o = np.argsort(D[i], kind="stable")[:K]
        g = idx[i]
        if set(o) != set(g):
            dk = D[i, o[-1]]
            diff = np.array(sorted(set(o) ^ set(g)))
            if not np.all(np.abs(D[i, diff] - dk) < 1e-9):
                bad += 1
        np.testing.assert_allclose(dist[i], D[i, g], atol=1e-4, rtol=0)
        # ordered by the FP32 re-scored distance: inversions only below its error (~1e-6)
        assert np.all(np.diff(D[i, g]) >= -1e-5)
    return bad


@pytest.mark.parametrize("precision", PRECISIONS)
def test_serve_matches_oracle(gcr, precision):
    from paper_2306_08792_gb300.serving import Gallery
    w = workloads.serving(seed=1, n_gallery=3000, d=128, n_clusters=150, n_requests=8)
    p = gcr.default_params(k=10, T=2, topk_out=50, precision=precision)
    G = Gallery(torch.from_numpy(w.gallery).cuda(), p)
    layers, degs = _gallery_host(G, p, 3000, 128)
    # gallery layers agree with offline GCR of the oracle (exact kNN, FP32 sums)
    ref_layers, ref_degs = oracle.gallery_layers(w.gallery, 10, p.gamma, 2)
    assert np.max(np.abs(layers - np.stack(ref_layers))) < 1e-4
    np.testing.assert_allclose(degs, np.stack(ref_degs), rtol=1e-4)
    Q = np.concatenate([w.queries(r) for r in range(4)])
    idx, dist = G.query(torch.from_numpy(Q).cuda())
    torch.cuda.synchronize()
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    # staged: the oracle's query steps on the GPU's layers and degrees
    xq = oracle.l2_normalize(Q)
    for t in range(2):
        xq = oracle.serve_oracle._query_step(xq, layers[t], degs[t], 10, p.gamma, True)
    assert _check_topk(layers[2], xq, idx, dist, 50) == 0


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_serve_seeded_splits_match_oracle(gcr, precision):
    """A gallery wide enough for every split of the sweep to see many column tiles: every
    search runs with admission floors (short split pools), the first from a sample of the
    gallery, the final one from the last pool's rows, their gallery lists and the sample. The
    certified top-K must still be the oracle's, with no row clamped below k."""
    from paper_2306_08792_gb300.serving import Gallery
    ng, d, K = 60000, 256, 100
    w = workloads.serving(seed=3, n_gallery=ng, d=d, n_clusters=3000, n_requests=6)
    p = gcr.default_params(k=20, T=2, topk_out=K, precision=precision)
    G = Gallery(torch.from_numpy(w.gallery).cuda(), p)
    layers, degs = _gallery_host(G, p, ng, d)
    Q = w.queries_of(40)  # 32 or more: the first search is seeded from the gallery sample too
    Xq = torch.from_numpy(Q).cuda()
    import ctypes
    from paper_2306_08792_gb300 import _lib
    need = _lib.load().gcr_serve_workspace_size(Q.shape[0], ng, d, ctypes.byref(p))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    idx = torch.empty(Q.shape[0], K, dtype=torch.int32, device="cuda")
    dist = torch.empty(Q.shape[0], K, dtype=torch.float32, device="cuda")
    stats = torch.zeros(_lib.GCR_STATS_LEN, dtype=torch.int64, device="cuda")
    G.serve(Xq, idx, dist, ws, stats)
    torch.cuda.synchronize()
    assert int(stats[5]) == 0  # GCR_STAT_CLAMPED
    xq = oracle.l2_normalize(Q)
    for t in range(2):
        xq = oracle.serve_oracle._query_step(xq, layers[t], degs[t], 20, p.gamma, True)
    assert _check_topk(layers[2], xq, idx.cpu().numpy(), dist.cpu().numpy(), K) == 0


@pytest.mark.parametrize("precision", PRECISIONS)
def test_serve_result_is_the_same_alone_and_in_the_mix(gcr, precision):
    from paper_2306_08792_gb300.serving import Gallery
    w = workloads.serving(seed=2, n_gallery=5000, d=256, n_clusters=300, n_requests=6)
    p = gcr.default_params(k=20, T=2, topk_out=100, precision=precision)
    G = Gallery(torch.from_numpy(w.gallery).cuda(), p)
    parts = [w.queries(r)[:7] for r in range(5)]
    mix_idx, mix_dist = G.query(torch.from_numpy(np.concatenate(parts)).cuda())
    mix_idx, mix_dist = mix_idx.cpu().numpy(), mix_dist.cpu().numpy()
    o = 0
    for part in parts:
        a_idx, a_dist = G.query(torch.from_numpy(part).cuda())
        b = part.shape[0]
        assert np.array_equal(a_idx.cpu().numpy(), mix_idx[o:o + b])
        np.testing.assert_allclose(a_dist.cpu().numpy(), mix_dist[o:o + b], atol=1e-6, rtol=0)
        o += b


def test_serving_loop_continuous_batching(gcr):
    from paper_2306_08792_gb300.serving import Gallery, Server, make_requests
    w = workloads.serving(seed=3, n_gallery=20000, d=256, n_clusters=1000, n_requests=60, rate=400.0, max_batch=64)
    p = gcr.default_params(k=20, T=2, topk_out=100, precision="bf16")
    G = Gallery(torch.from_numpy(w.gallery).cuda(), p)
    srv = Server(G, n_slots=3, max_batch=128)
    srv.warmup(sizes=(1, 2, 4, 8, 16, 32, 64, 128))
    reqs = make_requests(w, 60)
    res = srv.run(reqs)
    assert res["requests"] == 60 and res["p99_ms"] >= res["p50_ms"] > 0
    # every request's result equals a direct call on its queries alone
    for r in reqs[:12]:
        i, d = G.query(torch.from_numpy(r.queries).cuda())
        assert np.array_equal(i.cpu().numpy(), r.idx)
        np.testing.assert_allclose(d.cpu().numpy(), r.dist, atol=1e-6, rtol=0)


def test_serving_loop_memory_budget_binds(gcr):
    """A memory budget below what the slots could hold at once (4 slots, room for one full batch
    and a little more): requests whose batch would exceed it wait in the queue, are admitted as
    in-flight batches complete and free their workspace, the admitted footprint never exceeds the
    budget, and every result equals a direct call on the request's queries alone."""
    from paper_2306_08792_gb300.serving import Gallery, Server, make_requests, _bucket
    w = workloads.serving(seed=5, n_gallery=20000, d=256, n_clusters=1000, n_requests=48, rate=2000.0,
                          max_batch=64)
    p = gcr.default_params(k=20, T=2, topk_out=100, precision="tf32")
    G = Gallery(torch.from_numpy(w.gallery).cuda(), p)
    probe = Server(G, n_slots=1, max_batch=64)
    full = probe.ws_of(64)
    budget = full + probe.ws_of(8)
    del probe
    srv = Server(G, n_slots=4, max_batch=64, budget_bytes=budget)
    assert srv.budget == budget < 4 * full
    srv.warmup(sizes=(1, 2, 4, 8, 16, 32, 64))
    reqs = make_requests(w, 48, realtime=False)     # all waiting at once: the budget decides
    res = srv.run(reqs, realtime=False)
    assert res["requests"] == 48
    assert res["memory_waits"] > 0, res
    assert 0 < res["max_in_flight_bytes"] <= budget, res
    for r in reqs:
        assert r.done > 0 and srv.ws_of(_bucket(r.queries.shape[0])) <= budget
    for r in reqs[::4]:
        i, d = G.query(torch.from_numpy(r.queries).cuda())
        assert np.array_equal(i.cpu().numpy(), r.idx)
        np.testing.assert_allclose(d.cpu().numpy(), r.dist, atol=1e-6, rtol=0)


def test_serve_rejects_cross_camera_and_bad_topk(gcr):
    from paper_2306_08792_gb300 import _lib
    import ctypes
    lib = _lib.load()
    p = gcr.default_params(k=10, T=2, topk_out=50, cross_camera=1)
    assert lib.gcr_gallery_bytes(1000, 64, ctypes.byref(p)) == 0
    p = gcr.default_params(k=10, T=2, topk_out=200)
    assert lib.gcr_gallery_bytes(1000, 64, ctypes.byref(p)) == 0
