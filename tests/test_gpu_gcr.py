"""GPU parity tests: the CUDA path (through the C ABI) against the FP64 oracle.

Staged comparisons feed the oracle the GPU's own previous-stage output (upcast to FP64),
so near-ties created upstream are not blamed downstream. Tolerances:
  * kNN sets: identical except certified ties (oracle FP64 gap < 1e-9);
  * normalisation: 2 ulp of FP32 (the kernel scales in FP64);
  * operator entries, degrees: 1e-6 relative (FP32 weights of FP64-resolved edges);
  * one propagation layer: 2e-6 absolute on unit rows (FP32 sums of <= 4k+1 terms);
  * re-ranked distances: 1e-4 absolute (FP32 path), 2e-3 (BF16 tensor-core path; the kNN
    sets stay exact on both paths).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests import parity

pytestmark = pytest.mark.gpu

PRECISIONS = ["fp32", "bf16", "tf32"]
# the tensor-core modes share the compensated BF16 distance GEMM
DIST_TOL = {"fp32": 1e-4, "bf16": 2e-3, "tf32": 2e-3}


@pytest.fixture(scope="module")
def gcr():
    import paper_2306_08792_gb300 as g
    from paper_2306_08792_gb300 import build
    build.build()
    assert g.device_supported(0), "this library targets sm_103 GPUs"
    return g


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _graph_host(G):
    out = {}
    for f in ("nbr", "nbr_d2", "nbr_cr", "nbr_cr_d2", "deg_r", "deg_c", "deg_r_cr", "deg_c_cr",
              "op_rowptr", "op_len", "op_col", "op_val"):
        v = getattr(G, f)
        out[f] = v.cpu().numpy() if v is not None else None
    return out


def test_normalize_matches_fp64(gcr):
    X, _ = workloads.random_unit_like(0, 777, 260)
    X[5] = 0.0                                            # a zero row stays zero
    Y = gcr.gcr_normalize(_dev(X)).cpu().numpy()
    ref = oracle.l2_normalize(X)
    np.testing.assert_allclose(Y, ref, rtol=0, atol=2 * np.finfo(np.float32).eps)
    assert np.all(Y[5] == 0)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_knn_plain_workload(gcr, precision):
    w = workloads.plain()
    X0 = gcr.gcr_normalize(_dev(w.X))
    p = gcr.default_params(k=w.k, precision=precision)
    G = gcr.gcr_build_graph(X0, p)
    torch.cuda.synchronize()
    X64 = X0.double().cpu().numpy()
    r = parity.compare_knn(X64, np.arange(w.n), G.nbr.cpu().numpy(), w.k)
    assert r["mismatched"] == 0, r
    st = G.stats_dict()
    assert st["rows"] == w.n and st["band_failed"] == 0


@pytest.mark.parametrize("precision,pool", [(p, 0) for p in PRECISIONS] + [("tf32", 64)])
def test_knn_cross_camera(gcr, precision, pool):
    w = workloads.crosscam(seed=3, n_query=400, n_gallery=2600, d=256, n_clusters=120)
    X0 = gcr.gcr_normalize(_dev(w.X))
    cam = _dev(w.cam, torch.int32)
    p = gcr.default_params(k=w.k, cross_camera=1, alpha=0.7, precision=precision, pool=pool)
    G = gcr.gcr_build_graph(X0, p, cam)
    torch.cuda.synchronize()
    X64 = X0.double().cpu().numpy()
    r = parity.compare_knn(X64, np.arange(w.n), G.nbr.cpu().numpy(), w.k)
    assert r["mismatched"] == 0, r
    rc = parity.compare_knn(X64, np.arange(w.n), G.nbr_cr.cpu().numpy(), w.k, w.cam, cross=True)
    assert rc["mismatched"] == 0, rc
    nc = G.nbr_cr.cpu().numpy()
    assert np.all(w.cam[nc] != w.cam[:, None])


def test_knn_paired_splits_all_rows(gcr):
    """TF32 with 32-entry pools at a size where one 128-row block of d = 2048 per SM would not fit
    in half the L2 (8,900 rows: 70 row blocks, 73 MB), so two CTAs sweep the two column halves of
    each block (35 column tiles: 18 + 17, a ragged last tile and a ragged last row block) and
    merge their pools; every row's global and cross-camera kNN sets against the FP64 oracle."""
    w = workloads.crosscam(seed=21, n_query=900, n_gallery=8000, d=2048, n_clusters=350)
    X0 = gcr.gcr_normalize(_dev(w.X))
    cam = _dev(w.cam, torch.int32)
    p = gcr.default_params(k=w.k, cross_camera=1, alpha=0.7, precision="tf32")
    G = gcr.gcr_build_graph(X0, p, cam)
    torch.cuda.synchronize()
    X64 = X0.double().cpu().numpy()
    r = parity.compare_knn(X64, np.arange(w.n), G.nbr.cpu().numpy(), w.k)
    rc = parity.compare_knn(X64, np.arange(w.n), G.nbr_cr.cpu().numpy(), w.k, w.cam, cross=True)
    assert r["mismatched"] == 0 and rc["mismatched"] == 0, (r, rc)
    assert G.stats_dict()["band_failed"] == 0


@pytest.mark.parametrize("precision", ["fp32", "tf32"])
def test_build_graph_captured_in_cuda_graph(gcr, precision):
    """gcr_build_graph forks helper streams (the cross-camera graph's transpose, the row order)
    from the caller's stream and joins them back: after a first call has created them, a call
    can be captured in a CUDA graph, and a replay gives the direct call's graph."""
    import ctypes
    from paper_2306_08792_gb300 import _lib
    w = workloads.crosscam(seed=9, n_query=200, n_gallery=1300, d=128, n_clusters=70)
    X0 = gcr.gcr_normalize(_dev(w.X))
    cam = _dev(w.cam, torch.int32)
    p = gcr.default_params(k=w.k, cross_camera=1, alpha=0.7, precision=precision)
    ref = gcr.gcr_build_graph(X0, p, cam)
    torch.cuda.synchronize()
    need = _lib.load().gcr_build_graph_workspace_size(w.n, X0.shape[1], ctypes.byref(p))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    g = gcr.alloc_graph(w.n, p, X0.device)
    gcr.gcr_build_graph(X0, p, cam, graph=g, ws=ws)
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        gcr.gcr_build_graph(X0, p, cam, graph=g, ws=ws)
    for t in (g.nbr, g.nbr_cr, g.op_rowptr, g.op_len, g.row_order):
        t.fill_(-7)
    cg.replay()
    torch.cuda.synchronize()
    for name in ("nbr", "nbr_d2", "nbr_cr", "nbr_cr_d2", "deg_r", "deg_c", "op_rowptr", "op_len"):
        assert torch.equal(getattr(g, name), getattr(ref, name)), name
    # the row order only schedules the propagation: any permutation of the rows is valid
    assert np.array_equal(np.sort(g.row_order.cpu().numpy()), np.arange(w.n))
    rp, ln = ref.op_rowptr.cpu().numpy(), ref.op_len.cpu().numpy()
    col_r, val_r = ref.op_col.cpu().numpy(), ref.op_val.cpu().numpy()
    col_g, val_g = g.op_col.cpu().numpy(), g.op_val.cpu().numpy()
    for i in range(w.n):
        s0, s1 = rp[i], rp[i] + ln[i]
        assert np.array_equal(col_g[s0:s1], col_r[s0:s1]) and np.array_equal(val_g[s0:s1], val_r[s0:s1]), i


EDGE = [("fp32", 1, 8, 5), ("fp32", 5, 12, 10), ("fp32", 130, 68, 7), ("fp32", 300, 256, 0),
        ("fp32", 257, 36, 31), ("bf16", 1, 8, 5), ("bf16", 5, 16, 10), ("bf16", 130, 72, 7),
        ("bf16", 300, 256, 0), ("bf16", 257, 40, 31), ("bf16", 600, 200, 63), ("tf32", 1, 8, 5),
        ("tf32", 129, 24, 10), ("tf32", 130, 72, 7), ("tf32", 300, 256, 0), ("tf32", 257, 40, 31),
        ("tf32", 600, 200, 63)]


@pytest.mark.parametrize("precision,n,d,k", EDGE)
def test_knn_edge_shapes(gcr, precision, n, d, k):
    X, cam = workloads.random_unit_like(n, n, d, cams=3)
    X0 = gcr.gcr_normalize(_dev(X))
    p = gcr.default_params(k=k, cross_camera=1, alpha=0.5, precision=precision)
    if k >= 32 or precision != "fp32":
        p.pool = 64
    G = gcr.gcr_build_graph(X0, p, _dev(cam, torch.int32))
    torch.cuda.synchronize()
    X64 = X0.double().cpu().numpy()
    if k > 0:
        for nbr, cross in ((G.nbr, False), (G.nbr_cr, True)):
            r = parity.compare_knn(X64, np.arange(n), nbr.cpu().numpy(), k, cam, cross)
            assert r["mismatched"] == 0, (cross, r)
    # propagation through this graph matches the oracle's operator on the same sets
    g_o = oracle.build_graph(X64, k, p.gamma, cam, True, True, 0.5,
                             nbr=G.nbr.cpu().numpy(), nbr_cr=G.nbr_cr.cpu().numpy())
    Y = gcr.gcr_propagate(G, X0).cpu().numpy()
    np.testing.assert_allclose(Y, oracle.propagate(X64, g_o["M"]), atol=2e-6, rtol=0)


@pytest.mark.parametrize("precision", ["fp32", "tf32"])
def test_hub_row_transpose_and_propagation(gcr, precision):
    """A hub: one centre row is the nearest neighbour of almost every other row, so its
    transposed segment and its operator row hold thousands of entries (the long-segment sort
    and the block-per-row propagation). Degrees, operator and propagation of every row match
    the oracle; two runs are bit-identical."""
    rng = np.random.default_rng(7)
    n, d, k = 3000, 64, 5
    c = rng.standard_normal(d)
    c /= np.linalg.norm(c)
    X = c[None, :] + 0.55 * rng.standard_normal((n, d)) / np.sqrt(d)
    X[0] = c
    X0 = gcr.gcr_normalize(_dev(X.astype(np.float32)))
    p = gcr.default_params(k=k, precision=precision)
    if precision != "fp32":
        p.pool = 64
    G = gcr.gcr_build_graph(X0, p)
    Y = gcr.gcr_propagate(G, X0)
    G2 = gcr.gcr_build_graph(X0, p)
    Y2 = gcr.gcr_propagate(G2, X0)
    torch.cuda.synchronize()
    L = G.op_len.cpu().numpy()
    assert L.max() > 1024, L.max()          # the hub's row takes the long-row path
    assert torch.equal(Y, Y2) and torch.equal(G.deg_c, G2.deg_c)
    rp, ln = G.op_rowptr.cpu().numpy(), G.op_len.cpu().numpy()
    valid = np.concatenate([np.arange(rp[i], rp[i] + ln[i]) for i in range(n)])  # past len: unwritten
    assert np.array_equal(G.op_col.cpu().numpy()[valid], G2.op_col.cpu().numpy()[valid])
    assert np.array_equal(G.op_val.cpu().numpy()[valid], G2.op_val.cpu().numpy()[valid])
    X64 = X0.double().cpu().numpy()
    nbr = G.nbr.cpu().numpy()
    r = parity.compare_knn(X64, np.arange(n), nbr, k)
    assert r["mismatched"] == 0, r
    g_o = oracle.build_graph(X64, k, p.gamma, nbr=nbr)
    np.testing.assert_allclose(G.deg_c.cpu().numpy(), oracle.degrees(g_o["At"])[1], rtol=2e-6)
    np.testing.assert_allclose(Y.cpu().numpy(), oracle.propagate(X64, g_o["M"]), atol=2e-6, rtol=0)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_knn_exact_duplicates_and_ties(gcr, precision):
    """Duplicated rows tie exactly: only certified-tie swaps are allowed."""
    rng = np.random.default_rng(5)
    base = rng.standard_normal((60, 32)).astype(np.float32)
    X = np.concatenate([base, base[:20], base[:20]], axis=0)
    X0 = gcr.gcr_normalize(_dev(X))
    p = gcr.default_params(k=6, precision=precision)
    G = gcr.gcr_build_graph(X0, p)
    torch.cuda.synchronize()
    r = parity.compare_knn(X0.double().cpu().numpy(), np.arange(100), G.nbr.cpu().numpy(), 6)
    assert r["mismatched"] == 0, r


@pytest.mark.parametrize("symmetric", [1, 0])
@pytest.mark.parametrize("cross", [0, 1])
def test_operator_and_degrees_match_oracle(gcr, symmetric, cross):
    w = workloads.crosscam(seed=7, n_query=200, n_gallery=1100, d=128, n_clusters=60)
    X0 = gcr.gcr_normalize(_dev(w.X))
    p = gcr.default_params(k=12, symmetric=symmetric, cross_camera=cross, alpha=0.7)
    G = gcr.gcr_build_graph(X0, p, _dev(w.cam, torch.int32) if cross else None)
    torch.cuda.synchronize()
    h = _graph_host(G)
    X64 = X0.double().cpu().numpy()
    g_o = oracle.build_graph(X64, 12, p.gamma, w.cam, bool(cross), bool(symmetric), 0.7,
                             nbr=h["nbr"], nbr_cr=h["nbr_cr"] if cross else None)
    Dr, Dc = oracle.degrees(g_o["At"])
    np.testing.assert_allclose(h["deg_r"], Dr, rtol=1e-6)
    np.testing.assert_allclose(h["deg_c"], Dc, rtol=1e-6)
    # edge distances are FP32 roundings of FP64-resolved ones
    np.testing.assert_allclose(h["nbr_d2"], g_o["d2"], rtol=0, atol=2e-6)
    M = parity.dense_from_csr(h["op_rowptr"], h["op_len"], h["op_col"], h["op_val"], w.n)
    Mo = g_o["M"].toarray()
    np.testing.assert_allclose(M, Mo, rtol=0, atol=1e-6 * np.abs(Mo).max())
    # each operator row is sorted by column with no duplicates
    for i in range(0, w.n, 97):
        cols = h["op_col"][h["op_rowptr"][i]:h["op_rowptr"][i] + h["op_len"][i]]
        assert np.all(np.diff(cols) > 0)
    if symmetric and not cross:
        np.testing.assert_allclose(M, M.T, atol=1e-7)


def test_propagate_matches_oracle(gcr):
    w = workloads.plain(seed=2)
    X0 = gcr.gcr_normalize(_dev(w.X))
    p = gcr.default_params(k=w.k)
    G = gcr.gcr_build_graph(X0, p)
    X1 = gcr.gcr_propagate(G, X0)
    torch.cuda.synchronize()
    X64 = X0.double().cpu().numpy()
    g_o = oracle.build_graph(X64, w.k, p.gamma, nbr=G.nbr.cpu().numpy())
    ref = oracle.propagate(X64, g_o["M"])
    np.testing.assert_allclose(X1.cpu().numpy(), ref, atol=2e-6, rtol=0)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("topk", [0, 37])
def test_rerank_matches_oracle(gcr, precision, topk):
    w = workloads.plain(seed=4)
    X0 = gcr.gcr_normalize(_dev(w.X))
    p = gcr.default_params(topk_out=topk, precision=precision)
    idx, dist = gcr.gcr_rerank(X0[:w.n_query].contiguous(), X0[w.n_query:].contiguous(), p)
    torch.cuda.synchronize()
    X64 = X0.double().cpu().numpy()
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    K = topk or (w.n - w.n_query)
    assert idx.shape == (w.n_query, K)
    err, viol = parity.ranking_errors(X64[:w.n_query], X64[w.n_query:], idx, dist)
    tol = DIST_TOL[precision]
    assert err < tol and viol < 2 * tol, (err, viol)
    if topk == 0:
        assert np.all(np.sort(idx, axis=1) == np.arange(K)[None, :])
    # ranks agree with the oracle's where the oracle's distances are separated by > 2 tol
    o_idx, o_d = oracle.rerank(X64[:w.n_query], X64[w.n_query:], topk)
    sep = np.ones_like(o_d, dtype=bool)
    sep[:, 1:] &= np.diff(o_d, axis=1) > 2 * tol
    sep[:, :-1] &= np.diff(o_d, axis=1) > 2 * tol
    assert np.all(idx[sep] == o_idx[sep])


@pytest.mark.parametrize("ng", [2047, 2048, 3001, 4096, 4100, 8193, 16384])
def test_rerank_sort_sizes_and_ties(gcr, ng):
    """The full ranking across the sort's size classes (bitonic below 2048 keys, radix at and
    above), with exact duplicates in the gallery: the returned distances are non-decreasing,
    equal distances come in increasing gallery index, every gallery row appears once, and the
    distances match FP64 within the FP32 bound."""
    rng = np.random.default_rng(ng)
    d, nq = 64, 9
    G = rng.standard_normal((ng, d)).astype(np.float32)
    dup = rng.choice(ng, ng // 5, replace=False)
    G[dup] = G[rng.integers(0, ng, dup.size)]          # exact ties between gallery rows
    Q = rng.standard_normal((nq, d)).astype(np.float32)
    Q[0] = G[3]                                          # a query equal to a gallery row
    Xq = gcr.gcr_normalize(_dev(Q))
    Xg = gcr.gcr_normalize(_dev(G))
    idx, dist = gcr.gcr_rerank(Xq, Xg, gcr.default_params(topk_out=0))
    torch.cuda.synchronize()
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    assert np.all(np.sort(idx, axis=1) == np.arange(ng)[None, :])
    step = np.diff(dist, axis=1)
    assert np.all(step >= 0)
    assert np.all(np.diff(idx, axis=1)[step == 0] > 0)
    err, _ = parity.ranking_errors(Xq.double().cpu().numpy(), Xg.double().cpu().numpy(), idx, dist)
    assert err < DIST_TOL["fp32"]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_pipeline_end_to_end_plain(gcr, precision):
    """Whole GCR (normalise, T layers, re-rank) vs the oracle run from the same raw input.
    The kNN sets are exact on both paths, so X_T agrees to FP32 rounding; the re-ranked
    distances carry the distance GEMM's error (FP32 or BF16)."""
    w = workloads.plain(seed=1)
    p = gcr.default_params(k=w.k, T=w.T, precision=precision)
    idx, dist, XT, st = gcr.gcr_pipeline(_dev(w.X), w.n_query, p)
    torch.cuda.synchronize()
    Xo = oracle.gcr(w.X, w.k, p.gamma, w.T)
    err_x = float(np.max(np.abs(XT.cpu().numpy() - Xo)))
    assert err_x < 1e-4, err_x
    err, viol = parity.ranking_errors(Xo[:w.n_query], Xo[w.n_query:], idx.cpu().numpy(), dist.cpu().numpy())
    tol = DIST_TOL[precision]
    assert err < tol and viol < 2 * tol, (err, viol)
    assert st["band_failed"] == 0


@pytest.mark.parametrize("precision", ["fp32", "tf32"])
@pytest.mark.parametrize("topk", [0, 20])
def test_pipeline_host_buffers_match_device(gcr, precision, topk):
    """gcr_pipeline_host (host inputs, ranking copied back in query chunks on a second stream)
    returns exactly the ranking of gcr_pipeline on device buffers."""
    w = workloads.crosscam(seed=5, n_query=1100, n_gallery=2500, d=256, n_clusters=150)
    p = gcr.default_params(k=w.k, T=2, cross_camera=1, alpha=0.7, precision=precision, topk_out=topk)
    dev = gcr.Pipeline(w.n, w.n_query, w.d, p)
    idx_d, dist_d = dev(_dev(w.X), _dev(w.cam, torch.int32), keep_features=False)
    hp = gcr.HostPipeline(w.n, w.n_query, w.d, p)
    Xh = torch.from_numpy(w.X).pin_memory()
    camh = torch.from_numpy(w.cam.astype(np.int32)).pin_memory()
    for _ in range(2):  # twice: the copy stream and its events are reused
        hp.idx.fill_(-7)
        idx_h, dist_h = hp(Xh, camh)
        torch.cuda.synchronize()
        assert np.array_equal(idx_h.numpy(), idx_d.cpu().numpy())
        assert np.array_equal(dist_h.numpy(), dist_d.cpu().numpy())


@pytest.mark.parametrize("precision", PRECISIONS)
def test_pipeline_determinism(gcr, precision):
    w = workloads.crosscam(seed=11, n_query=300, n_gallery=1700, d=192, n_clusters=80)
    p = gcr.default_params(k=w.k, T=2, cross_camera=1, alpha=0.7, precision=precision)
    pl = gcr.Pipeline(w.n, w.n_query, w.d, p)
    X, cam = _dev(w.X), _dev(w.cam, torch.int32)
    a = [t.clone() for t in pl(X, cam)] + [pl.X_final.clone()]
    b = [t.clone() for t in pl(X, cam)] + [pl.X_final.clone()]
    for u, v in zip(a, b):
        assert torch.equal(u, v)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_full_size_crosscam_sampled(gcr, precision):
    """Market-1501-shaped workload (3,368 + 15,913, d = 2048, 6 cameras) at full size, in the
    launch configuration the benchmark times; kNN sets, operator and propagation are checked on
    a seeded sample of rows, the re-ranking on a sample of queries."""
    w = workloads.crosscam()
    p = gcr.default_params(k=w.k, T=w.T, cross_camera=1, alpha=w.alpha, precision=precision)
    X0 = gcr.gcr_normalize(_dev(w.X))
    cam = _dev(w.cam, torch.int32)
    G = gcr.gcr_build_graph(X0, p, cam)
    X1 = gcr.gcr_propagate(G, X0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(w.n, 160, replace=False))
    X64 = X0.double().cpu().numpy()
    nbr, nbrc = G.nbr.cpu().numpy(), G.nbr_cr.cpu().numpy()
    r = parity.compare_knn(X64, rows, nbr[rows], w.k)
    rc = parity.compare_knn(X64, rows, nbrc[rows], w.k, w.cam, cross=True)
    assert r["mismatched"] == 0 and rc["mismatched"] == 0, (r, rc)
    # propagation of sampled rows from the full GPU graph, operator rebuilt by the oracle
    g_o = oracle.build_graph(X64, w.k, p.gamma, w.cam, True, True, w.alpha, nbr=nbr, nbr_cr=nbrc)
    ref = oracle.propagate(X64, g_o["M"][rows])
    np.testing.assert_allclose(X1.cpu().numpy()[rows], ref, atol=2e-6, rtol=0)
    # whole pipeline: ranking of sampled queries against the oracle's distances on X_T
    idx, dist, XT, st = gcr.gcr_pipeline(_dev(w.X), w.n_query, p, cam)
    torch.cuda.synchronize()
    XT64 = XT.double().cpu().numpy()
    q = np.sort(rng.choice(w.n_query, 48, replace=False))
    err, viol = parity.ranking_errors(XT64[q], XT64[w.n_query:], idx.cpu().numpy()[q], dist.cpu().numpy()[q])
    tol = DIST_TOL[precision]
    assert err < tol and viol < 2 * tol, (err, viol)
    assert st["band_failed"] == 0


@pytest.mark.parametrize("precision", ["tf32"])
def test_full_size_zipf_sampled(gcr, precision):
    """Large-scale workload (1,000 + 200,000, d = 512, 10,000 Zipf(1.1)-sized clusters, k = 30,
    T = 3) at full size, every layer staged against the oracle: the kNN sets of layers 1, 2 and 3
    on a 5 % row sample (10,050 rows), each layer's oracle fed the GPU's own features of the
    previous layer, with no pair left uncertified (later layers contract the large clusters to
    near-identical rows, which the ball search certifies); the propagation of layer 1 on 1,000
    rows; and the top-100 re-ranking of 64 seeded queries against the oracle's distances on the
    GPU's X_T. The full ranking of 200,000 gallery rows per query is outside the segmented sort
    (16,384 keys per query), so the certified top-K search is used."""
    w = workloads.zipf()
    p = gcr.default_params(k=w.k, T=w.T, precision=precision, topk_out=100)
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(w.n, w.n // 20, replace=False))
    X = gcr.gcr_normalize(_dev(w.X))
    for t in range(w.T):
        G = gcr.gcr_build_graph(X, p)
        Xn = gcr.gcr_propagate(G, X)
        torch.cuda.synchronize()
        st = G.stats_dict()
        assert st["band_failed"] == 0 and st["saturated"] == 0 and st["rows"] == w.n, (t, st)
        X64 = X.double().cpu().numpy()
        nbr = G.nbr.cpu().numpy()
        r = parity.compare_knn(X64, rows, nbr[rows], w.k)
        print(f"zipf layer {t + 1}: staged kNN {r}; {st}")
        assert r["mismatched"] == 0, (t, r, st)
        if t == 0:
            sub = rows[:: max(1, rows.size // 1000)][:1000]
            g_o = oracle.build_graph(X64, w.k, p.gamma, nbr=nbr)
            ref = oracle.propagate(X64, g_o["M"][sub])
            np.testing.assert_allclose(Xn.cpu().numpy()[sub], ref, atol=2e-6, rtol=0)
            del g_o
        del X64, G
        X = Xn
    del X, Xn
    idx, dist, XT, st = gcr.gcr_pipeline(_dev(w.X), w.n_query, p)
    torch.cuda.synchronize()
    assert st["band_failed"] == 0, st
    q = np.sort(rng.choice(w.n_query, 64, replace=False))
    XT64 = XT.double().cpu().numpy()
    D = oracle.sq_dist(XT64[q], XT64[w.n_query:])
    idx, dist = idx.cpu().numpy()[q], dist.cpu().numpy()[q]
    exact = 0
    for t in range(len(q)):
        o = np.argsort(D[t], kind="stable")[:100]
        g = idx[t]
        diff = sorted(set(o) ^ set(g))
        # the exact top-100 set, up to certified FP64 ties at the 100th distance
        assert not diff or np.all(np.abs(D[t, diff] - D[t, o[-1]]) < 1e-9), (t, len(diff))
        exact += 1
        np.testing.assert_allclose(dist[t], D[t, g], atol=1e-4, rtol=0)
        assert np.all(np.diff(D[t, g]) >= -1e-5)
    print(f"zipf {precision}: {exact}/{len(q)} sampled queries with the exact top-100 set; {st}")


@pytest.mark.parametrize("precision", PRECISIONS)
def test_topk_rerank_beyond_sort_limit(gcr, precision):
    """Top-K re-ranking of a 20,000-row gallery (beyond the 16,384-key segment sort) goes through
    the certified pool search: exact top-K sets (up to certified ties), FP32 distances."""
    w = workloads.plain(seed=8, n_query=64, n_gallery=20000, d=128, n_clusters=400)
    X0 = gcr.gcr_normalize(_dev(w.X))
    p = gcr.default_params(topk_out=100, precision=precision)
    idx, dist = gcr.gcr_rerank(X0[:64].contiguous(), X0[64:].contiguous(), p)
    torch.cuda.synchronize()
    X64 = X0.double().cpu().numpy()
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    assert idx.shape == (64, 100)
    D = oracle.sq_dist(X64[:64], X64[64:])
    for i in range(64):
        o = np.argsort(D[i], kind="stable")[:100]
        if set(o) != set(idx[i]):
            diff = np.array(sorted(set(o) ^ set(idx[i])))
            assert np.all(np.abs(D[i, diff] - D[i, o[-1]]) < 1e-9)
        np.testing.assert_allclose(dist[i], D[i, idx[i]], atol=1e-4, rtol=0)
        assert np.all(np.diff(D[i, idx[i]]) >= -1e-5)
    full = gcr.default_params(topk_out=0, precision=precision)
    with pytest.raises(gcr.GcrError):
        gcr.gcr_rerank(X0[:64].contiguous(), X0[64:].contiguous(), full)
