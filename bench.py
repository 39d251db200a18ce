#!/usr/bin/env python
"""Benchmark of the whole GCR re-ranking pipeline on one GB300 (or N replicas).

A step is one pass of the hot path over the cross-camera workload with the Market-1501
shape (3,368 queries + 15,913 gallery, d = 2048, 6 cameras, k = 20, T = 2, alpha = 0.7):
normalise, T x (similarity GEMM + streaming top-k, certified refinement, weights/degrees/
operator, propagation), then the re-ranked distance GEMM and the per-query sort.
The metric is re-ranked queries/s = queries / step time. The primary path is BF16 tensor
cores + certified FP32/FP64 refinement; the plain FP32 path is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). With --impl reference the FP64 CPU oracle is timed instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "re-ranked queries/s, BF16+refine vs plain FP32 at stated error; p50/p99 latency"
UNIT = "queries/s"
WORKLOAD = ("crosscam: 3,368 queries + 15,913 gallery (Market-1501 shape), d=2048, 751 identity "
            "clusters + 20% distractors, ReLU features, 6 cameras; k=20, T=2, gamma=0.2, alpha=0.7, "
            "symmetric operator, global + cross-camera graphs, full gallery ranking per query")
L2_FLUSH_BYTES = 256 << 20
FP32_LANES_PER_SM = 128
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense tensor rates of the GB300 (PFLOP/s)
N_SMS = 152


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["auto", "tf32", "bf16", "fp32"], default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-zipf", action="store_true", help="skip the 200,000-row Zipf workload")
    ap.add_argument("--no-video", action="store_true", help="skip the GCRV video workload")
    ap.add_argument("--no-local", action="store_true", help="skip the DSFP (Algorithm 1) comparison")
    ap.add_argument("--no-quality", action="store_true", help="skip the retrieval-quality measurements")
    ap.add_argument("--serving-requests", type=int, default=10000,
                    help="requests of the serving run of the headline precision (the others serve 1,000)")
    ap.add_argument("--pool", type=int, default=0, help="candidate pool per row (0: library default)")
    ap.add_argument("--only", choices=["zipf"], default=None,
                    help="run one workload alone and print its object (profiling runs)")
    ap.add_argument("--zipf-gallery", type=int, default=200000,
                    help="gallery rows of the zipf workload (a smaller case for --only zipf profiling runs)")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="gcr_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def result(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                except Exception:
                    continue
                rows.append((ts, parts))
        os.unlink(self.path)
        inwin = [p for ts, p in rows if self.t0 is None or (self.t0 - 1.0 <= ts <= self.t1 + 1.0)]
        use = inwin or [p for _, p in rows]
        sm = [float(p[2]) for p in use if p[2].replace(".", "").isdigit()]
        mx = [float(p[3]) for p in use if p[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in use for i in range(4) if p[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(use)}


# ------------------------------------------------------------------------------------ oracle arm
def oracle_sample_step(w, rows_knn=96, rows_q=96, rows_prop=2000, seed=0):
    """Times the FP64 oracle on bounded row samples of the workload and scales each stage
    linearly to the full workload. Returns (estimated seconds for one full step, detail).
    kNN: both graphs for `rows_knn` random rows against all rows; graph + propagation: the
    operator of the first `rows_prop` rows built from their own kNN lists (searched before the
    timer starts) and one propagation; re-ranking: `rows_q` random queries against the gallery."""
    import numpy as np
    import oracle

    rng = np.random.default_rng(seed)
    X0 = oracle.l2_normalize(w.X)
    n, nq = w.n, w.n_query
    rows = rng.choice(n, rows_knn, replace=False)
    t0 = time.perf_counter()
    oracle.knn_rows(X0, rows, w.k)
    oracle.knn_rows(X0, rows, w.k, w.cam, cross_camera=True)
    t_knn = time.perf_counter() - t0
    sub = np.arange(rows_prop)
    Xs = X0[sub]
    nbr, _ = oracle.knn(Xs, w.k)
    nbr_cr, _ = oracle.knn(Xs, w.k, w.cam[sub], cross_camera=True)
    t0 = time.perf_counter()
    g = oracle.build_graph(Xs, w.k, w.gamma, w.cam[sub], True, True, w.alpha, nbr=nbr, nbr_cr=nbr_cr)
    oracle.propagate(Xs, g["M"])
    t_prop = time.perf_counter() - t0
    q = rng.choice(nq, rows_q, replace=False)
    t0 = time.perf_counter()
    oracle.rerank(X0[q], X0[nq:])
    t_rr = time.perf_counter() - t0
    est = w.T * (t_knn * n / rows_knn + t_prop * n / rows_prop) + t_rr * nq / rows_q
    return est, dict(t_knn=t_knn, t_prop=t_prop, t_rerank=t_rr)


# sample of the CPU baseline printed beside our arm (about 10-12 s of oracle work on 16 cores),
# and the smaller per-step sample of the reference arm (a 20-step run stays within a minute)
CPU_SAMPLE = dict(rows_knn=6144, rows_q=3072, rows_prop=6000)
REF_SAMPLE = dict(rows_knn=384, rows_q=192, rows_prop=2000)


def cpu_sample_description(rows_knn, rows_q, rows_prop):
    return (f"FP64 oracle stages on row samples of the same workload, each scaled linearly to the full "
            f"step: kNN (global + cross-camera) of {rows_knn} of 19,281 rows per layer, graph + propagation "
            f"of the first {rows_prop} rows (on their own kNN lists), re-ranking of {rows_q} of 3,368 queries")


def run_reference(a):
    import numpy as np  # noqa: F401
    import workloads
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workloads.crosscam()
    for _ in range(a.warmup):
        oracle_sample_step(w, rows_knn=32, rows_q=32, rows_prop=500)
    ests = []
    t_start = time.perf_counter()
    for s in range(a.steps):
        est, _ = oracle_sample_step(w, seed=s, **REF_SAMPLE)
        ests.append(est)
    wall = time.perf_counter() - t_start
    ms = statistics.mean(ests) * 1e3
    v = w.n_query / (ms / 1e3)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)", "parallelism": "single process"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": cpu_sample_description(**REF_SAMPLE), "wall_s": wall},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------ our arm
def _src_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2306_08792_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel_key, files):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t.get(kernel_key)
        if e and e.get("src_hash") == _src_hash(files):
            return e.get("bytes_per_launch")
    except Exception:
        pass
    return None


def time_path(gcr, torch, w, X, cam, precision, steps, warmup, dist, pool=0):
    from paper_2306_08792_gb300 import _lib
    p = gcr.default_params(k=w.k, T=w.T, cross_camera=1, alpha=w.alpha, gamma=w.gamma, precision=precision,
                           pool=pool)
    pl = gcr.Pipeline(w.n, w.n_query, w.d, p)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        pl(X, cam, keep_features=False)
    torch.cuda.synchronize()
    lib = _lib.load()
    import ctypes
    S = _lib.GCR_STAGES
    ms_arr = (ctypes.c_double * S)()
    la = (ctypes.c_int64 * S)()
    ca = (ctypes.c_int64 * S)()
    lib.gcr_profile_enable(1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    pl.stats.zero_()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for s in range(steps):
        flush.zero_()                           # evict L2 between steps (outside the timed events)
        evs[s][0].record(stream)
        pl(X, cam, keep_features=False)
        evs[s][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    per = [a.elapsed_time(b) for a, b in evs]
    lib.gcr_profile_read(ms_arr, la, ca, S)
    lib.gcr_profile_enable(0)
    stages = {name: {"ms": ms_arr[i] / steps, "launches": la[i] / steps, "calls": ca[i] / steps}
              for i, name in enumerate(_lib.STAGE_NAMES)}
    launches = sum(v["launches"] for v in stages.values()) * steps
    return dict(ms=statistics.mean(per), ms_median=statistics.median(per), stages=stages, launches=launches,
                stats=pl.stats_dict(), pipeline=pl, params=p)


def time_e2e(gcr, torch, w, Xh, camh, p, steps, warmup):
    """The same re-ranking through the public host-buffer entry point (gcr_pipeline_host):
    every step copies the inputs from page-locked host memory and delivers the whole ranking
    to page-locked host memory inside the timed region."""
    stream = torch.cuda.current_stream()
    hp = gcr.HostPipeline(w.n, w.n_query, w.d, p)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        hp(Xh, camh)
    torch.cuda.synchronize()
    per = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hp(Xh, camh)
        b.record(stream)
        b.synchronize()
        per.append(a.elapsed_time(b))
    h2d = Xh.numel() * 4 + camh.numel() * 4
    d2h = hp.idx.numel() * 4 + hp.dist.numel() * 4
    # the median: a step that meets a host-side stall (seen now and then on shared hosts) does
    # not move it; the mean is reported beside it
    return statistics.median(per), statistics.mean(per), h2d, d2h, hp


def sampled_error(torch, pl, w, nsample=8):
    """Max |returned distance - FP64 distance on the returned features| over sampled queries."""
    import numpy as np
    XT = pl.X_final.double().cpu().numpy()
    q = np.random.default_rng(0).choice(w.n_query, nsample, replace=False)
    idx = pl.idx.cpu().numpy()[q].astype(np.int64)
    dist = pl.dist.cpu().numpy()[q].astype(np.float64)
    G = XT[w.n_query:]
    err = 0.0
    for t, qi in enumerate(q):
        diff = G[idx[t]] - XT[qi][None, :]
        d = np.sum(diff * diff, axis=1)
        err = max(err, float(np.max(np.abs(d - dist[t]))))
    return err


def capture_staged(gcr, torch, X, cam, p, nq, rows, queries):
    """An untimed layer-by-layer run of the same path (gcr_build_graph, gcr_propagate,
    gcr_rerank), keeping on the host what the oracle comparison of the CPU-baseline leg needs:
    each layer's input features X_{t-1} and kNN lists, the propagated rows of the sample, X_T
    and the ranking of the sampled queries. No oracle here."""
    Xt = gcr.gcr_normalize(X)
    layers = []
    for t in range(p.T):
        G = gcr.gcr_build_graph(Xt, p, cam)
        Xn = gcr.gcr_propagate(G, Xt)
        torch.cuda.synchronize()
        layers.append({"X": Xt.cpu().numpy(), "nbr": G.nbr.cpu().numpy(),
                       "nbr_cr": G.nbr_cr.cpu().numpy() if G.nbr_cr is not None else None,
                       "X_next_rows": Xn.cpu().numpy()[rows], "stats": G.stats_dict()})
        del G
        Xt = Xn
    idx, dist = gcr.gcr_rerank(Xt[:nq].contiguous(), Xt[nq:].contiguous(), p)
    torch.cuda.synchronize()
    return {"layers": layers, "XT": Xt.cpu().numpy(), "idx": idx.cpu().numpy()[queries],
            "dist": dist.cpu().numpy()[queries], "rows": rows, "queries": queries, "p": p, "nq": nq}


def serving_bench(gcr, torch, precision, n_requests):
    """Serving workload: 500,000 x 256 resident gallery (25,000 clusters), k = 20, T = 2, top-100;
    Poisson arrivals at 200 requests/s with log-uniform batch sizes in 1..512. Returns latency
    percentiles and throughput of the continuous-batching loop (real time, then saturation)."""
    import numpy as np
    import workloads
    from paper_2306_08792_gb300.serving import Gallery, Server, make_requests
    w = workloads.serving(n_requests=n_requests)
    p = gcr.default_params(k=w.k, T=w.T, topk_out=100, precision=precision)
    t0 = time.perf_counter()
    G = Gallery(torch.from_numpy(w.gallery).cuda(), p)
    build_s = time.perf_counter() - t0
    # device time of one gcr_serve call per batch size (CUDA events, after warm-up)
    per_batch = {}
    for b in (1, 8, 64, 512):
        q = torch.from_numpy(w.queries_of(b)).cuda()
        for _ in range(3):
            G.query(q)
        torch.cuda.synchronize()
        ts = []
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            G.query(q)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        per_batch[str(b)] = round(statistics.median(ts), 3)
    srv = Server(G, n_slots=4, max_batch=512)
    srv.warmup()
    reqs = make_requests(w, n_requests)
    rt = srv.run(reqs)
    sat = srv.run(make_requests(w, n_requests, realtime=False), realtime=False)
    # served rows kept for the oracle comparison of the CPU-baseline leg: 64 query rows drawn
    # from the real-time run's requests, with the gallery's stored layers and degrees
    rng = np.random.default_rng(11)
    picks = [(int(r), int(rng.integers(reqs[r].queries.shape[0]))) for r in rng.choice(len(reqs), 64)]
    T, ng, d = p.T, w.gallery.shape[0], w.gallery.shape[1]
    L = (T + 1) * ng * d * 4
    off = (L + 255) // 256 * 256
    staged = {"Q": np.stack([reqs[r].queries[i] for r, i in picks]),
              "idx": np.stack([reqs[r].idx[i] for r, i in picks]),
              "dist": np.stack([reqs[r].dist[i] for r, i in picks]),
              "layers": G.state[:L].view(torch.float32).reshape(T + 1, ng, d).cpu().numpy(),
              "degs": G.state[off:off + T * ng * 4].view(torch.float32).reshape(T, ng).cpu().numpy(),
              "k": w.k, "gamma": p.gamma, "T": T, "K": p.topk_out}
    del srv, G
    torch.cuda.empty_cache()
    return {"precision": precision, "gallery_build_s": build_s, "_staged": staged,
            "offered_requests_per_s": 200.0, "requests": n_requests,
            "p50_ms": rt["p50_ms"], "p99_ms": rt["p99_ms"], "queries_per_s": rt["queries_per_s"],
            "saturation_queries_per_s": sat["queries_per_s"], "saturation_p99_ms": sat["p99_ms"],
            "batch_device_ms": per_batch,
            "launches": rt["launches"]}


def zipf_bench(gcr, torch, precision, steps, warmup, staged=True, n_gallery=200000):
    """Large-scale workload: 1,000 queries + 200,000 gallery, d = 512, 10,000 Zipf(1.1)-sized
    clusters, k = 30, T = 3, top-100 re-ranking (the certified top-K search; the full ranking of
    200,000 rows per query is outside the segmented sort). Step time, stage times and the HBM
    roofline of the propagation kernel (algorithmic bytes per layer = 2*n*d*4 + nnz*8)."""
    import workloads
    from paper_2306_08792_gb300 import _lib
    import ctypes
    w = workloads.zipf(n_gallery=n_gallery)
    p = gcr.default_params(k=w.k, T=w.T, precision=precision, topk_out=100)
    X = torch.from_numpy(w.X).cuda()
    pl = gcr.Pipeline(w.n, w.n_query, w.d, p)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        pl(X, None, keep_features=False)
    torch.cuda.synchronize()
    lib = _lib.load()
    S = _lib.GCR_STAGES
    ms_arr, la, ca = (ctypes.c_double * S)(), (ctypes.c_int64 * S)(), (ctypes.c_int64 * S)()
    lib.gcr_profile_enable(1)
    stream = torch.cuda.current_stream()
    per = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pl(X, None, keep_features=False)
        b.record(stream)
        b.synchronize()
        per.append(a.elapsed_time(b))
    lib.gcr_profile_read(ms_arr, la, ca, S)
    lib.gcr_profile_enable(0)
    stages = {name: round(ms_arr[i] / steps, 4) for i, name in enumerate(_lib.STAGE_NAMES)}
    # operator entries of one layer's graph (layer 1), for the propagation's algorithmic bytes
    X0 = gcr.gcr_normalize(X)
    G = gcr.gcr_build_graph(X0, p)
    nnz = int(G.op_len.sum().item())
    bytes_layer = 2.0 * w.n * w.d * 4 + nnz * 8.0
    prop_ms = stages["propagate"] / w.T
    peaks, psrc = _peaks()
    gbs = bytes_layer / (prop_ms / 1e3) / 1e9
    ms = statistics.mean(per)
    del pl, G, X0
    import numpy as np
    rng = np.random.default_rng(3)
    if staged:
        staged = capture_staged(gcr, torch, X, None, p, w.n_query,
                                np.sort(rng.choice(w.n, w.n // 20, replace=False)),
                                np.sort(rng.choice(w.n_query, 64, replace=False)))
    del X
    torch.cuda.empty_cache()
    return {"_staged": staged, "_cfg": dict(k=w.k, gamma=w.gamma, cam=None, cross=False, alpha=1.0, topk=100,
                                            sample="5% of the rows (10,050) per layer, 64 queries"),
            "workload": f"zipf: 1,000 queries + {w.n - w.n_query:,} gallery, d=512, 10,000 Zipf(1.1) clusters, k=30, "
                        "T=3, top-100 re-ranking",
            "precision": precision, "steps": steps, "warmup": warmup, "ms_per_step": ms,
            "queries_per_s": w.n_query / (ms / 1e3), "stages_ms": stages,
            "propagate_roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                   "frac": gbs / peaks["hbm_gbs"], "peak_source": f"hbm_gbs of {psrc}",
                                   "bytes_per_layer": bytes_layer, "nnz": nnz, "ms_per_layer": prop_ms},
            "sim_gemm_tflops": 2.0 * w.n * w.n * w.d / (stages["sim_gemm"] / w.T / 1e3) / 1e12}


def video_bench(gcr, torch, precision, steps, warmup):
    """GCRV video workload (Algorithm 2): 1,980 query + 11,310 gallery tracklets of 2-100 frames
    (about 678k frames of d = 2048), 6 cameras, lambda = 10: the profile vectors of Eq. 17, then
    GCR with the global and cross-camera graphs on them (k = 20, T = 2, full ranking). Times the
    profiles and the re-ranking separately and together."""
    import workloads
    w = workloads.video()
    frames = torch.from_numpy(w.frames).cuda()
    off = torch.from_numpy(w.trk_off).cuda()
    cam = torch.from_numpy(w.trk_cam.astype("int32")).cuda()
    C = int(w.trk_cam.shape[0])
    ncam = int(w.trk_cam.max()) + 1
    p = gcr.default_params(k=w.k, T=w.T, cross_camera=1, alpha=0.7, precision=precision)
    pl = gcr.Pipeline(C, w.n_query, frames.shape[1], p)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def one(ev):
        ev[0].record(stream)
        W = gcr.gcrv_profiles(frames, off, cam, ncam, w.lam)
        ev[1].record(stream)
        pl(W, cam, keep_features=False)
        ev[2].record(stream)

    for _ in range(warmup):
        one([torch.cuda.Event(enable_timing=True) for _ in range(3)])
    torch.cuda.synchronize()
    prof, rr = [], []
    for _ in range(steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        one(ev)
        ev[2].synchronize()
        prof.append(ev[0].elapsed_time(ev[1]))
        rr.append(ev[1].elapsed_time(ev[2]))
    F, d = frames.shape
    ms = statistics.mean(prof) + statistics.mean(rr)
    import numpy as np
    W = gcr.gcrv_profiles(frames, off, cam, ncam, w.lam)
    rng = np.random.default_rng(4)
    staged = capture_staged(gcr, torch, W, cam, p, w.n_query, np.sort(rng.choice(C, 2000, replace=False)),
                            np.sort(rng.choice(w.n_query, 32, replace=False)))
    staged["W"] = W.cpu().numpy()
    del pl, frames, W
    torch.cuda.empty_cache()
    return {"_staged": staged, "_cfg": dict(k=w.k, gamma=w.gamma, cam=w.trk_cam, cross=True, alpha=0.7, topk=0,
                                            sample="2,000 of 13,290 tracklets per layer, 32 queries, "
                                                   "Eq. 17 residual of 3 tracklets per camera", video=w),
            "workload": f"video: {w.n_query:,} query + {C - w.n_query:,} gallery tracklets, {F:,} frames of "
                        f"d={d}, 6 cameras, lambda={w.lam}; GCR k={w.k}, T={w.T}, cross-camera, full ranking",
            "precision": precision, "steps": steps, "warmup": warmup, "ms_per_step": ms,
            "queries_per_s": w.n_query / (ms / 1e3), "profiles_ms": statistics.mean(prof),
            "rerank_ms": statistics.mean(rr),
            "frames_gb_per_s": F * d * 4 / (statistics.mean(prof) / 1e3) / 1e9,
            "gram_tflops": 2.0 * d * d * F / (statistics.mean(prof) / 1e3) / 1e12}


def local_bench(gcr, torch, w, X, precision, steps, warmup):
    """DSFP (Algorithm 1, "GCR_Local" of the paper's timing table) against global GCR with the
    same plain graph, on the crosscam features (19,281 x 2048, no camera graph), k = 20,
    T = 2, gamma = 0.2, full ranking: one step = the feature update plus the re-ranking
    (gcr_dsfp then gcr_rerank, against gcr_pipeline). Stage times from the stage profiler."""
    from paper_2306_08792_gb300 import _lib
    import ctypes
    p = gcr.default_params(k=w.k, T=w.T, gamma=w.gamma, cross_camera=0, precision=precision)
    ds = gcr.Dsfp(w.n, w.d, p)
    pl = gcr.Pipeline(w.n, w.n_query, w.d, p)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    nq = w.n_query

    def dsfp_step():
        out = ds(X)
        gcr.gcr_rerank(out[:nq], out[nq:], p)

    def gcr_step():
        pl(X, None, keep_features=False)

    lib = _lib.load()
    S = _lib.GCR_STAGES
    res = {}
    for name, fn in (("dsfp", dsfp_step), ("gcr_plain", gcr_step)):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        lib.gcr_profile_enable(1)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for s in range(steps):
            flush.zero_()
            evs[s][0].record(stream)
            fn()
            evs[s][1].record(stream)
        torch.cuda.synchronize()
        ms_arr = (ctypes.c_double * S)()
        la = (ctypes.c_int64 * S)()
        ca = (ctypes.c_int64 * S)()
        lib.gcr_profile_read(ms_arr, la, ca, S)
        lib.gcr_profile_enable(0)
        res[name] = {"ms": statistics.mean([a.elapsed_time(b) for a, b in evs]),
                     "stages": {nm: round(ms_arr[i] / steps, 4) for i, nm in enumerate(_lib.STAGE_NAMES)}}
    m = w.k + 1
    # the local kernel (stage "propagate" of gcr_dsfp): m(m+1)/2 Gram dot products and the
    # m-term output row per image, 2 FLOP per multiply-add
    flops = w.n * (m * (m + 1) / 2 + m) * w.d * 2.0
    kms = res["dsfp"]["stages"]["propagate"]
    peaks, psrc = _peaks()
    alu = N_SMS * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    del ds, pl
    torch.cuda.empty_cache()
    return {"workload": f"crosscam features ({w.n:,} x {w.d}) with the plain graph (no camera graph), k={w.k}, "
                        f"T={w.T}, gamma={w.gamma}, full ranking",
            "precision": precision, "steps": steps, "warmup": warmup,
            "dsfp_ms_per_step": res["dsfp"]["ms"], "dsfp_queries_per_s": nq / (res["dsfp"]["ms"] / 1e3),
            "gcr_plain_ms_per_step": res["gcr_plain"]["ms"],
            "gcr_plain_queries_per_s": nq / (res["gcr_plain"]["ms"] / 1e3),
            "speedup_dsfp_vs_gcr": res["gcr_plain"]["ms"] / res["dsfp"]["ms"],
            "dsfp_stages_ms": res["dsfp"]["stages"], "gcr_plain_stages_ms": res["gcr_plain"]["stages"],
            "local_kernel": {"kernel": "dsfp_kernel", "bound": "alu", "ms": kms, "flops": flops,
                             "achieved_tflops": flops / (kms / 1e3) / 1e12 if kms > 0 else None, "peak": alu,
                             "frac": flops / (kms / 1e3) / 1e12 / alu if kms > 0 else None,
                             "peak_source": f"FP32 FMA: 152 SMs x 128 lanes x 2 x sm_max_mhz of {psrc}"},
            "paper": "Sec. IV-F timing table (24-core CPU, Market-1501): GCR 24 s, GCR_Local 10 s"}


def profile_ablation(gcr, torch):
    """Mean profiles (Eq. 10) against the profile vectors of Eq. 17, each as is and followed by
    GCR with both graphs (Algorithm 2), on a video set whose cameras add offsets to the frames
    (mAP / Rank-1, cross-camera protocol on tracklets)."""
    import workloads
    v = workloads.video(n_query=500, n_gallery=2500, d=512, n_ids=400, max_len=40, sigma_trk=0.8, cam_bias=0.8)
    nq = v.n_query
    frames = torch.from_numpy(v.frames).cuda()
    off = torch.from_numpy(v.trk_off).cuda()
    cam = torch.from_numpy(v.trk_cam.astype("int32")).cuda()
    lab = torch.from_numpy(v.trk_label.astype("int32")).cuda()
    ql, gl, qc, gc = lab[:nq].contiguous(), lab[nq:].contiguous(), cam[:nq].contiguous(), cam[nq:].contiguous()

    def score(idx):
        s = gcr.retrieval_summary(*gcr.gcr_eval_retrieval(idx, ql, gl, qc, gc, protocol=1), ranks=(1,))
        return {"mAP": round(s["mAP"], 4), "rank1": round(s["rank1"], 4)}

    p = gcr.default_params(k=20, T=2, gamma=0.2, alpha=0.7, cross_camera=1, precision="tf32")
    out = {"workload": f"video: {nq} query + {v.C - nq} gallery tracklets of 2-40 frames ({v.frames.shape[0]:,} "
                       f"frames, d=512), 400 identities, tracklet spread 0.8, camera offsets 0.8, lambda={v.lam}"}
    for name, W in (("mean_profile", gcr.gcrv_mean_profiles(frames, off)),
                    ("pvg", gcr.gcrv_profiles(frames, off, cam, int(v.trk_cam.max()) + 1, v.lam))):
        Wn = gcr.gcr_normalize(W)
        out[name] = score(gcr.gcr_rerank(Wn[:nq], Wn[nq:], p)[0])
        out[name + "_gcr"] = score(gcr.gcr_pipeline(W, nq, p, cam)[0])
    return out


def quality_bench(gcr, torch):
    """Retrieval quality (mAP, Rank-1/5 under the cross-camera protocol: same-identity
    same-camera gallery items removed) on the ``camera_bias`` workload (Market-1501 shape,
    look-alike identities, per-camera offsets): the original features, global GCR with the
    plain graph, GCR with the cross-camera graph (Eq. 9), and DSFP (Algorithm 1), all TF32;
    then a sweep of k, T, gamma and alpha around the paper's defaults (GCR + cross-camera).
    Rankings and their evaluation run on the GPU (gcr_rerank / gcr_pipeline / gcr_dsfp,
    gcr_eval_retrieval)."""
    import workloads
    w = workloads.camera_bias()
    nq = w.n_query
    X = torch.from_numpy(w.X).cuda()
    cam = torch.from_numpy(w.cam).cuda()
    ql = torch.from_numpy(w.label[:nq].astype("int32")).cuda()
    gl = torch.from_numpy(w.label[nq:].astype("int32")).cuda()
    qc, gc = cam[:nq].contiguous(), cam[nq:].contiguous()

    def score(idx):
        ap, first = gcr.gcr_eval_retrieval(idx, ql, gl, qc, gc, protocol=1)
        s = gcr.retrieval_summary(ap, first, ranks=(1, 5))
        return {"mAP": round(s["mAP"], 4), "rank1": round(s["rank1"], 4), "rank5": round(s["rank5"], 4)}

    t0 = time.perf_counter()
    base = gcr.default_params(k=20, T=2, gamma=0.2, alpha=0.7, precision="tf32")
    Xn = gcr.gcr_normalize(X)
    out = {"original": score(gcr.gcr_rerank(Xn[:nq], Xn[nq:], base)[0])}

    def run(**kw):
        p = gcr.default_params(**{**dict(k=20, T=2, gamma=0.2, alpha=0.7, precision="tf32"), **kw})
        c = cam if p.cross_camera else None
        return score(gcr.gcr_pipeline(X, nq, p, c)[0])

    out["gcr_global"] = run(cross_camera=0)
    out["gcr_cross_camera"] = run(cross_camera=1)
    XL, _ = gcr.gcr_dsfp(X, gcr.default_params(k=20, T=2, gamma=0.2, precision="tf32"))
    out["dsfp"] = score(gcr.gcr_rerank(XL[:nq], XL[nq:], base)[0])
    sweep = []
    for k in (10, 15, 20, 30):
        for T in (1, 2, 3):
            sweep.append({"k": k, "T": T, "gamma": 0.2, "alpha": 0.7, **run(cross_camera=1, k=k, T=T)})
    for g in (0.1, 0.5, 1.0):
        sweep.append({"k": 20, "T": 2, "gamma": g, "alpha": 0.7, **run(cross_camera=1, gamma=g)})
    for a in (0.0, 0.3, 0.5, 0.9, 1.0):
        sweep.append({"k": 20, "T": 2, "gamma": 0.2, "alpha": a, **run(cross_camera=1, alpha=a)})
    out["sweep_gcr_cross_camera"] = sweep
    del X, Xn, XL
    out["video_profiles"] = profile_ablation(gcr, torch)
    torch.cuda.empty_cache()
    return {"workload": f"camera_bias: {nq:,} queries + {w.n - nq:,} gallery, d={w.d}, {w.params['n_clusters']} "
                        f"identities in groups of {w.params['ids_per_group']} look-alikes, 20% distractors, "
                        f"{w.params['n_cams']} cameras with offsets (cam_bias={w.params['cam_bias']})",
            "protocol": "cross-camera (same identity and camera removed); mAP = mean precision at each hit",
            "defaults": "k=20, T=2, gamma=0.2, alpha=0.7, TF32 search, full ranking", **out,
            "wall_s": time.perf_counter() - t0}


# ------------------------------------------------------------------ error against the oracle
# These run in the CPU-baseline leg (the FP64 oracle on the host cores), on the staged outputs
# the GPU part kept: the oracle is fed the GPU's own previous-stage outputs.
TIE = 1e-9   # a kNN mismatch is a certified tie when the FP64 gap to the k-th is below this


def _knn_vs_oracle(oracle, np, X64, rows, gpu_nbr, k, cam=None, cross=False):
    o_idx, o_d2 = oracle.knn_rows(X64, rows, k, cam, cross)
    mism = ties = 0
    worst = 0.0
    for t, r in enumerate(rows):
        g = set(int(j) for j in gpu_nbr[t] if j >= 0)
        o = set(int(j) for j in o_idx[t] if j >= 0)
        if g == o:
            continue
        valid = o_d2[t][np.isfinite(o_d2[t])]
        if len(g) != len(o) or valid.size == 0:
            mism += 1
            continue
        diff = np.array(sorted(g ^ o), dtype=np.int64)
        dd = X64[diff] - X64[r][None, :]
        gaps = np.abs(np.sum(dd * dd, axis=1) - valid[-1])
        worst = max(worst, float(gaps.max()))
        if np.all(gaps < TIE):
            ties += 1
        else:
            mism += 1
    return {"mismatched": mism, "certified_ties": ties, "worst_tie_gap": worst}


def staged_vs_oracle(oracle, np, st, cfg):
    """kNN sets and propagation of every layer on the sampled rows, and the final ranking of the
    sampled queries, against the FP64 oracle run on the GPU's previous-stage outputs."""
    rows, k = st["rows"], cfg["k"]
    out = {"sample": cfg["sample"], "tie_gap": TIE, "layers": []}
    for t, L in enumerate(st["layers"]):
        X64 = L["X"].astype(np.float64)
        rec = {"layer": t + 1, "search_stats": L["stats"],
               "knn": _knn_vs_oracle(oracle, np, X64, rows, L["nbr"][rows], k)}
        if cfg["cross"]:
            rec["knn_cross_camera"] = _knn_vs_oracle(oracle, np, X64, rows, L["nbr_cr"][rows], k, cfg["cam"], True)
        g_o = oracle.build_graph(X64, k, cfg["gamma"], cfg["cam"], cfg["cross"], True, cfg["alpha"],
                                 nbr=L["nbr"], nbr_cr=L["nbr_cr"])
        ref = oracle.propagate(X64, g_o["M"][rows])
        rec["max_propagation_err"] = float(np.max(np.abs(L["X_next_rows"] - ref)))
        out["layers"].append(rec)
        del X64, g_o
    XT = st["XT"].astype(np.float64)
    nq, q = st["nq"], st["queries"]
    D = oracle.sq_dist(XT[q], XT[nq:])
    idx = st["idx"].astype(np.int64)
    dq = np.take_along_axis(D, idx, axis=1)
    out["queries"] = int(len(q))
    out["max_dist_err"] = float(np.max(np.abs(dq - st["dist"])))
    out["max_order_violation"] = float(np.max(np.maximum(0.0, dq[:, :-1] - dq[:, 1:]))) if dq.shape[1] > 1 else 0.0
    if cfg["topk"]:
        bad = 0
        for t in range(len(q)):
            o = np.argsort(D[t], kind="stable")[:cfg["topk"]]
            diff = sorted(set(o) ^ set(idx[t]))
            if diff and not np.all(np.abs(D[t, diff] - D[t, o[-1]]) < TIE):
                bad += 1
        out["topk_mismatched_queries"] = bad
    return out


def profiles_vs_oracle(oracle, np, W, v, per_cam=3):
    """Eq. 17 profiles: the FP64 normal-equation residual ||(X_s^T X_s + lambda n_s I) w - (mu_c -
    mu_s)|| / ||mu_c - mu_s|| of sampled tracklets of every camera (cond <= 1 + 1/lambda, so the
    profile's relative error is at most that factor times the residual)."""
    rng = np.random.default_rng(0)
    off, worst = v.trk_off, 0.0
    for s in np.unique(v.trk_cam):
        members = np.nonzero(v.trk_cam == s)[0]
        fr = np.concatenate([np.arange(off[c], off[c + 1]) for c in members])
        Xs = oracle.l2_normalize(v.frames[fr])
        mu_s = Xs.mean(axis=0)
        for c in rng.choice(members, min(per_cam, members.size), replace=False):
            rhs = oracle.l2_normalize(v.frames[off[c]:off[c + 1]]).mean(axis=0) - mu_s
            w = W[c].astype(np.float64)
            res = Xs.T @ (Xs @ w) + v.lam * Xs.shape[0] * w - rhs
            worst = max(worst, float(np.linalg.norm(res) / np.linalg.norm(rhs)))
        del Xs
    return {"max_relative_residual": worst, "tracklets_per_camera": per_cam,
            "max_relative_profile_err_bound": worst * (1.0 + 1.0 / v.lam)}


def serving_vs_oracle(oracle, np, st):
    """Staged oracle query steps (the serving form of Eq. 6/7 with the gallery frozen) on the
    GPU's stored gallery layers and degrees, for the sampled served query rows."""
    xq = oracle.l2_normalize(st["Q"])
    layers = st["layers"]
    for t in range(st["T"]):
        xq = oracle.serve_oracle._query_step(xq, layers[t].astype(np.float64), st["degs"][t].astype(np.float64),
                                             st["k"], st["gamma"], True)
    GT = layers[st["T"]].astype(np.float64)
    D = oracle.sq_dist(xq, GT)
    idx = st["idx"].astype(np.int64)
    dq = np.take_along_axis(D, idx, axis=1)
    bad = 0
    for t in range(idx.shape[0]):
        o = np.argsort(D[t], kind="stable")[:st["K"]]
        diff = sorted(set(o) ^ set(idx[t]))
        if diff and not np.all(np.abs(D[t, diff] - D[t, o[-1]]) < TIE):
            bad += 1
    return {"sample": f"{idx.shape[0]} served query rows from the real-time run", "tie_gap": TIE,
            "topk_mismatched_queries": bad, "max_dist_err": float(np.max(np.abs(dq - st["dist"]))),
            "max_order_violation": float(np.max(np.maximum(0.0, dq[:, :-1] - dq[:, 1:])))}


# ------------------------------------------------------------------ reduced-precision bounds
# Rounding of a row to each candidate GEMM operand type, from the types' definitions: TF32 and
# BF16 keep 10 and 7 explicit mantissa bits (round to nearest even); e4m3 keeps 3, with an
# exponent range that a per-row scale max|x| / 448 maps the row into (subnormals below 2^-6).
def _round_mantissa(np, x, bits, min_exp=None):
    ax = np.abs(x)
    e = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
    if min_exp is not None:
        e = np.maximum(e, min_exp)
    step = np.exp2(e - bits)
    return np.round(x / step) * step


def rounded_rows(np, X, kind):
    if kind == "tf32":
        return _round_mantissa(np, X, 10)
    if kind == "bf16":
        return _round_mantissa(np, X, 7)
    scale = np.max(np.abs(X), axis=1, keepdims=True) / 448.0
    scale = np.where(scale > 0, scale, 1.0)
    return _round_mantissa(np, X / scale, 3, min_exp=-6) * scale


def certification_rates(np, oracle, X32, rows, k, kinds=("fp8_e4m3", "bf16", "tf32"), pool_mult=4):
    """For sampled rows: can a pool of pool_mult * k candidates, searched with a GEMM on operands
    of each type, certify the k nearest? Every score left out of such a pool is at most its last
    approximate score, so within delta of the (pool+1)-th exact score; the k-th must clear that by
    2 delta: s_(k) - s_(pool+1) > 2 delta_i, delta_i = ||x^_i|| max||e_j|| + ||e_i|| max||x_j|| +
    gamma_(d+32) ||x^_i|| max||x^_j|| (x^ the rounded row, e = x^ - x, FP32 accumulation)."""
    X = X32.astype(np.float64)
    n, d = X.shape
    kp = pool_mult * k
    S = X[rows] @ X.T
    S[np.arange(len(rows)), rows] = -np.inf
    top = -np.sort(-S, axis=1)[:, :kp + 1]
    gap = top[:, k - 1] - top[:, kp]
    gacc = (d + 32) * 2.0 ** -23
    out = {"rows": int(len(rows)), "pool": kp, "median_gap_k_to_pool": float(np.median(gap))}
    for kind in kinds:
        Xr = rounded_rows(np, X, kind)
        E = Xr - X
        en = np.linalg.norm(E, axis=1)
        an = np.linalg.norm(Xr, axis=1)
        bn = np.linalg.norm(X, axis=1)
        delta = an[rows] * en.max() + en[rows] * bn.max() + gacc * an[rows] * an.max()
        out[kind] = {"certified_share": float(np.mean(gap > 2.0 * delta)), "median_delta": float(np.median(delta))}
    return out


def oracle_full_times(oracle, np, workloads):
    """The FP64 oracle timed over whole workloads: the plain one (500 + 2,000 rows, d = 256) and
    the video one (GCRV, Algorithm 2: profiles then GCR with both graphs, full ranking)."""
    out = {}
    w = workloads.plain()
    t0 = time.perf_counter()
    Xo = oracle.gcr(w.X, w.k, w.gamma, w.T)
    oracle.rerank(Xo[:w.n_query], Xo[w.n_query:])
    dt = time.perf_counter() - t0
    out["plain"] = {"seconds": dt, "queries_per_s": w.n_query / dt,
                    "workload": "500 queries + 2,000 gallery, d=256, k=20, T=2, full ranking"}
    v = workloads.video()
    t0 = time.perf_counter()
    Xv = oracle.gcrv(v.frames, v.trk_off, v.trk_cam, v.lam, v.k, v.gamma, v.T, alpha=v.alpha)
    oracle.rerank(Xv[:v.n_query], Xv[v.n_query:])
    dt = time.perf_counter() - t0
    out["video"] = {"seconds": dt, "queries_per_s": v.n_query / dt,
                    "workload": "1,980 + 11,310 tracklets (675,977 frames, d=2048), Eq. 17 profiles, k=20, T=2, "
                                "cross-camera, full ranking"}
    out["cores"] = os.cpu_count()
    return out


def max_over_ranks(value: float, dist, device=None) -> float:
    """Largest value over all ranks (the slowest replica sets the job's time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, queries_per_replica: int, ms_max: float) -> float:
    """Whole-job queries/s of `world` independent replicas timed by the slowest one."""
    return world * queries_per_replica / (ms_max / 1e3)


def run_ours(a):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
        torch.cuda.set_device(local)
        dist = td
    else:
        torch.cuda.set_device(0)
    from paper_2306_08792_gb300 import build
    build.build()
    import paper_2306_08792_gb300 as gcr
    import workloads

    if not gcr.device_supported(torch.cuda.current_device()):
        raise SystemExit("libgcr needs an sm_103 GPU")
    if a.only == "zipf":
        z = zipf_bench(gcr, torch, "tf32" if a.precision == "auto" else a.precision, a.steps, a.warmup, staged=False,
                       n_gallery=a.zipf_gallery)
        z.pop("_staged", None)
        z.pop("_cfg", None)
        z["max_device_bytes"] = torch.cuda.max_memory_allocated()
        print(json.dumps(z), flush=True)
        return
    w = workloads.crosscam()
    Xh = torch.from_numpy(w.X).pin_memory()
    camh = torch.from_numpy(w.cam).pin_memory()
    X = Xh.cuda()
    cam = camh.cuda()

    from paper_2306_08792_gb300 import _lib
    prec_order = ["tf32", "bf16", "fp32"] if a.precision == "auto" else [a.precision]
    results = {}
    sampler = ClockSampler(local)
    sampler.mark_start()
    for prec in prec_order:
        try:
            results[prec] = time_path(gcr, torch, w, X, cam, prec, a.steps, a.warmup, dist,
                                      a.pool if prec != "fp32" else 0)
        except gcr.GcrError as e:
            if a.precision != "auto":
                raise
            results[prec] = {"error": str(e)}
    sampler.mark_end()
    clocks = sampler.result()
    # the headline is the fastest mode; every mode returns the same certified neighbour sets
    primary = min((p for p in prec_order if "ms" in results[p]), key=lambda p: results[p]["ms"])
    R = results[primary]
    ms = max_over_ranks(R["ms"], dist, "cuda")
    value = job_throughput(world, w.n_query, ms)

    e2e_ms, e2e_mean, h2d, d2h, hp = time_e2e(gcr, torch, w, Xh, camh, R["params"], max(7, a.steps), 3)
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")
    # one more untimed run that keeps the features, for the sampled error check
    R["pipeline"](X, cam, keep_features=True)
    torch.cuda.synchronize()
    err = sampled_error(torch, R["pipeline"], w)
    rng = np.random.default_rng(2)
    cross_staged = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cross_staged = capture_staged(gcr, torch, X, cam, R["params"], w.n_query,
                                      np.sort(rng.choice(w.n, 2000, replace=False)),
                                      np.sort(rng.choice(w.n_query, 32, replace=False)))

    peaks, psrc = _peaks()
    n, d = w.n, w.d
    flops = 2.0 * n * n * d
    sg = R["stages"]["sim_gemm"]
    per_launch_ms = sg["ms"] / max(sg["calls"], 1)
    achieved = flops / (per_launch_ms / 1e3) / 1e12
    if primary == "bf16":
        peak = peaks["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_source": f"bf16_tflops (burst) of {psrc}",
                "kernel": "umma_kernel POOL, BF16 (similarity GEMM + streaming top-k)",
                "traffic": _traffic("umma_pool", ["umma.cu", "pool.cuh"])}
    elif primary == "tf32":
        # TF32 dense peak: the measured BF16 peak x the nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s)
        peak = peaks["bf16_tflops"] * TF32_PER_BF16
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "peak_source": f"bf16_tflops (burst) of {psrc} x {TF32_PER_BF16:.4f} (nominal tf32/bf16)",
                "kernel": "umma_kernel POOL, TF32 (similarity GEMM + streaming top-k)",
                "traffic": _traffic("umma_pool_tf32", ["umma.cu", "pool.cuh"])}
    else:
        peak = N_SMS * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_source": f"FP32 FMA: 152 SMs x 128 lanes x 2 x sm_max_mhz of {psrc}",
                "kernel": "sgemm_pool_kernel (similarity GEMM + streaming top-k)",
                "traffic": _traffic("sgemm_pool", ["sgemm.cu", "pool.cuh"])}
    roof["flops_per_launch"] = flops
    roof["ms_per_launch"] = per_launch_ms
    roof["share_of_step"] = sg["ms"] / R["ms"]

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if primary == "fp32" else primary, "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": primary,
                       "l2": "flushed between steps (256 MB write outside the timed events); X is 158 MB > L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof,
            "e2e": {"value": job_throughput(world, w.n_query, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "ms_per_step_mean": e2e_mean,
                    "statistic": "median of steps", "api": "gcr_pipeline_host"},
            "gpu_launches": int(R["launches"]), "clocks": clocks,
            "stages_ms": {k: round(v["ms"], 4) for k, v in R["stages"].items()},
            "knn_stats": R["stats"], "max_dist_err_fp64_sampled": err}
    for prec in prec_order:
        if prec != primary:
            o = results[prec]
            if "ms" in o:
                line[f"{prec}_path"] = {"value": world * w.n_query / (o["ms"] / 1e3), "ms_per_step": o["ms"],
                                        "stages_ms": {k: round(v["ms"], 4) for k, v in o["stages"].items()},
                                        "knn_stats": o["stats"]}
                line["speedup_vs_" + prec] = o["ms"] / R["ms"]
            else:
                line[f"{prec}_path"] = o
    if rank == 0 and world == 1 and not a.no_zipf:
        try:
            line["zipf"] = zipf_bench(gcr, torch, primary if primary != "fp32" else "tf32", 3, 3)
        except gcr.GcrError as e:
            line["zipf"] = {"error": str(e)}
    if rank == 0 and world == 1 and not a.no_local:
        try:
            line["local"] = local_bench(gcr, torch, w, X, primary if primary != "fp32" else "tf32", 5, 3)
        except gcr.GcrError as e:
            line["local"] = {"error": str(e)}
    if rank == 0 and world == 1 and not a.no_quality:
        try:
            line["quality"] = quality_bench(gcr, torch)
        except gcr.GcrError as e:
            line["quality"] = {"error": str(e)}
    if rank == 0 and world == 1 and not a.no_video:
        try:
            line["video"] = video_bench(gcr, torch, primary if primary != "fp32" else "tf32", 3, 3)
        except gcr.GcrError as e:
            line["video"] = {"error": str(e)}
    if rank == 0 and world == 1 and not a.no_serving:
        serving = {}
        for prec in prec_order:
            try:
                nreq = a.serving_requests if prec == primary else min(1000, a.serving_requests)
                serving[prec] = serving_bench(gcr, torch, prec, nreq)
            except gcr.GcrError as e:
                serving[prec] = {"error": str(e)}
        line["serving"] = {"workload": "500,000 x 256 resident gallery, 25,000 clusters, k=20, T=2, top-100; "
                                       "Poisson 200 req/s, batch log-uniform 1..512, 4 slots, CUDA graphs",
                           **serving}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        est, det = oracle_sample_step(w, **CPU_SAMPLE)
        line["cpu_baseline"] = {"value": w.n_query / est, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": cpu_sample_description(**CPU_SAMPLE), "wall_s": time.perf_counter() - t0,
                                "stage_s": det}
        # error of every result against the oracle, fed the GPU's previous-stage outputs
        t0 = time.perf_counter()
        line["vs_oracle"] = staged_vs_oracle(oracle, np, cross_staged, dict(
            k=w.k, gamma=w.gamma, cam=w.cam, cross=True, alpha=w.alpha, topk=0,
            sample="2,000 of 19,281 rows per layer (both graphs), 32 queries (full ranking)"))
        z = line.get("zipf", {})
        if "_staged" in z:
            z["vs_oracle"] = staged_vs_oracle(oracle, np, z["_staged"], z["_cfg"])
        v = line.get("video", {})
        if "_staged" in v:
            v["vs_oracle"] = staged_vs_oracle(oracle, np, v["_staged"], v["_cfg"])
            v["vs_oracle"]["profiles"] = profiles_vs_oracle(oracle, np, v["_staged"]["W"], v["_cfg"]["video"])
        for prec, sv in line.get("serving", {}).items():
            if isinstance(sv, dict) and "_staged" in sv:
                sv["vs_oracle"] = serving_vs_oracle(oracle, np, sv["_staged"])
        line["vs_oracle"]["wall_s_all_workloads"] = time.perf_counter() - t0
        # whether reduced-precision GEMM operands (FP8 e4m3 with a per-row scale, BF16, TF32)
        # could certify the kNN of each layer from a pool of 4k candidates
        t0 = time.perf_counter()
        rng = np.random.default_rng(7)
        study = {"crosscam": [], "zipf": []}
        for L in cross_staged["layers"]:
            r = np.sort(rng.choice(L["X"].shape[0], 1000, replace=False))
            study["crosscam"].append(certification_rates(np, oracle, L["X"], r, w.k))
        if "_staged" in z:
            for L in z["_staged"]["layers"]:
                r = np.sort(rng.choice(L["X"].shape[0], 1000, replace=False))
                study["zipf"].append(certification_rates(np, oracle, L["X"], r, z["_cfg"]["k"]))
        study["wall_s"] = time.perf_counter() - t0
        line["precision_study"] = study
        # the oracle over whole workloads (small plain and video)
        line["cpu_baseline"]["full_runs"] = oracle_full_times(oracle, np, workloads)
    for obj in [line.get("zipf", {}), line.get("video", {})] + list(line.get("serving", {}).values()):
        if isinstance(obj, dict):
            obj.pop("_staged", None)
            obj.pop("_cfg", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
