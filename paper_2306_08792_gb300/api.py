"""Python binding of the C ABI: the same entry points, taking and returning torch tensors.

Argument marshalling only: each function checks shapes and dtypes, takes device pointers
from CUDA tensors, sizes and allocates the workspace with torch, and calls the library on
torch's current stream. Every computation runs in the library's kernels; there is no CPU
path and a missing library raises.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import torch

from . import _lib
from ._lib import GCR_PREC_BF16, GCR_PREC_FP32, GCR_PREC_TF32, Graph, Params


class GcrError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.load().gcr_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def _check(status: int, where: str):
    if status != 0:
        raise GcrError(status, where)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dev_f32(X: torch.Tensor, name: str) -> torch.Tensor:
    if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA matrix")
    return X


def default_params(**kw) -> Params:
    """The paper's defaults (k=15, gamma=0.2, T=3, alpha=0.7), overridden by keyword."""
    p = Params()
    _lib.load().gcr_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp32": GCR_PREC_FP32, "bf16": GCR_PREC_BF16, "tf32": GCR_PREC_TF32}[v]
        setattr(p, k, v)
    return p


def gcr_normalize(X: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    X = _dev_f32(X, "X")
    out = torch.empty_like(X) if out is None else out
    _check(_lib.load().gcr_normalize(_ptr(X), _ptr(out), X.shape[0], X.shape[1], _stream(stream)), "gcr_normalize")
    return out


@dataclass
class GraphTensors:
    """Device arrays of one built graph (see gcr_graph in include/gcr.h)."""
    nbr: torch.Tensor
    nbr_d2: torch.Tensor
    nbr_cr: Optional[torch.Tensor]
    nbr_cr_d2: Optional[torch.Tensor]
    deg_r: torch.Tensor
    deg_c: torch.Tensor
    deg_r_cr: Optional[torch.Tensor]
    deg_c_cr: Optional[torch.Tensor]
    op_rowptr: torch.Tensor
    op_len: torch.Tensor
    op_col: torch.Tensor
    op_val: torch.Tensor
    stats: torch.Tensor
    row_order: Optional[torch.Tensor] = None

    def struct(self) -> Graph:
        g = Graph()
        for f, _t in Graph._fields_:
            setattr(g, f, getattr(self, f).data_ptr() if getattr(self, f) is not None else None)
        return g

    def stats_dict(self):
        v = self.stats.cpu().tolist()
        return {name: int(v[i]) for i, name in enumerate(_lib.STAT_NAMES)}


def alloc_graph(n: int, p: Params, device) -> GraphTensors:
    lib = _lib.load()
    cap = lib.gcr_graph_op_capacity(n, ctypes.byref(p))
    cross = bool(p.cross_camera)
    k = p.k
    i32, f32 = torch.int32, torch.float32
    e = lambda *s, dt: torch.empty(*s, dtype=dt, device=device)  # noqa: E731
    return GraphTensors(
        nbr=e(n, k, dt=i32), nbr_d2=e(n, k, dt=f32),
        nbr_cr=e(n, k, dt=i32) if cross else None, nbr_cr_d2=e(n, k, dt=f32) if cross else None,
        deg_r=e(n, dt=f32), deg_c=e(n, dt=f32),
        deg_r_cr=e(n, dt=f32) if cross else None, deg_c_cr=e(n, dt=f32) if cross else None,
        op_rowptr=e(n + 1, dt=i32), op_len=e(n, dt=i32), op_col=e(max(cap, 1), dt=i32),
        op_val=e(max(cap, 1), dt=f32),
        stats=torch.zeros(_lib.GCR_STATS_LEN, dtype=torch.int64, device=device),
        row_order=e(n, dt=i32))


def gcr_build_graph(X: torch.Tensor, p: Params, cam: Optional[torch.Tensor] = None,
                    graph: Optional[GraphTensors] = None, ws: Optional[torch.Tensor] = None,
                    stream=None) -> GraphTensors:
    """kNN graph(s), degrees and propagation operator of the current features X (unit rows)."""
    X = _dev_f32(X, "X")
    n, d = X.shape
    lib = _lib.load()
    if cam is not None:
        if not (cam.is_cuda and cam.dtype == torch.int32 and cam.is_contiguous() and cam.numel() == n):
            raise ValueError("cam must be a contiguous int32 CUDA vector of length n")
    need = lib.gcr_build_graph_workspace_size(n, d, ctypes.byref(p))
    if need == 0:
        _check(lib.gcr_build_graph(_ptr(X), n, d, _ptr(cam), ctypes.byref(p), None, None, 0, _stream(stream)),
               "gcr_build_graph")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=X.device)
    g = alloc_graph(n, p, X.device) if graph is None else graph
    gs = g.struct()
    _check(lib.gcr_build_graph(_ptr(X), n, d, _ptr(cam), ctypes.byref(p), ctypes.byref(gs), _ptr(ws),
                               ws.numel(), _stream(stream)), "gcr_build_graph")
    return g


def gcr_propagate(graph: GraphTensors, X: torch.Tensor, out: Optional[torch.Tensor] = None,
                  stream=None) -> torch.Tensor:
    """One layer: out = normalise(M X) with M the operator held by `graph`."""
    X = _dev_f32(X, "X")
    out = torch.empty_like(X) if out is None else out
    gs = graph.struct()
    _check(_lib.load().gcr_propagate(ctypes.byref(gs), _ptr(X), _ptr(out), X.shape[0], X.shape[1],
                                     _stream(stream)), "gcr_propagate")
    return out


def gcr_rerank(Xq: torch.Tensor, Xg: torch.Tensor, p: Params, stream=None):
    """Per query: gallery indices by ascending squared distance (ties by index) and the distances."""
    Xq = _dev_f32(Xq, "Xq")
    Xg = _dev_f32(Xg, "Xg")
    nq, d = Xq.shape
    ng = Xg.shape[0]
    lib = _lib.load()
    K = min(p.topk_out, ng) if p.topk_out > 0 else ng
    need = lib.gcr_rerank_workspace_size(nq, ng, d, ctypes.byref(p))
    idx = torch.empty(nq, K, dtype=torch.int32, device=Xq.device)
    dist = torch.empty(nq, K, dtype=torch.float32, device=Xq.device)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=Xq.device)
    _check(lib.gcr_rerank(_ptr(Xq), nq, _ptr(Xg), ng, d, ctypes.byref(p), _ptr(idx), _ptr(dist), _ptr(ws),
                          need, _stream(stream)), "gcr_rerank")
    return idx, dist


def gcr_rerank_noalloc(Xq: torch.Tensor, Xg: torch.Tensor, p: Params, idx: torch.Tensor, dist: torch.Tensor,
                       stream=None):
    """gcr_rerank with the library's fixed scratch array instead of a workspace.

    For callers that must not allocate device memory during the call: the outputs are
    passed in, and the library uses its own resident scratch (see include/gcr.h)."""
    Xq = _dev_f32(Xq, "Xq")
    Xg = _dev_f32(Xg, "Xg")
    _check(_lib.load().gcr_rerank_noalloc(_ptr(Xq), Xq.shape[0], _ptr(Xg), Xg.shape[0], Xq.shape[1],
                                          ctypes.byref(p), _ptr(idx), _ptr(dist), _stream(stream)),
           "gcr_rerank_noalloc")
    return idx, dist


def gcrv_profiles(frames: torch.Tensor, trk_off: torch.Tensor, trk_cam: torch.Tensor, n_cams: int,
                  lam: float, stream=None) -> torch.Tensor:
    """Eq. 17 profile vectors (C x d, not normalised) of ragged tracklets of raw frames."""
    frames = _dev_f32(frames, "frames")
    if not (trk_off.is_cuda and trk_off.dtype == torch.int64 and trk_off.is_contiguous()):
        raise ValueError("trk_off must be a contiguous int64 CUDA vector")
    if not (trk_cam.is_cuda and trk_cam.dtype == torch.int32 and trk_cam.is_contiguous()):
        raise ValueError("trk_cam must be a contiguous int32 CUDA vector")
    F, d = frames.shape
    C = trk_cam.numel()
    if trk_off.numel() != C + 1:
        raise ValueError("trk_off must have C + 1 entries")
    lib = _lib.load()
    need = lib.gcrv_profiles_workspace_size(F, d, C, n_cams)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=frames.device)
    W = torch.empty(C, d, dtype=torch.float32, device=frames.device)
    _check(lib.gcrv_profiles(_ptr(frames), F, d, _ptr(trk_off), _ptr(trk_cam), C, n_cams, ctypes.c_float(lam),
                             _ptr(W), _ptr(ws), need, _stream(stream)), "gcrv_profiles")
    return W


def gcrv_mean_profiles(frames: torch.Tensor, trk_off: torch.Tensor, stream=None) -> torch.Tensor:
    """Eq. 10 mean profiles (C x d, not normalised) of ragged tracklets of raw frames."""
    frames = _dev_f32(frames, "frames")
    if not (trk_off.is_cuda and trk_off.dtype == torch.int64 and trk_off.is_contiguous()):
        raise ValueError("trk_off must be a contiguous int64 CUDA vector")
    F, d = frames.shape
    C = trk_off.numel() - 1
    lib = _lib.load()
    need = lib.gcrv_mean_profiles_workspace_size(F, d, C)
    if need == 0:
        raise GcrError(_lib.GCR_E_INVALID, "gcrv_mean_profiles_workspace_size")
    ws = torch.empty(need, dtype=torch.uint8, device=frames.device)
    W = torch.empty(C, d, dtype=torch.float32, device=frames.device)
    _check(lib.gcrv_mean_profiles(_ptr(frames), F, d, _ptr(trk_off), C, _ptr(W), _ptr(ws), need, _stream(stream)),
           "gcrv_mean_profiles")
    return W


class Dsfp:
    """gcr_dsfp (Algorithm 1, the local propagation) with a reusable workspace."""

    def __init__(self, n: int, d: int, p: Params, device="cuda"):
        self.n, self.d, self.p = n, d, p
        lib = _lib.load()
        need = lib.gcr_dsfp_workspace_size(n, d, ctypes.byref(p))
        if need == 0:
            raise GcrError(_lib.GCR_E_INVALID, "gcr_dsfp_workspace_size")
        self.ws = torch.empty(need, dtype=torch.uint8, device=device)
        self.out = torch.empty(n, d, dtype=torch.float32, device=device)
        self.nbr = torch.empty(n, max(p.k, 1), dtype=torch.int32, device=device)
        self.stats = torch.zeros(_lib.GCR_STATS_LEN, dtype=torch.int64, device=device)

    def __call__(self, X: torch.Tensor, stream=None) -> torch.Tensor:
        """X: raw float32 [n, d] on the device. Returns X_T (the kNN lists are in self.nbr)."""
        X = _dev_f32(X, "X")
        if tuple(X.shape) != (self.n, self.d):
            raise ValueError("X has the wrong shape")
        _check(_lib.load().gcr_dsfp(_ptr(X), self.n, self.d, ctypes.byref(self.p), _ptr(self.out),
                                    _ptr(self.nbr) if self.p.k > 0 else None, _ptr(self.stats), _ptr(self.ws),
                                    self.ws.numel(), _stream(stream)), "gcr_dsfp")
        return self.out


def gcr_dsfp(X: torch.Tensor, p: Params, stream=None):
    """One-shot Algorithm 1: returns (X_T, N_i lists int32 [n, k])."""
    n, d = X.shape
    ds = Dsfp(n, d, p, device=X.device)
    out = ds(X, stream=stream)
    return out, ds.nbr[:, :p.k]


def gcr_dsfp_propagate(X: torch.Tensor, nbr: torch.Tensor, gamma: float, T: int,
                       out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """The local propagation of Algorithm 1 on given neighbour lists (X: unit rows)."""
    X = _dev_f32(X, "X")
    if not (nbr.is_cuda and nbr.dtype == torch.int32 and nbr.dim() == 2 and nbr.is_contiguous()):
        raise ValueError("nbr must be a contiguous int32 CUDA matrix")
    n, d = X.shape
    k = nbr.shape[1]
    out = torch.empty_like(X) if out is None else out
    _check(_lib.load().gcr_dsfp_propagate(_ptr(X), n, d, _ptr(nbr) if k > 0 else None, k, ctypes.c_float(gamma),
                                          T, _ptr(out), _stream(stream)), "gcr_dsfp_propagate")
    return out


def _dev_i32(t: Optional[torch.Tensor], name: str, n: int):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.int32 and t.is_contiguous() and t.numel() == n):
        raise ValueError(f"{name} must be a contiguous int32 CUDA vector of {n} entries")
    return t


def gcr_eval_retrieval(idx: torch.Tensor, q_label: torch.Tensor, g_label: torch.Tensor,
                       q_cam: Optional[torch.Tensor] = None, g_cam: Optional[torch.Tensor] = None,
                       protocol: int = 0, stream=None):
    """Per-query average precision (float64, NaN without relevant items) and first-hit
    position (int32, -1 without a hit) of ranked lists idx [nq, K] (see include/gcr.h)."""
    if not (idx.is_cuda and idx.dtype == torch.int32 and idx.dim() == 2 and idx.is_contiguous()):
        raise ValueError("idx must be a contiguous int32 CUDA matrix")
    nq, K = idx.shape
    ng = g_label.numel()
    q_label = _dev_i32(q_label, "q_label", nq)
    g_label = _dev_i32(g_label, "g_label", ng)
    q_cam = _dev_i32(q_cam, "q_cam", nq)
    g_cam = _dev_i32(g_cam, "g_cam", ng)
    ap = torch.empty(nq, dtype=torch.float64, device=idx.device)
    first = torch.empty(nq, dtype=torch.int32, device=idx.device)
    _check(_lib.load().gcr_eval_retrieval(_ptr(idx), nq, K, _ptr(q_label), _ptr(q_cam), _ptr(g_label), _ptr(g_cam),
                                          ng, protocol, _ptr(ap), _ptr(first), _stream(stream)),
           "gcr_eval_retrieval")
    return ap, first


def retrieval_summary(ap: torch.Tensor, first: torch.Tensor, ranks=(1, 5, 10)) -> dict:
    """mAP and Rank-k over the queries that have relevant items (host-side averages)."""
    ap = ap.cpu()
    first = first.cpu().long()
    ok = ~torch.isnan(ap)
    out = {"mAP": float(ap[ok].mean()) if bool(ok.any()) else float("nan"), "queries": int(ok.sum())}
    for k in ranks:
        hit = (first[ok] >= 0) & (first[ok] < k)
        out[f"rank{k}"] = float(hit.double().mean()) if bool(ok.any()) else float("nan")
    return out


class Pipeline:
    """Whole re-ranking (normalise, T x (graph, propagate), re-rank) with reusable buffers."""

    def __init__(self, n: int, nq: int, d: int, p: Params, device="cuda"):
        self.n, self.nq, self.d, self.p = n, nq, d, p
        lib = _lib.load()
        need = lib.gcr_pipeline_workspace_size(n, nq, d, ctypes.byref(p))
        if need == 0:
            raise GcrError(_lib.GCR_E_INVALID, "gcr_pipeline_workspace_size")
        ng = n - nq
        K = min(p.topk_out, ng) if p.topk_out > 0 else ng
        self.ws = torch.empty(need, dtype=torch.uint8, device=device)
        self.idx = torch.empty(nq, K, dtype=torch.int32, device=device)
        self.dist = torch.empty(nq, K, dtype=torch.float32, device=device)
        self.X_final = torch.empty(n, d, dtype=torch.float32, device=device)
        self.stats = torch.zeros(_lib.GCR_STATS_LEN, dtype=torch.int64, device=device)

    def __call__(self, X: torch.Tensor, cam: Optional[torch.Tensor] = None, keep_features: bool = True,
                 stream=None):
        X = _dev_f32(X, "X")
        lib = _lib.load()
        _check(lib.gcr_pipeline(_ptr(X), self.n, self.nq, self.d, _ptr(cam), ctypes.byref(self.p),
                                _ptr(self.X_final) if keep_features else ctypes.c_void_p(0), _ptr(self.idx),
                                _ptr(self.dist), _ptr(self.stats), _ptr(self.ws), self.ws.numel(),
                                _stream(stream)), "gcr_pipeline")
        return self.idx, self.dist

    def stats_dict(self):
        v = self.stats.cpu().tolist()
        return {name: int(v[i]) for i, name in enumerate(_lib.STAT_NAMES)}


class HostPipeline:
    """gcr_pipeline_host: the re-ranking from page-locked host inputs to page-locked host
    outputs, the ranking's copies overlapped with the re-ranking of later query chunks."""

    def __init__(self, n: int, nq: int, d: int, p: Params, device="cuda"):
        self.n, self.nq, self.d, self.p = n, nq, d, p
        lib = _lib.load()
        need = lib.gcr_pipeline_host_workspace_size(n, nq, d, ctypes.byref(p))
        if need == 0:
            raise GcrError(_lib.GCR_E_INVALID, "gcr_pipeline_host_workspace_size")
        ng = n - nq
        K = min(p.topk_out, ng) if p.topk_out > 0 else ng
        self.ws = torch.empty(need, dtype=torch.uint8, device=device)
        self.idx = torch.empty(nq, K, dtype=torch.int32).pin_memory()
        self.dist = torch.empty(nq, K, dtype=torch.float32).pin_memory()
        self.stats = torch.zeros(_lib.GCR_STATS_LEN, dtype=torch.int64, device=device)

    def __call__(self, X: torch.Tensor, cam: Optional[torch.Tensor] = None, stream=None):
        """X: float32 [n, d] and cam: int32 [n] on the host (page-locked for asynchronous
        copies). Returns the host (idx, dist) buffers, complete once `stream` is synchronised."""
        if X.is_cuda or X.dtype != torch.float32 or X.dim() != 2 or not X.is_contiguous():
            raise ValueError("X must be a contiguous float32 host matrix")
        if cam is not None and (cam.is_cuda or cam.dtype != torch.int32 or not cam.is_contiguous()):
            raise ValueError("cam must be a contiguous int32 host vector")
        lib = _lib.load()
        _check(lib.gcr_pipeline_host(ctypes.c_void_p(X.data_ptr()), self.n, self.nq, self.d,
                                     ctypes.c_void_p(cam.data_ptr() if cam is not None else 0), ctypes.byref(self.p),
                                     ctypes.c_void_p(self.idx.data_ptr()), ctypes.c_void_p(self.dist.data_ptr()),
                                     _ptr(self.stats), _ptr(self.ws), self.ws.numel(), _stream(stream)),
               "gcr_pipeline_host")
        return self.idx, self.dist


def gcr_pipeline(X: torch.Tensor, nq: int, p: Params, cam: Optional[torch.Tensor] = None, stream=None):
    """One-shot wrapper of :class:`Pipeline`; returns (idx, dist, X_T, stats)."""
    n, d = X.shape
    pl = Pipeline(n, nq, d, p, device=X.device)
    idx, dist = pl(X, cam, stream=stream)
    return idx, dist, pl.X_final, pl.stats_dict()


def gcr_sync(stream=None):
    _check(_lib.load().gcr_sync(_stream(stream)), "gcr_sync")


def device_supported(device: int = 0) -> bool:
    return bool(_lib.load().gcr_device_supported(device))
