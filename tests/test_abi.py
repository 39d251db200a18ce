"""The C ABI library builds, loads and exports what include/gcr.h declares (CPU only).

These tests only call host-side functions (status strings, defaults, size queries and
argument validation, which returns before anything reaches the GPU).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_08792_gb300 import build, _lib
    build.build()
    return _lib.load()


def _declared():
    with open(os.path.join(ROOT, "include", "gcr.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b((?:gcr|gcrv)_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    from paper_2306_08792_gb300 import _lib
    declared = _declared()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
        assert name in _lib.PROTOTYPES, name


def test_status_strings(lib):
    assert lib.gcr_status_string(0) == b"ok"
    assert lib.gcr_status_string(2) == b"workspace too small"
    assert lib.gcr_status_string(99) == b"unknown status"


def test_defaults_are_the_papers(lib):
    """Library defaults equal the values the paper prints (tests/golden/paper_defaults.txt)."""
    from paper_2306_08792_gb300._lib import Params
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_defaults.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    p = Params()
    lib.gcr_default_params(ctypes.byref(p))
    assert p.k == vals["k"] and p.T == vals["T"]
    assert abs(p.gamma - vals["gamma"]) < 1e-7 and abs(p.alpha - vals["alpha"]) < 1e-7
    assert p.symmetric == 1


def _params(lib, **kw):
    from paper_2306_08792_gb300._lib import Params
    p = Params()
    lib.gcr_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_workspace_queries(lib):
    p = _params(lib, k=20)
    a = lib.gcr_build_graph_workspace_size(1000, 256, ctypes.byref(p))
    b = lib.gcr_build_graph_workspace_size(2000, 256, ctypes.byref(p))
    assert 0 < a < b
    assert lib.gcr_graph_op_capacity(1000, ctypes.byref(p)) == 1000 * (1 + 2 * 20)
    p2 = _params(lib, k=20, cross_camera=1)
    assert lib.gcr_graph_op_capacity(1000, ctypes.byref(p2)) == 1000 * (1 + 4 * 20)
    assert lib.gcr_build_graph_workspace_size(1000, 256, ctypes.byref(p2)) > a
    assert lib.gcr_rerank_workspace_size(100, 900, 256, ctypes.byref(p)) > 100 * 900 * 4
    assert lib.gcr_pipeline_workspace_size(1000, 100, 256, ctypes.byref(p)) > a


@pytest.mark.parametrize("bad", [dict(k=-1), dict(k=128), dict(k=32, pool=32), dict(gamma=0.0), dict(gamma=-1.0),
                                 dict(cross_camera=1, alpha=1.5), dict(precision=7), dict(precision=3), dict(pool=48),
                                 dict(pool=256),
                                 dict(symmetric=2)])
def test_invalid_params_rejected_on_host(lib, bad):
    p = _params(lib, **bad)
    assert lib.gcr_build_graph_workspace_size(1000, 256, ctypes.byref(p)) == 0
    from paper_2306_08792_gb300._lib import Graph
    g = Graph()
    st = lib.gcr_build_graph(ctypes.c_void_p(16), 1000, 256, ctypes.c_void_p(16), ctypes.byref(p),
                             ctypes.byref(g), ctypes.c_void_p(16), 1 << 30, None)
    assert st == 1  # GCR_E_INVALID


def test_unsupported_shapes(lib):
    p = _params(lib, k=10)
    assert lib.gcr_normalize(ctypes.c_void_p(16), ctypes.c_void_p(32), 10, 6, None) == 5
    pb = _params(lib, k=10, precision=1)
    from paper_2306_08792_gb300._lib import Graph
    g = Graph()
    assert lib.gcr_build_graph(ctypes.c_void_p(16), 100, 12, None, ctypes.byref(pb), ctypes.byref(g),
                               ctypes.c_void_p(16), 1 << 30, None) == 5
    assert lib.gcr_rerank_workspace_size(10, 20000, 256, ctypes.byref(p)) == 0
    # TF32 operands: rows of d % 8 == 0 (the distance GEMM shares the compensated BF16 operands);
    # a 32-entry pool is allowed under TF32, not under BF16
    pt = _params(lib, k=10, precision=2)
    assert lib.gcr_build_graph(ctypes.c_void_p(16), 100, 12, None, ctypes.byref(pt), ctypes.byref(g),
                               ctypes.c_void_p(16), 1 << 30, None) == 5
    assert lib.gcr_build_graph_workspace_size(100, 16, ctypes.byref(pt)) > 0
    assert lib.gcr_rerank_workspace_size(10, 100, 12, ctypes.byref(pt)) == 0
    pb32 = _params(lib, k=10, precision=1, pool=32)
    assert lib.gcr_build_graph(ctypes.c_void_p(16), 100, 16, None, ctypes.byref(pb32), ctypes.byref(g),
                               ctypes.c_void_p(16), 1 << 30, None) == 5
    assert lib.gcr_build_graph_workspace_size(100, 16, ctypes.byref(_params(lib, k=10, precision=2, pool=32))) > 0


def test_default_pool_leaves_a_margin_past_k(lib):
    # the default pool holds k plus max(12, k/2) candidates: k = 20 fits in 32, k = 30 needs 64,
    # k = 100 needs 128 (visible through the workspace, which scales with the pool)
    def ws(k, **kw):
        return lib.gcr_build_graph_workspace_size(1000, 256, ctypes.byref(_params(lib, k=k, **kw)))
    assert ws(20) == ws(20, pool=32)
    assert ws(30) == ws(30, pool=64)
    assert ws(100) == ws(100, pool=128)
    assert ws(10, precision=1) == ws(10, precision=1, pool=64)


def test_tf32_operand_copy_is_larger_than_bf16(lib):
    # the rounded operand copy holds 4 bytes per element under TF32, 2 under BF16
    pb = _params(lib, k=10, precision=1)
    pt = _params(lib, k=10, precision=2)
    wb = lib.gcr_build_graph_workspace_size(1000, 256, ctypes.byref(pb))
    wt = lib.gcr_build_graph_workspace_size(1000, 256, ctypes.byref(pt))
    assert wt - wb >= 1000 * 256 * 2


def test_null_and_short_workspace(lib):
    p = _params(lib, k=10)
    from paper_2306_08792_gb300._lib import Graph
    g = Graph()
    for f in ("nbr", "nbr_d2", "deg_r", "deg_c", "op_rowptr", "op_len", "op_col", "op_val"):
        setattr(g, f, 16)
    assert lib.gcr_build_graph(ctypes.c_void_p(16), 100, 64, None, ctypes.byref(p), ctypes.byref(g),
                               None, 0, None) == 2
    assert lib.gcr_build_graph(ctypes.c_void_p(16), 100, 64, None, ctypes.byref(p), ctypes.byref(g),
                               ctypes.c_void_p(16), 100, None) == 2
    g.op_len = None
    assert lib.gcr_build_graph(ctypes.c_void_p(16), 100, 64, None, ctypes.byref(p), ctypes.byref(g),
                               ctypes.c_void_p(16), 1 << 30, None) == 1
    # cross-camera without camera ids
    pc = _params(lib, k=10, cross_camera=1)
    assert lib.gcr_build_graph(ctypes.c_void_p(16), 100, 64, None, ctypes.byref(pc), ctypes.byref(g),
                               ctypes.c_void_p(16), 1 << 30, None) == 1


def test_product_package_does_not_import_oracle():
    import subprocess
    import sys
    code = ("import sys, paper_2306_08792_gb300; "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "False"


def test_gcrv_validation_on_host(lib):
    assert lib.gcrv_profiles_workspace_size(1000, 128, 50, 6) > 0
    assert lib.gcrv_profiles_workspace_size(1000, 128, 50, 65) == 0      # at most 64 cameras
    assert lib.gcrv_profiles_workspace_size(1000, 130, 50, 6) == 0       # d % 4
    p = ctypes.c_void_p(16)
    assert lib.gcrv_profiles(p, 1000, 128, p, p, 50, 6, ctypes.c_float(0.0), p, p, 1 << 30, None) == 1
    assert lib.gcrv_profiles(p, 1000, 130, p, p, 50, 6, ctypes.c_float(10.0), p, p, 1 << 30, None) == 5
    assert lib.gcrv_profiles(p, 1000, 128, p, p, 50, 6, ctypes.c_float(10.0), p, p, 100, None) == 2
    assert lib.gcrv_profiles(None, 1000, 128, p, p, 50, 6, ctypes.c_float(10.0), p, p, 1 << 30, None) == 1


def test_serving_validation_on_host(lib):
    p = _params(lib, k=20, T=2, topk_out=100)
    assert lib.gcr_gallery_bytes(500000, 256, ctypes.byref(p)) > 3 * 500000 * 256 * 4
    assert lib.gcr_serve_workspace_size(512, 500000, 256, ctypes.byref(p)) > 0
    assert lib.gcr_serve_workspace_size(0, 500000, 256, ctypes.byref(p)) == 0
    for bad in (dict(topk_out=0), dict(topk_out=128), dict(cross_camera=1), dict(T=-1)):
        kw = dict(k=20, T=2, topk_out=100)
        kw.update(bad)
        q = _params(lib, **kw)
        assert lib.gcr_gallery_bytes(500000, 256, ctypes.byref(q)) == 0, bad
    # the state keeps the last gallery graph's kNN lists (the final search's seed candidates):
    # ng * k int32, the only region that grows with k
    p30 = _params(lib, k=30, T=2, topk_out=100)
    grow = lib.gcr_gallery_bytes(500000, 256, ctypes.byref(p30)) - lib.gcr_gallery_bytes(500000, 256, ctypes.byref(p))
    assert 500000 * 10 * 4 <= grow < 500000 * 10 * 4 + 512
    v = ctypes.c_void_p(16)
    assert lib.gcr_serve(v, 1 << 40, 500000, v, 8, 256, ctypes.byref(p), v, v, None, None, 0, None) == 2
    assert lib.gcr_serve(None, 1 << 40, 500000, v, 8, 256, ctypes.byref(p), v, v, None, v, 1 << 40, None) == 1


def test_dsfp_validation_on_host(lib):
    p = _params(lib, k=20, T=2)
    assert lib.gcr_dsfp_workspace_size(1000, 256, ctypes.byref(p)) > 1000 * 256 * 4
    for bad in (dict(cross_camera=1), dict(T=-1), dict(k=65, pool=128), dict(gamma=0.0)):
        kw = dict(k=20, T=2)
        kw.update(bad)
        q = _params(lib, **kw)
        assert lib.gcr_dsfp_workspace_size(1000, 256, ctypes.byref(q)) == 0, bad
    v = ctypes.c_void_p(16)
    w = ctypes.c_void_p(4096)
    big = 1 << 40
    # missing or aliased buffers, then the error classes of the parameters
    assert lib.gcr_dsfp(None, 1000, 256, ctypes.byref(p), w, None, None, v, big, None) == 1
    assert lib.gcr_dsfp(v, 1000, 256, ctypes.byref(p), v, None, None, w, big, None) == 1
    assert lib.gcr_dsfp(v, 1000, 256, ctypes.byref(p), w, None, None, None, 0, None) == 2
    assert lib.gcr_dsfp(v, 1000, 256, ctypes.byref(p), w, None, None, v, 100, None) == 2
    assert lib.gcr_dsfp(v, 1000, 256, ctypes.byref(_params(lib, k=20, T=2, cross_camera=1)), w, None, None, v,
                        big, None) == 1
    assert lib.gcr_dsfp(v, 1000, 256, ctypes.byref(_params(lib, k=65, T=2, pool=128)), w, None, None, v,
                        big, None) == 5
    assert lib.gcr_dsfp(v, 1000, 258, ctypes.byref(p), w, None, None, v, big, None) == 5
    g = ctypes.c_float(0.2)
    assert lib.gcr_dsfp_propagate(v, 1000, 256, v, 20, ctypes.c_float(0.0), 2, w, None) == 1
    assert lib.gcr_dsfp_propagate(v, 1000, 256, v, 20, g, -1, w, None) == 1
    assert lib.gcr_dsfp_propagate(v, 1000, 256, None, 20, g, 2, w, None) == 1
    assert lib.gcr_dsfp_propagate(v, 1000, 256, v, 20, g, 2, v, None) == 1
    assert lib.gcr_dsfp_propagate(v, 1000, 256, v, 65, g, 2, w, None) == 5
    assert lib.gcr_dsfp_propagate(v, 1000, 258, v, 20, g, 2, w, None) == 5


def test_misaligned_feature_matrices_rejected_on_host(lib):
    # feature matrices are moved as 16-byte vectors: a base off the 16-byte grid is refused
    p = _params(lib, k=10, T=2)
    a, m = ctypes.c_void_p(4096), ctypes.c_void_p(4100)
    assert lib.gcr_normalize(m, a, 100, 64, None) == 1
    assert lib.gcr_normalize(a, m, 100, 64, None) == 1
    assert lib.gcr_dsfp(m, 100, 64, ctypes.byref(p), a, None, None, a, 1 << 40, None) == 1
    assert lib.gcr_dsfp(a, 100, 64, ctypes.byref(p), m, None, None, a, 1 << 40, None) == 1
    assert lib.gcr_dsfp_propagate(m, 100, 64, a, 10, ctypes.c_float(0.2), 2, ctypes.c_void_p(8192), None) == 1
    q = _params(lib, k=10, T=2, topk_out=5)
    assert lib.gcr_rerank(m, 10, a, 90, 64, ctypes.byref(q), a, a, a, 1 << 40, None) == 1
    assert lib.gcr_pipeline(m, 100, 10, 64, None, ctypes.byref(q), None, a, a, None, a, 1 << 40, None) == 1


def test_eval_validation_on_host(lib):
    v = ctypes.c_void_p(16)
    assert lib.gcr_eval_retrieval(None, 10, 5, v, v, v, v, 20, 0, v, v, None) == 1
    assert lib.gcr_eval_retrieval(v, 0, 5, v, v, v, v, 20, 0, v, v, None) == 1
    assert lib.gcr_eval_retrieval(v, 10, 0, v, v, v, v, 20, 0, v, v, None) == 1
    assert lib.gcr_eval_retrieval(v, 10, 5, v, v, v, v, 0, 0, v, v, None) == 1
    assert lib.gcr_eval_retrieval(v, 10, 5, v, v, v, v, 20, 2, v, v, None) == 1
    assert lib.gcr_eval_retrieval(v, 10, 5, v, None, v, v, 20, 1, v, v, None) == 1
    assert lib.gcr_eval_retrieval(v, 10, 5, v, v, v, v, 20, 0, None, v, None) == 1


def test_mean_profiles_validation_on_host(lib):
    assert lib.gcrv_mean_profiles_workspace_size(1000, 128, 50) >= 4000
    assert lib.gcrv_mean_profiles_workspace_size(1000, 130, 50) == 0
    assert lib.gcrv_mean_profiles_workspace_size(0, 128, 50) == 0
    p = ctypes.c_void_p(16)
    assert lib.gcrv_mean_profiles(p, 1000, 130, p, 50, p, p, 1 << 30, None) == 5
    assert lib.gcrv_mean_profiles(p, 1000, 128, p, 50, p, p, 100, None) == 2
    assert lib.gcrv_mean_profiles(None, 1000, 128, p, 50, p, p, 1 << 30, None) == 1
    assert lib.gcrv_mean_profiles(p, 1000, 128, p, 0, p, p, 1 << 30, None) == 1


def test_python_constants_match_the_header():
    """The binding's counter and stage tables follow the enums of include/gcr.h."""
    import re
    from paper_2306_08792_gb300 import _lib
    with open(os.path.join(ROOT, "include", "gcr.h")) as f:
        h = f.read()
    val = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(GCR_[A-Z0-9_]+)\s*=\s*(\d+)", h)}
    assert val["GCR_STATS_LEN"] == _lib.GCR_STATS_LEN == len(_lib.STAT_NAMES)
    for i, name in enumerate(_lib.STAT_NAMES):
        assert val["GCR_STAT_" + name.upper()] == i
    assert val["GCR_STAGES"] == _lib.GCR_STAGES
    for i, name in enumerate(_lib.STAGE_NAMES):
        assert val["GCR_STAGE_" + name.upper()] == i
