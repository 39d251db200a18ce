"""GPU parity tests of DSFP (Algorithm 1, the local propagation) through the C ABI against
the FP64 oracle.

The local propagation is compared on the same neighbour lists as the oracle (the GPU's own
lists in the full-search tests, whose sets are checked separately against the oracle's
exact kNN). Tolerance of the output rows (unit vectors): DSFP_TOL absolute. The kernel
forms the local Gram matrix with FP32 dot products over d terms, summed in 4-term FMA runs
per column group and then across the groups (error ~sqrt(d/4) 2^-24 relative, ~1e-6 at
d = 4096), derives the squared distances from it (G_uu + G_vv - 2 G_uv), weights them by
exp(-d2 / gamma) (an absolute distance error e moves a weight by e / gamma relative), and
runs the m x m recurrence in FP32 (~m 2^-24 per step). A weight error moves the output by
at most its size times the spread of the local rows around x_i (< 1 on a unit sphere), so
the bound is a few 1e-6 for gamma = 0.2; the measured errors on these cases are <= 1.2e-7.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests import parity

pytestmark = pytest.mark.gpu

DSFP_TOL = 5e-6
GAMMA = 0.2


@pytest.fixture(scope="module")
def gcr():
    import paper_2306_08792_gb300 as g
    from paper_2306_08792_gb300 import build
    build.build()
    assert g.device_supported(0), "this library targets sm_103 GPUs"
    return g


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _unit32(X):
    return oracle.l2_normalize(X).astype(np.float32)


@pytest.mark.parametrize("n,d,k,T", [(300, 256, 0, 2), (300, 256, 1, 2), (400, 132, 5, 1), (600, 256, 20, 2),
                                     (500, 260, 20, 3), (300, 256, 20, 0), (160, 256, 64, 2), (200, 4096, 12, 2)])
def test_local_propagation_matches_oracle(gcr, n, d, k, T):
    w = workloads.plain(seed=1, n_query=n // 5, n_gallery=n - n // 5, d=d)
    U32 = _unit32(w.X)
    U64 = U32.astype(np.float64)
    nbr = oracle.knn(U64, k)[0].astype(np.int32) if k > 0 else np.zeros((n, 0), np.int32)
    if k > 2:
        nbr[3, k // 2:] = -1                        # rows with absent neighbours are skipped
        nbr[7, :] = -1
    Y = gcr.gcr_dsfp_propagate(_dev(U32), _dev(nbr, torch.int32), GAMMA, T).cpu().numpy()
    rows = range(n) if k <= 20 else range(0, n, 4)
    ref = np.array([oracle.dsfp_local(U64, i, nbr[i], GAMMA, T) for i in rows])
    err = np.abs(Y[list(rows)] - ref).max()
    print(f"dsfp local n={n} d={d} k={k} T={T}: max |err| {err:.2e}")
    assert err < DSFP_TOL, err
    np.testing.assert_allclose(np.linalg.norm(Y, axis=1), 1.0, atol=1e-6)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "tf32"])
def test_dsfp_search_and_propagation(gcr, precision):
    w = workloads.plain(seed=2, n_query=200, n_gallery=900, d=256)
    p = gcr.default_params(k=20, T=2, gamma=GAMMA, precision=precision)
    X = _dev(w.X)
    out, nbr = gcr.gcr_dsfp(X, p)
    Xn = gcr.gcr_normalize(X).double().cpu().numpy()
    nbr = nbr.cpu().numpy()
    res = parity.compare_knn(Xn, np.arange(Xn.shape[0]), nbr, 20)
    assert res["mismatched"] == 0, res
    ref = np.array([oracle.dsfp_local(Xn, i, nbr[i], GAMMA, 2) for i in range(Xn.shape[0])])
    err = np.abs(out.cpu().numpy() - ref).max()
    print(f"dsfp search+propagation {precision}: max |err| {err:.2e}")
    assert err < DSFP_TOL, err


def test_dsfp_no_neighbours_is_normalisation(gcr):
    X, _ = workloads.random_unit_like(3, 257, 64)
    p = gcr.default_params(k=0, T=2, gamma=GAMMA)
    out, _ = gcr.gcr_dsfp(_dev(X), p)
    np.testing.assert_allclose(out.cpu().numpy(), oracle.l2_normalize(X), atol=1e-6, rtol=0)


def test_dsfp_k_past_the_sample_count(gcr):
    # 9 samples, k = 12: every row keeps the 8 others, the remaining slots are -1
    X, _ = workloads.random_unit_like(4, 9, 32)
    p = gcr.default_params(k=12, T=2, gamma=1.0)
    out, nbr = gcr.gcr_dsfp(_dev(X), p)
    nbr = nbr.cpu().numpy()
    assert (nbr[:, 8:] == -1).all() and (np.sort(nbr[:, :8], axis=1) >= 0).all()
    U = oracle.l2_normalize(X)
    ref, _ = oracle.dsfp(X, 12, 1.0, 2)
    assert np.abs(out.cpu().numpy() - ref).max() < DSFP_TOL
    assert np.array_equal(np.sort(nbr[:, :8], axis=1), np.array([[j for j in range(9) if j != i] for i in range(9)]))
    assert U.shape == (9, 32)


def test_dsfp_full_size_sampled(gcr):
    # the crosscam features (19,281 x 2048) with the plain graph, k = 20, T = 2, TF32 search:
    # sampled rows against the oracle (kNN sets, then the local propagation on those sets)
    w = workloads.crosscam()
    p = gcr.default_params(k=20, T=2, gamma=GAMMA, precision="tf32")
    X = _dev(w.X)
    ds = gcr.Dsfp(w.n, w.d, p)
    out = ds(X).cpu().numpy()
    nbr = ds.nbr.cpu().numpy()
    Xn = gcr.gcr_normalize(X).double().cpu().numpy()
    rows = np.random.default_rng(0).choice(w.n, 48, replace=False)
    res = parity.compare_knn(Xn, rows, nbr[rows], 20)
    assert res["mismatched"] == 0, res
    ref = np.array([oracle.dsfp_local(Xn, i, nbr[i], GAMMA, 2) for i in rows])
    err = np.abs(out[rows] - ref).max()
    print(f"dsfp full size sampled: max |err| {err:.2e}")
    assert err < DSFP_TOL, err
    st = ds.stats.cpu().numpy()
    assert st[0] == w.n and st[2] == 0     # every row searched, no band overflow
