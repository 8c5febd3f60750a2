"""Elementary (projection) DPP sampler, Algorithm 2 / Theorem 2, on the GPU.

With the same uniforms, the GPU draw must select the oracle's indices in the
oracle's order up to the first step whose target u_j S lies within 1e-9 S of a
running-sum boundary (there another summation order may legitimately pick the
neighbouring position), and on draws without such a step: log P(Y) within
1e-10 relative and the returned Cholesky factor of K_Y within 1e-10.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu

GAP = 1e-9


@pytest.fixture(scope="module")
def dpp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as m
    return m


def _compare(s, ref, k):
    got = s.sample.cpu().numpy()
    close = np.flatnonzero(ref.margin <= GAP)
    j0 = int(close[0]) if len(close) else k
    assert np.array_equal(got[:j0], ref.sample[:j0]), int(np.flatnonzero(got[:j0] != ref.sample[:j0])[0])
    r = s.result()
    assert r["status"] & 3 == 0, r
    if j0 == k:
        assert r["n_kept"] == k
        assert abs(r["logp"] - ref.logp) <= 1e-10 * max(1.0, abs(ref.logp)), (r["logp"], ref.logp)
        if s.chol is not None:
            assert np.abs(s.chol.cpu().numpy()[:k, :k] - ref.chol).max() < 1e-10
        keep = s.keep.cpu().numpy()
        assert keep.sum() == k and np.all(keep[ref.sample] == 1)
    return j0


@pytest.mark.parametrize("n,k", [(1, 1), (2, 1), (33, 5), (100, 25), (300, 1), (1000, 250),
                                 (777, 777), (2000, 100)])
def test_elementary_matches_oracle(dpp, n, k):
    import torch
    K = W.hermitian_kernel(n, seed=n + k, kind="projection", rank=k)
    Kd = torch.from_numpy(K).cuda()
    for seed in range(3):
        u = O.uniforms(seed, 0, k)
        ref = O.sample_elementary(K, k, u)
        s = dpp.sample_elementary(Kd, k, seed=seed, chol=True)
        torch.cuda.synchronize()
        _compare(s, ref, k)


def test_elementary_given_uniforms_and_empty(dpp):
    import torch
    n, k = 500, 40
    K = W.hermitian_kernel(n, seed=9, kind="projection", rank=k)
    u = np.random.default_rng(1).uniform(0.0, 1.0, k)
    ref = O.sample_elementary(K, k, u)
    s = dpp.sample_elementary(torch.from_numpy(K).cuda(), k, uniforms=torch.from_numpy(u),
                              chol=True)
    torch.cuda.synchronize()
    _compare(s, ref, k)
    e = dpp.sample_elementary(torch.from_numpy(K).cuda(), 0)
    torch.cuda.synchronize()
    assert e.sample.numel() == 0 and e.result()["n_kept"] == 0
    assert int(e.keep.sum().item()) == 0


def test_elementary_capped_grid(dpp):
    """Few CTAs (many positions each, the owner scans a long range)."""
    import torch
    from paper_1905_00165_gb300 import _lib
    n, k = 3000, 300
    K = W.hermitian_kernel(n, seed=4, kind="projection", rank=k)
    ref = O.sample_elementary(K, k, O.uniforms(2, 0, k))
    old = _lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS)
    _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, 8)
    try:
        s = dpp.sample_elementary(torch.from_numpy(K).cuda(), k, seed=2, chol=True)
        torch.cuda.synchronize()
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, old)
    _compare(s, ref, k)


def test_elementary_spanning_trees(dpp):
    """The transfer-current kernel of a grid graph is a projection of rank
    V - 1: every elementary draw is a spanning tree with log P = -log tau."""
    import torch
    d = 20
    K, edges, V = W.ust_grid_kernel(d)
    ref = -W.grid_spanning_tree_log_count(d)
    Kd = torch.from_numpy(K).cuda()
    for seed in range(3):
        s = dpp.sample_elementary(Kd, V - 1, seed=seed)
        torch.cuda.synchronize()
        keep = s.keep.cpu().numpy().astype(bool)
        assert O.is_spanning_tree(edges[keep], V)
        assert abs(s.result()["logp"] - ref) <= 1e-9 * abs(ref)


def test_elementary_paper_workload_n5000(dpp):
    """The paper's elementary-sampler workload (n = 5000, ranks 10, 100,
    500): parity with the oracle on one draw each."""
    import torch
    n = 5000
    for k in (10, 100, 500):
        K = W.hermitian_kernel(n, seed=k, kind="projection", rank=k, device="cuda")
        ref = O.sample_elementary(K, k, O.uniforms(0, 0, k))
        s = dpp.sample_elementary(torch.from_numpy(K).cuda(), k, seed=0, chol=True)
        torch.cuda.synchronize()
        _compare(s, ref, k)
