"""Distribution and multi-draw parity of the CUDA samplers.

* The 256-draw FP64 configuration (n = 512, K = Q diag(lam) Q^T, lam ~ U(0,1),
  Philox seeds 0..255): every draw against the FP64 oracle, decision by
  decision up to its first borderline pivot, log P within 1e-10.
* The same 256 draws as one batched launch (256 instances of one kernel, seed
  s = instance index via the instance counter) against the oracle.
* Empirical law of 65 536 batched GPU draws of an n = 10 kernel against the
  exact P(Y) = |det(K - 1_{Y^c})| from enumeration of all 1024 subsets
  (Theorem 1): a chi-squared test over the subsets with expected count >= 5,
  and inclusion frequencies against diag(K).
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from tests._parity import compare_draw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as m
    return m


def test_fp64_256_draws_n512_match_oracle(dpp):
    import torch
    n = 512
    K = W.hermitian_kernel(n, seed=0, kind="uniform")
    Kd = torch.from_numpy(K).cuda()
    borderline = 0
    for seed in range(256):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_ldl(K, u)
        s = dpp.sample_hermitian(Kd, seed=seed, precision="fp64")
        torch.cuda.synchronize()
        _, b = compare_draw(s.keep.cpu().numpy(), s.logp, s.pivots.cpu().numpy(), ref, u)
        borderline += int(b)
    assert borderline <= 2  # expected count ~ 256 * 2 * 1e-9 * n


def test_batched_256_instances_n512_match_oracle(dpp):
    import torch
    n = 512
    K = W.hermitian_kernel(n, seed=0, kind="uniform")
    Kd = torch.from_numpy(K).cuda()
    b = dpp.sample_batched([Kd] * 256, seed=7, instance=list(range(256)), want_pivots=True)
    torch.cuda.synchronize()
    res = b.results()
    for i in range(256):
        u = O.uniforms(7, i, n)
        ref = O.sample_ldl(K, u)
        compare_draw(b.keep[i][:n].cpu().numpy(), res[i]["logp"],
                     b.pivots[i][:n].cpu().numpy(), ref, u, logp_rtol=1e-6, piv_atol=1e-4)


def test_batched_law_n10_chi_squared(dpp):
    import torch
    n, draws = 10, 65536
    K = W.hermitian_kernel(n, seed=3, kind="uniform")
    probs = O.enumerate_probs(K)
    assert abs(probs.sum() - 1.0) < 1e-12
    Kd = torch.from_numpy(K).cuda()
    b = dpp.sample_batched([Kd] * draws, seed=11, instance=list(range(draws)))
    torch.cuda.synchronize()
    keep = torch.stack([k[:n] for k in b.keep]).cpu().numpy().astype(np.int64)
    masks = (keep << np.arange(n)[None, :]).sum(axis=1)
    counts = np.bincount(masks, minlength=1 << n).astype(np.float64)
    expected = probs * draws
    big = expected >= 5.0
    chi2 = float((((counts - expected) ** 2) / np.where(big, expected, 1.0))[big].sum())
    dof = int(big.sum()) - 1
    # chi-squared with dof degrees of freedom: mean dof, sd sqrt(2 dof); 6 sd
    assert chi2 < dof + 6.0 * np.sqrt(2.0 * dof), (chi2, dof)
    assert counts[~big].sum() <= expected[~big].sum() + 6.0 * np.sqrt(expected[~big].sum() + 1)
    freq = keep.mean(axis=0)
    sd = np.sqrt(np.diag(K) * (1 - np.diag(K)) / draws)
    assert np.all(np.abs(freq - np.diag(K)) <= 6.0 * sd + 1e-12)
