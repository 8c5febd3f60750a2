"""Greedy maximum-likelihood variant (the remark after Prop. 1) on the GPU.

Every Bernoulli draw is replaced by its more likely outcome: keep j iff the
conditional inclusion probability d_j exceeds 1/2 (a tie rejects). The
reference is the oracle's independently written greedy LDL^H loop
(``oracle.greedy_ldl``, pinned on the CPU). Decisions are compared up to the
first pivot within 1e-9 of 1/2, where rounding order may decide either way.
For general K the LU form on K = D^{-1} S D must give the greedy set of the
Hermitian S (Prop. 2: diagonal similarity keeps every principal minor).
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as m
    return m


def _compare(keep, logp, pivots, ref, rtol, piv_atol, gap=1e-9):
    n = len(ref.keep)
    piv = np.asarray(ref.pivots, dtype=np.float64)
    pre = np.where(ref.keep == 1, piv, piv + 1.0)
    close = np.flatnonzero(np.abs(pre - 0.5) <= gap)
    j0 = int(close[0]) if len(close) else n
    keep = np.asarray(keep)[:n]
    assert np.array_equal(keep[:j0], ref.keep[:j0]), int(np.flatnonzero(keep[:j0] != ref.keep[:j0])[0])
    if pivots is not None:
        err = np.abs(np.asarray(pivots)[:j0] - piv[:j0])
        assert err.size == 0 or err.max() <= piv_atol, float(err.max())
    if j0 == n:
        assert abs(logp - ref.logp) <= rtol * max(1.0, abs(ref.logp)), (logp, ref.logp)
    return j0


@pytest.mark.parametrize("precision", ["fp64", "3xtf32", "bf16x6"])
@pytest.mark.parametrize("n", [1, 33, 300, 1100, 3000])
def test_greedy_hermitian_matches_oracle(dpp, precision, n):
    import torch
    from paper_1905_00165_gb300 import _lib
    K = W.hermitian_kernel(n, seed=100 + n, kind="beta")
    ref = O.greedy_ldl(K)
    s = dpp.greedy_hermitian(torch.from_numpy(K).cuda(), precision=precision)
    torch.cuda.synchronize()
    r = s.result()
    assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE | _lib.DPP_RES_RECOMPUTE) == 0, r
    rtol, atol = (1e-10, 1e-9) if precision == "fp64" else (1e-6, 1e-4)
    _compare(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, rtol, atol)


def test_greedy_borderline_half_is_recomputed(dpp):
    """A diagonal kernel with most pivots at 1/2 +- 1e-8, closer to 1/2 than
    FP32 can resolve: the mixed path must recompute each of them in FP64 and
    decide it exactly."""
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 200
    rng = np.random.default_rng(5)
    d = np.where(rng.random(n) < 0.5, 0.5 + 1e-8, 0.5 - 1e-8)
    d[::3] = rng.uniform(0.05, 0.95, len(d[::3]))
    K = np.diag(d)
    ref = O.greedy_ldl(K)
    assert np.array_equal(ref.keep, (d > 0.5).astype(np.uint8))
    s = dpp.greedy_hermitian(torch.from_numpy(K).cuda(), precision="bf16x6")
    torch.cuda.synchronize()
    r = s.result()
    assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_RECOMPUTE) == 0, r
    assert np.array_equal(s.keep.cpu().numpy()[:n], ref.keep)
    assert abs(r["logp"] - ref.logp) <= 1e-9 * abs(ref.logp)


@pytest.mark.parametrize("precision", ["fp64", "bf16x6"])
def test_greedy_lu_equals_greedy_of_similar_hermitian(dpp, precision):
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 700
    K, S = W.lu_similarity_kernel(n, seed=8)
    ref = O.greedy_ldl(S)
    Kd = torch.from_numpy(np.ascontiguousarray(K.T)).cuda().t()
    s = dpp.greedy_lu(Kd, precision=precision)
    torch.cuda.synchronize()
    r = s.result()
    assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE) == 0, r
    rtol = 1e-9 if precision == "fp64" else 1e-6
    _compare(s.keep.cpu().numpy(), r["logp"], None, ref, rtol, None)


def test_greedy_complex_hermitian(dpp):
    """Complex Hermitian K: the greedy set from the FP64 and mixed paths and the
    oracle's complex LDL^H with every threshold at 1/2 agree."""
    import torch
    n = 500
    K = W.hermitian_kernel(n, seed=77, kind="uniform", complex_=True)
    ref = O.sample_ldl(K, np.full(n, 0.5))
    Kd = torch.from_numpy(np.ascontiguousarray(K.T)).cuda().t()
    for precision, rtol in (("fp64", 1e-10), ("bf16x6", 1e-6)):
        s = dpp.greedy_hermitian(Kd, precision=precision)
        torch.cuda.synchronize()
        _compare(s.keep.cpu().numpy(), s.result()["logp"], None, ref, rtol, None)


def test_greedy_n16384_mixed_equals_fp64_path(dpp):
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 16384
    Kd = W.hermitian_kernel(n, seed=0, kind="beta", device="cuda", return_torch=True).contiguous()
    g64 = dpp.greedy_hermitian(Kd, precision="fp64")
    gmx = dpp.greedy_hermitian(Kd, precision="3xtf32")
    torch.cuda.synchronize()
    r64, rmx = g64.result(), gmx.result()
    assert rmx["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE | _lib.DPP_RES_RECOMPUTE) == 0
    k64 = g64.keep.cpu().numpy()
    p64 = g64.pivots.cpu().numpy()
    pre = np.where(k64 == 1, p64, p64 + 1.0)
    close = np.flatnonzero(np.abs(pre - 0.5) <= 1e-9)
    j0 = int(close[0]) if len(close) else n
    kmx = gmx.keep.cpu().numpy()
    assert np.array_equal(kmx[:j0], k64[:j0])
    if j0 == n:
        assert abs(rmx["logp"] - r64["logp"]) <= 1e-6 * abs(r64["logp"])
    print(f"greedy n={n}: |Y| = {int(k64.sum())}, log P = {r64['logp']:.6f}, "
          f"mixed recomputed {rmx['n_borderline']} pivots near 1/2")
