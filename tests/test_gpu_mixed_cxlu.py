"""Mixed-precision complex LU path (non-Hermitian complex K) against the oracle.

Kernels: K = D^{-1} S D with S complex Hermitian (spectrum in [0, 1]) and D a
log-normal diagonal with complex phases (the principal minors of S, Section
2), and the Aztec-diamond tiling kernels built by Kenyon's formula (Section
1). Every decision whose uniform is farther than 1e-9 from the oracle's
pivot must equal the oracle's (pivots inside the borderline band are
recomputed in FP64 with the two-sided complex identity), log P(Y) agrees
within 1e-6 relative, and every Aztec draw is a tiling with log P =
-(d (d + 1) / 2) ln 2.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from tests._parity import compare_draw, pre_decision_pivots

pytestmark = pytest.mark.gpu

MIXED_LOGP_RTOL = 1e-6


@pytest.fixture(scope="module")
def dpp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as m
    return m


def _run(dpp, K, seed=0, precision="3xtf32", uniforms=None, factor=False):
    import torch
    Kd = K if isinstance(K, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(K)).cuda()
    u = None if uniforms is None else torch.from_numpy(uniforms).cuda()
    s = dpp.sample_lu(Kd, seed=seed, precision=precision, uniforms=u, factor=factor)
    torch.cuda.synchronize()
    return s


def _bad(lib):
    return lib.DPP_RES_TIMEOUT | lib.DPP_RES_NONFINITE | lib.DPP_RES_RECOMPUTE


def _cpiv(s):
    p = s.pivots.cpu().numpy()
    return p[0::2] + 1j * p[1::2]


@pytest.mark.parametrize("precision", ["3xtf32", "bf16x6"])
@pytest.mark.parametrize("n", [1, 31, 33, 100, 129, 257, 600, 1100])
def test_cxlu_parity(dpp, n, precision):
    from paper_1905_00165_gb300 import _lib
    K, _ = W.lu_similarity_kernel(n, seed=n + 5, complex_=True)
    for seed in range(3):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_lu(K, u)
        s = _run(dpp, K, seed, precision)
        r = s.result()
        assert r["status"] & _bad(_lib) == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                     logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)
        assert r["n_kept"] == int(s.keep.sum().item())


@pytest.mark.parametrize("precision", ["3xtf32", "bf16x6"])
@pytest.mark.parametrize("d", [2, 5, 10, 20])
def test_cxlu_aztec_tilings_match_oracle(dpp, d, precision):
    """Aztec diamonds of order 2..20 (n = 16..1600): oracle parity, every
    draw a tiling, log P the closed form."""
    from paper_1905_00165_gb300 import _lib
    K, edges, nb = W.aztec_kernel(d)
    n = K.shape[0]
    lt = W.aztec_log_tilings(d)
    for seed in range(2):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_lu(K, u)
        s = _run(dpp, K, seed, precision)
        r = s.result()
        assert r["status"] & _bad(_lib) == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                     logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-3)
        assert W.is_perfect_matching(edges, s.keep.cpu().numpy(), nb)
        assert abs(r["logp"] + lt) <= MIXED_LOGP_RTOL * lt


@pytest.mark.parametrize("precision", ["3xtf32", "bf16x6"])
def test_cxlu_forced_borderline(dpp, precision):
    """Uniforms 1e-8 from the oracle's pivots (on the side that keeps its
    decision), at the edges of 32-wide panels and 128-wide outer blocks:
    each is recomputed in FP64 and decided exactly; the recomputed pivots
    equal the oracle's to 1e-10."""
    from paper_1905_00165_gb300 import _lib
    n = 1500
    K, _ = W.lu_similarity_kernel(n, seed=23, complex_=True)
    u = O.uniforms(6, 0, n)
    ref = O.sample_lu(K, u)
    pre = pre_decision_pivots(ref)
    targets = [0, 5, 31, 32, 127, 128, 129, 255, 256, 700, 1023, 1024, 1499]
    for j in targets:
        u[j] = pre[j] - 1e-8 if ref.keep[j] else pre[j] + 1e-8
    ref2 = O.sample_lu(K, u)
    assert np.array_equal(ref2.keep, ref.keep)
    s = _run(dpp, K, uniforms=u, precision=precision)
    r = s.result()
    assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_RECOMPUTE) == 0, r
    assert r["n_borderline"] >= len(targets) - 1, r  # pivot 0 is exact in any precision
    assert np.array_equal(s.keep.cpu().numpy(), ref2.keep)
    assert abs(r["logp"] - ref2.logp) <= MIXED_LOGP_RTOL * abs(ref2.logp)
    gp = _cpiv(s)
    for j in targets:
        assert abs(gp[j] - ref2.pivots[j]) < 1e-10, (j, gp[j], ref2.pivots[j])


def test_cxlu_factor_matches_oracle(dpp):
    """The exported factor (L below, U = D U~ above) equals the oracle's
    in-place LU of K - 1_{Y^c} to FP32-level accuracy, decisions forced."""
    n = 650
    K, _ = W.lu_similarity_kernel(n, seed=9, complex_=True)
    keep = O.sample_lu(K, O.uniforms(1, 0, n)).keep
    u = O.forced_uniforms(keep)
    ref = O.sample_lu(K, u)
    for precision in ("3xtf32", "bf16x6"):
        s = _run(dpp, K, uniforms=u, precision=precision, factor=True)
        assert np.array_equal(s.keep.cpu().numpy(), ref.keep)
        F = s.factor.cpu().numpy()
        scale = np.maximum(1.0, np.abs(ref.A))
        err = float(np.max(np.abs(F - ref.A) / scale))
        assert err < 1e-4, (precision, err)


@pytest.mark.parametrize("ctas,outer", [(8, 128), (16, 64), (40, 32)])
def test_cxlu_small_grids_and_outer_blocks(dpp, ctas, outer):
    """Few CTAs per launch (few recompute servers, many tiles
    per CTA) and narrower outer blocks."""
    from paper_1905_00165_gb300 import _lib
    n = 1200
    K, _ = W.lu_similarity_kernel(n, seed=31, complex_=True)
    old = (_lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS), _lib.get_tuning(_lib.DPP_TUNE_OUTER_BLOCK))
    _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, ctas)
    _lib.set_tuning(_lib.DPP_TUNE_OUTER_BLOCK, outer)
    try:
        u = O.uniforms(2, 0, n)
        ref = O.sample_lu(K, u)
        s = _run(dpp, K, 2)
        r = s.result()
        assert r["status"] & _bad(_lib) == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                     logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, old[0])
        _lib.set_tuning(_lib.DPP_TUNE_OUTER_BLOCK, old[1])


def _band_ratio(dmx, ref, K):
    """|d_mixed - d_oracle| / (2^-22 sqrt(j+1) (|K_jj| + s_j)), s_j = sum_k |L_jk U_kj|."""
    Lm = np.tril(ref.A, -1)
    Um = np.triu(ref.A, 1)
    sj = np.sum(np.abs(Lm) * np.abs(Um.T), axis=1)
    n = len(sj)
    scale = 2.0 ** -22 * np.sqrt(np.arange(n) + 1.0) * (np.abs(np.diag(K)) + sj)
    return np.abs(dmx - ref.pivots) / scale


@pytest.mark.parametrize("precision", ["3xtf32", "bf16x6"])
def test_cxlu_band_margin(dpp, precision):
    """With the decisions forced to the oracle's (so that nothing is
    recomputed), every mixed pivot of a similarity kernel and of the order-30
    Aztec diamond lies within c / 8 of the band unit."""
    from paper_1905_00165_gb300 import _lib
    c = _lib.get_tuning(_lib.DPP_TUNE_TAU_SAFETY)
    worst = 0.0
    cases = [W.lu_similarity_kernel(2000, seed=41, complex_=True)[0], W.aztec_kernel(30)[0]]
    for K in cases:
        n = K.shape[0]
        ref0 = O.sample_lu(K, O.uniforms(0, 0, n))
        u = O.forced_uniforms(ref0.keep)
        ref = O.sample_lu(K, u)
        s = _run(dpp, K, uniforms=u, precision=precision)
        assert s.result()["n_borderline"] == 0
        ratio = _band_ratio(_cpiv(s), ref, K)
        worst = max(worst, float(ratio.max()))
        print(f"n={n}: max ratio {float(ratio.max()):.3e} at j={int(ratio.argmax())}")
    assert worst < c / 8.0


def test_cxlu_greedy_matches_oracle(dpp):
    """Greedy maximum-likelihood variant on the complex LU path: keep iff
    Re d_j > 1/2, the sampler's rule with every u_j = 1/2."""
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 900
    K, _ = W.lu_similarity_kernel(n, seed=13, complex_=True)
    ref = O.sample_lu(K, np.full(n, 0.5))
    g = dpp.greedy_lu(torch.from_numpy(K).cuda(), precision="3xtf32")
    torch.cuda.synchronize()
    r = g.result()
    assert r["status"] & _bad(_lib) == 0, r
    compare_draw(g.keep.cpu().numpy(), r["logp"], None, ref, np.full(n, 0.5),
                 logp_rtol=MIXED_LOGP_RTOL)


def test_cxlu_concurrent_streams(dpp):
    """Four draws on four streams with a capped grid give the draws made one
    after another."""
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 800
    K, _ = W.lu_similarity_kernel(n, seed=7, complex_=True)
    Kd = torch.from_numpy(K).cuda()
    old = _lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS)
    _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, 38)
    try:
        seq = []
        for seed in range(4):
            s = dpp.sample_lu(Kd, seed=seed, precision="3xtf32")
            torch.cuda.synchronize()
            seq.append((s.keep.clone(), s.pivots.clone(), s.logp))
        streams = [torch.cuda.Stream() for _ in range(4)]
        conc = []
        for seed, st in enumerate(streams):
            with torch.cuda.stream(st):
                conc.append(dpp.sample_lu(Kd, seed=seed, precision="3xtf32"))
        torch.cuda.synchronize()
        for (k, p, lp), s in zip(seq, conc):
            assert torch.equal(k, s.keep) and torch.equal(p, s.pivots) and lp == s.logp
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, old)


def _fp64_and_mixed(dpp, Kd, seed, precision="3xtf32"):
    import torch
    s64 = dpp.sample_lu(Kd, seed=seed, precision="fp64")
    smx = dpp.sample_lu(Kd, seed=seed, precision=precision)
    torch.cuda.synchronize()
    return s64, smx


def test_cxlu_aztec_order50(dpp):
    """Order 50 (n = 10000), the largest diamond whose Kenyon kernel the FP64
    input generator builds accurately (cond(Kast) ~ 1e14): the mixed draw
    is a tiling, its log P is -1275 ln 2 to 1e-6 relative, and its
    decisions are the FP64 GPU path's."""
    from paper_1905_00165_gb300 import _lib
    d = 50
    Kd, edges, nb = W.aztec_kernel(d, device="cuda", return_torch=True)
    lt = W.aztec_log_tilings(d)
    s64, smx = _fp64_and_mixed(dpp, Kd, 0)
    r = smx.result()
    assert r["status"] & _bad(_lib) == 0, r
    km = smx.keep.cpu().numpy()
    assert W.is_perfect_matching(edges, km, nb)
    assert abs(r["logp"] + lt) <= MIXED_LOGP_RTOL * lt
    assert np.array_equal(km, s64.keep.cpu().numpy())


def test_cxlu_equals_fp64_on_ill_conditioned_order60(dpp):
    """Order 60 (n = 14400): the kernel built in FP64 carries the rounding of
    an inverse with cond(Kast) ~ 1e17, so neither path draws a tiling (the
    pivots leave [0, 1]); the mixed path must still take every decision of
    the FP64 chain on this input, with log P to 1e-6 relative."""
    from paper_1905_00165_gb300 import _lib
    d = 60
    Kd, edges, nb = W.aztec_kernel(d, device="cuda", return_torch=True)
    for precision in ("3xtf32", "bf16x6"):
        s64, smx = _fp64_and_mixed(dpp, Kd, 0, precision)
        r, r64 = smx.result(), s64.result()
        assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE) == 0, r
        assert np.array_equal(smx.keep.cpu().numpy(), s64.keep.cpu().numpy())
        assert abs(r["logp"] - r64["logp"]) <= MIXED_LOGP_RTOL * abs(r64["logp"])
