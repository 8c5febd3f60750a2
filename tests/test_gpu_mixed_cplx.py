"""Mixed-precision Hermitian path for complex K against the FP64 oracle.

K = Q diag(lam) Q^H with Q Haar-unitary. Every decision whose uniform is
farther than 1e-9 from the oracle's pivot must equal the oracle's (a pivot in
the borderline band is recomputed in FP64 from K), log P(Y) within 1e-6
relative, on both operand splits of the two real tensor-core contractions.
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


def _run(dpp, K, seed=0, precision="bf16x6", uniforms=None, factor=False):
    import torch
    Kd = torch.from_numpy(np.ascontiguousarray(K)).cuda()
    u = None if uniforms is None else torch.from_numpy(uniforms).cuda()
    s = dpp.sample_hermitian(Kd, seed=seed, precision=precision, uniforms=u, factor=factor)
    torch.cuda.synchronize()
    return s


def _bad(lib):
    return lib.DPP_RES_TIMEOUT | lib.DPP_RES_NONFINITE | lib.DPP_RES_RECOMPUTE


@pytest.mark.parametrize("precision", ["bf16x6", "3xtf32"])
@pytest.mark.parametrize("n", [1, 33, 100, 300, 600])
def test_mixed_complex_parity(dpp, n, precision):
    from paper_1905_00165_gb300 import _lib
    K = W.hermitian_kernel(n, seed=n + 5, kind="uniform", complex_=True)
    for seed in range(3):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_ldl(K, u)
        s = _run(dpp, K, seed, precision)
        r = s.result()
        assert r["status"] & _bad(_lib) == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                     logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)


@pytest.mark.parametrize("precision", ["bf16x6", "3xtf32"])
def test_mixed_complex_forced_borderline(dpp, precision):
    """Uniforms 1e-8 from the oracle's pivots (keeping its decisions), across
    inner panels and outer blocks: each must be recomputed in FP64."""
    from paper_1905_00165_gb300 import _lib
    n = 700
    K = W.hermitian_kernel(n, seed=31, kind="beta", complex_=True)
    u = O.uniforms(6, 0, n)
    ref = O.sample_ldl(K, u)
    pre = pre_decision_pivots(ref)
    targets = [0, 5, 31, 32, 40, 255, 256, 300, 511, 600, 699]
    for j in targets:
        u[j] = pre[j] - 1e-8 if ref.keep[j] else pre[j] + 1e-8
    ref2 = O.sample_ldl(K, u)
    assert np.array_equal(ref2.keep, ref.keep)
    s = _run(dpp, K, uniforms=u, precision=precision)
    r = s.result()
    assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_RECOMPUTE) == 0, r
    assert r["n_borderline"] >= len(targets) - 1, r
    assert np.array_equal(s.keep.cpu().numpy(), ref2.keep)
    assert abs(r["logp"] - ref2.logp) <= MIXED_LOGP_RTOL * abs(ref2.logp)
    gp = s.pivots.cpu().numpy()
    for j in targets:
        assert abs(gp[j] - ref2.pivots[j]) < 1e-10, (j, gp[j], ref2.pivots[j])


def test_mixed_complex_factor_matches_oracle(dpp):
    n = 420
    K = W.hermitian_kernel(n, seed=8, kind="beta", complex_=True)
    keep = O.sample_ldl(K, O.uniforms(1, 0, n)).keep
    u = O.forced_uniforms(keep)
    ref = O.sample_ldl(K, u)
    s = _run(dpp, K, uniforms=u, factor=True)
    assert np.array_equal(s.keep.cpu().numpy(), ref.keep)
    F = np.tril(s.factor.cpu().numpy())
    err = float(np.max(np.abs(F - np.tril(ref.A))))
    assert err < 1e-4, err


def test_mixed_complex_small_grid(dpp):
    """8 CTAs: one helper owns every chunk of the outer block and the workers
    have more chunks than shared-memory slots."""
    from paper_1905_00165_gb300 import _lib
    n = 1500
    K = W.hermitian_kernel(n, seed=41, kind="beta", complex_=True)
    old = _lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS)
    _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, 8)
    try:
        u = O.uniforms(3, 0, n)
        ref = O.sample_ldl(K, u)
        s = _run(dpp, K, 3)
        r = s.result()
        assert r["status"] & _bad(_lib) == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                     logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, old)


@pytest.mark.parametrize("n,seeds,kind", [(4096, (0, 1), "beta"), (16384, (0,), "beta"),
                                          (16384, (1,), "projection")])
def test_mixed_complex_matches_fp64_path(dpp, n, seeds, kind):
    """The complex configurations at their measured sizes (n = 4096 and 16384,
    Beta(1/2,1/2) spectrum or a rank-n/4 projection): the mixed path draws the
    FP64 GPU path's set up to the first pivot within 1e-9 of its uniform; log P
    within the mixed tolerance."""
    import torch
    from paper_1905_00165_gb300 import _lib
    Kd = W.hermitian_kernel(n, seed=0, kind=kind, complex_=True, device="cuda",
                            return_torch=True).contiguous()
    for seed in seeds:
        ref = dpp.sample_hermitian(Kd, seed=seed, precision="fp64")
        mix = dpp.sample_hermitian(Kd, seed=seed, precision="bf16x6")
        torch.cuda.synchronize()
        rr, rm = ref.result(), mix.result()
        assert rm["status"] & _bad(_lib) == 0, rm
        u = dpp.uniforms(seed, 0, n).cpu().numpy()
        kr = ref.keep.cpu().numpy()
        pr = ref.pivots.cpu().numpy()
        pre = np.where(kr == 1, pr, pr + 1.0)
        close = np.flatnonzero(np.abs(u - pre) <= 1e-9)
        j0 = int(close[0]) if len(close) else n
        km = mix.keep.cpu().numpy()
        assert np.array_equal(km[:j0], kr[:j0]), int(np.flatnonzero(km[:j0] != kr[:j0])[0])
        if j0 == n:
            assert abs(rm["logp"] - rr["logp"]) <= MIXED_LOGP_RTOL * abs(rr["logp"])


def test_mixed_complex_projection_matches_oracle_n4096(dpp):
    """A complex rank-n/4 projection kernel (n = 4096) against one oracle draw:
    decisions up to the first borderline pivot, |Y| = rank, log P."""
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 4096
    K = W.hermitian_kernel(n, seed=3, kind="projection", complex_=True, device="cuda")
    Kd = torch.from_numpy(np.ascontiguousarray(K.T)).cuda().t()
    u = O.uniforms(2, 0, n)
    ref = O.sample_ldl(K, u)
    assert int(ref.keep.sum()) == n // 4
    s = dpp.sample_hermitian(Kd, seed=2, precision="3xtf32")
    torch.cuda.synchronize()
    r = s.result()
    assert r["status"] & _bad(_lib) == 0, r
    compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                 logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)
    assert r["n_kept"] == n // 4
