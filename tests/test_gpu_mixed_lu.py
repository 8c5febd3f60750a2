"""Mixed-precision general (LU) path against the FP64 oracle.

K = D^{-1} S D (S symmetric with spectrum in [0, 1], D log-normal): a
non-symmetric kernel with the principal minors of S. As for the Hermitian
mixed path, every decision whose uniform is farther than 1e-9 from the
oracle's pivot must equal the oracle's (a pivot inside the borderline band is
recomputed in FP64 with the two-sided identity), and log P(Y) agrees within
1e-6 relative.
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
    s = dpp.sample_lu(Kd, seed=seed, precision=precision, uniforms=u, factor=factor)
    torch.cuda.synchronize()
    return s


def _bad(lib):
    return lib.DPP_RES_TIMEOUT | lib.DPP_RES_NONFINITE | lib.DPP_RES_RECOMPUTE


@pytest.fixture(params=[0, 3], ids=["chunked", "split"])
def pipeline(request, dpp):
    """Panel pipeline: chunked (workers stream the rows below during the
    decisions) or split (the rows below in a separate wide launch)."""
    from paper_1905_00165_gb300 import _lib
    old = _lib.get_tuning(_lib.DPP_TUNE_PANEL_PIPELINE)
    _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, request.param)
    yield request.param
    _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, old)


@pytest.mark.parametrize("precision", ["bf16x6", "3xtf32"])
@pytest.mark.parametrize("n", [1, 31, 33, 100, 257, 300, 600, 1100])
def test_mixed_lu_parity(dpp, pipeline, n, precision):
    from paper_1905_00165_gb300 import _lib
    K, _ = W.lu_similarity_kernel(n, seed=n + 11)
    for seed in range(3):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_lu(K, u)
        s = _run(dpp, K, seed, precision)
        r = s.result()
        assert r["status"] & _bad(_lib) == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                     logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)
        assert r["n_kept"] == int(s.keep.sum().item())


def test_mixed_lu_similarity_twin(dpp):
    """LU of K = D^{-1} S D draws what LDL^T of S draws (same principal
    minors, Section 2), on the mixed paths of both forms."""
    import torch
    n = 700
    K, S = W.lu_similarity_kernel(n, seed=3)
    for seed in range(3):
        a = _run(dpp, K, seed)
        b = dpp.sample_hermitian(torch.from_numpy(S).cuda(), seed=seed, precision="bf16x6")
        torch.cuda.synchronize()
        u = O.uniforms(seed, 0, n)
        ref = O.sample_lu(K, u)
        pre = pre_decision_pivots(ref)
        close = np.flatnonzero(np.abs(u - pre) <= 1e-9)
        j0 = int(close[0]) if len(close) else n
        assert np.array_equal(a.keep.cpu().numpy()[:j0], b.keep.cpu().numpy()[:j0])
        if j0 == n:
            assert abs(a.logp - b.logp) <= 2 * MIXED_LOGP_RTOL * abs(b.logp)


@pytest.mark.parametrize("precision", ["bf16x6", "3xtf32"])
def test_mixed_lu_forced_borderline(dpp, pipeline, precision):
    """Uniforms 1e-8 from the oracle's pivots (on the side that keeps its
    decision), at the start, middle and end of inner panels and outer blocks:
    each pivot must be recomputed in FP64 and decided exactly."""
    from paper_1905_00165_gb300 import _lib
    n = 1500
    K, _ = W.lu_similarity_kernel(n, seed=21)
    u = O.uniforms(4, 0, n)
    ref = O.sample_lu(K, u)
    pre = pre_decision_pivots(ref)
    targets = [0, 5, 31, 32, 40, 255, 256, 300, 511, 777, 1023, 1024, 1280, 1499]
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
    gp = s.pivots.cpu().numpy()
    for j in targets:
        assert abs(gp[j] - ref2.pivots[j]) < 1e-10, (j, gp[j], ref2.pivots[j])


def test_mixed_lu_factor_matches_oracle(dpp):
    """The exported factor (L below, U = D U~ above) equals the oracle's
    in-place LU of K - 1_{Y^c} to FP32-level accuracy, with the same
    decisions forced through explicit uniforms."""
    n = 650
    K, _ = W.lu_similarity_kernel(n, seed=8)
    keep = O.sample_lu(K, O.uniforms(1, 0, n)).keep
    u = O.forced_uniforms(keep)
    ref = O.sample_lu(K, u)
    for precision in ("bf16x6", "3xtf32"):
        s = _run(dpp, K, uniforms=u, precision=precision, factor=True)
        assert np.array_equal(s.keep.cpu().numpy(), ref.keep)
        F = s.factor.cpu().numpy()
        scale = np.maximum(1.0, np.abs(ref.A))
        err = float(np.max(np.abs(F - ref.A) / scale))
        assert err < 1e-4, (precision, err)


def test_mixed_lu_rejects_in_place(dpp):
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 64
    K, _ = W.lu_similarity_kernel(n, seed=2)
    Kd = torch.from_numpy(K).cuda().t().contiguous().t()
    L = dpp.load()
    keep = torch.empty(n, dtype=torch.uint8, device="cuda")
    raw = torch.zeros(_lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    need = dpp.workspace_size(_lib.DPP_OP_SAMPLE_LU, n, _lib.DPP_R64, _lib.DPP_PREC_BF16X6, 0)
    assert need > 0
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    st = L.dpp_sample_lu(Kd.data_ptr(), n, n, _lib.DPP_R64, _lib.DPP_PREC_BF16X6, 0, 0, None,
                         keep.data_ptr(), Kd.data_ptr(), None, raw.data_ptr(), ws.data_ptr(),
                         need, torch.cuda.current_stream().cuda_stream)
    assert st == _lib.DPP_ERR_INVALID_ARG


def test_mixed_lu_matches_fp64_path_n8192(dpp):
    """The LU workload at its measured size (n = 8192, sigma = 0.5): the mixed
    path draws the FP64 GPU path's set up to the first pivot within 1e-9 of
    its uniform, and log P agrees to the mixed tolerance."""
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 8192
    K, _ = W.lu_similarity_kernel(n, seed=0, device="cuda")
    Kd = torch.from_numpy(np.ascontiguousarray(K)).cuda()
    for seed in (0, 1):
        ref = dpp.sample_lu(Kd, seed=seed, precision="fp64")
        mix = dpp.sample_lu(Kd, seed=seed, precision="bf16x6")
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


def test_mixed_lu_small_grid(dpp):
    """8 CTAs per launch: one helper owns all of the outer block's chunks and
    each worker has more chunks than shared-memory slots."""
    from paper_1905_00165_gb300 import _lib
    n = 3600
    K, _ = W.lu_similarity_kernel(n, seed=29)
    old = _lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS)
    _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, 8)
    try:
        u = O.uniforms(5, 0, n)
        ref = O.sample_lu(K, u)
        s = _run(dpp, K, 5)
        r = s.result()
        assert r["status"] & _bad(_lib) == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                     logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, old)
