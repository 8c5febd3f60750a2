"""Mixed-precision (3xTF32 / FP32 SIMT) Hermitian path against the FP64 oracle.

The mixed path must draw the oracle's set on every decision whose uniform is
farther than 1e-9 from the pivot: outside its borderline band an FP32-derived
pivot cannot flip a decision, and inside it the pivot is recomputed in FP64.
log P(Y) is reported against the oracle with a relative tolerance of 1e-6
(FP32 working precision of the factors; the pivots themselves are FP64).
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


_PREC = {"p": "3xtf32"}


@pytest.fixture(params=[(1, "3xtf32", 0), (0, "3xtf32", 0), (0, "bf16x6", 0), (0, "bf16x6", 1),
                        (0, "3xtf32", 3)],
                ids=["simt", "tcgen05-3xtf32", "tcgen05-bf16x6", "tcgen05-bf16x6-single-helper",
                     "tcgen05-3xtf32-split"])
def update_kernel(request, dpp):
    """Trailing-update kernel (SIMT FP32 or tensor cores), operand split and
    panel pipeline (0: automatic, the chunked one on a full grid; 1: single
    helper; 3: split, the rows below the outer block in their own launch)."""
    from paper_1905_00165_gb300 import _lib
    kern, prec, pipe = request.param
    old = _lib.get_tuning(_lib.DPP_TUNE_UPDATE_KERNEL)
    oldp = _lib.get_tuning(_lib.DPP_TUNE_PANEL_PIPELINE)
    _lib.set_tuning(_lib.DPP_TUNE_UPDATE_KERNEL, kern)
    _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, pipe)
    _PREC["p"] = prec
    yield request.param
    _PREC["p"] = "3xtf32"
    _lib.set_tuning(_lib.DPP_TUNE_UPDATE_KERNEL, old)
    _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, oldp)


def _run(dpp, K, seed=0, uniforms=None, factor=False, precision=None):
    import torch
    Kd = torch.from_numpy(np.ascontiguousarray(K)).cuda()
    u = None if uniforms is None else torch.from_numpy(uniforms).cuda()
    s = dpp.sample_hermitian(Kd, seed=seed, precision=precision or _PREC["p"], uniforms=u,
                             factor=factor)
    torch.cuda.synchronize()
    return s


@pytest.mark.parametrize("n", [1, 31, 33, 100, 257, 300, 600, 1100])
def test_mixed_parity(dpp, update_kernel, n):
    from paper_1905_00165_gb300 import _lib
    K = W.hermitian_kernel(n, seed=n + 3, kind="uniform")
    for seed in range(3):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_ldl(K, u)
        s = _run(dpp, K, seed)
        r = s.result()
        assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE | _lib.DPP_RES_RECOMPUTE) == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                     logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)


def test_forced_borderline_pivots_are_recomputed(dpp, update_kernel):
    """Uniforms placed 1e-8 from the oracle's pivots (on the side that keeps the
    oracle's decision): every one lies inside the mixed path's error band, so
    each must be recomputed in FP64 and decided exactly."""
    from paper_1905_00165_gb300 import _lib
    n = 700
    K = W.hermitian_kernel(n, seed=21, kind="beta")
    u = O.uniforms(4, 0, n)
    ref = O.sample_ldl(K, u)
    pre = pre_decision_pivots(ref)
    targets = [0, 5, 31, 32, 40, 255, 256, 300, 511, 600, 699]
    for j in targets:
        u[j] = pre[j] - 1e-8 if ref.keep[j] else pre[j] + 1e-8
    ref2 = O.sample_ldl(K, u)
    assert np.array_equal(ref2.keep, ref.keep)
    s = _run(dpp, K, uniforms=u)
    r = s.result()
    assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_RECOMPUTE) == 0, r
    assert r["n_borderline"] >= len(targets) - 1, r  # pivot 0 is exact in any precision
    assert np.array_equal(s.keep.cpu().numpy(), ref2.keep)
    assert abs(r["logp"] - ref2.logp) <= MIXED_LOGP_RTOL * abs(ref2.logp)
    gp = s.pivots.cpu().numpy()
    for j in targets:
        assert abs(gp[j] - ref2.pivots[j]) < 1e-10, (j, gp[j], ref2.pivots[j])


@pytest.mark.parametrize("precision", ["bf16x6", "3xtf32"])
def test_forced_borderline_deep_pivots(dpp, precision):
    """Borderline pivots deep into a larger kernel (many 32-row blocks and
    worker CTAs in the recompute wavefronts), including the last index and
    the first and last row of an outer block."""
    from paper_1905_00165_gb300 import _lib
    n = 3000
    K = W.hermitian_kernel(n, seed=5, kind="beta")
    u = O.uniforms(9, 0, n)
    ref = O.sample_ldl(K, u)
    pre = pre_decision_pivots(ref)
    targets = [1000, 1279, 1280, 2047, 2500, 2999]
    for j in targets:
        u[j] = pre[j] - 1e-8 if ref.keep[j] else pre[j] + 1e-8
    ref2 = O.sample_ldl(K, u)
    s = _run(dpp, K, uniforms=u, precision=precision)
    r = s.result()
    assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_RECOMPUTE) == 0, r
    assert r["n_borderline"] >= len(targets), r
    assert np.array_equal(s.keep.cpu().numpy(), ref2.keep)
    gp = s.pivots.cpu().numpy()
    for j in targets:
        assert abs(gp[j] - ref2.pivots[j]) < 1e-10, (j, gp[j], ref2.pivots[j])


def test_mixed_projection_and_spanning_trees(dpp, update_kernel):
    n = 640
    K = W.hermitian_kernel(n, seed=2, kind="projection")
    for seed in range(3):
        assert int(_run(dpp, K, seed).keep.sum().item()) == n // 4
    d = 16
    K, edges, V = W.ust_grid_kernel(d)
    ref = -W.grid_spanning_tree_log_count(d)
    for seed in range(3):
        s = _run(dpp, K, seed)
        keep = s.keep.cpu().numpy().astype(bool)
        assert O.is_spanning_tree(edges[keep], V)
        assert abs(s.logp - ref) < MIXED_LOGP_RTOL * abs(ref)


def test_tensor_core_update_matches_simt(dpp):
    """Same forced decisions through both trailing-update kernels: the mixed
    factors agree to FP32-level accuracy."""
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 900
    K = W.hermitian_kernel(n, seed=5, kind="beta")
    keep = O.sample_ldl(K, O.uniforms(1, 0, n)).keep
    u = O.forced_uniforms(keep)
    facs = []
    old = _lib.get_tuning(_lib.DPP_TUNE_UPDATE_KERNEL)
    try:
        for kern, prec in ((1, "3xtf32"), (0, "3xtf32"), (0, "bf16x6")):
            _lib.set_tuning(_lib.DPP_TUNE_UPDATE_KERNEL, kern)
            s = _run(dpp, K, uniforms=u, factor=True, precision=prec)
            facs.append(np.tril(s.factor.cpu().numpy()))
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_UPDATE_KERNEL, old)
    ref = np.tril(O.sample_ldl(K, u).A)
    errs = [float(np.max(np.abs(f - ref))) for f in facs]
    assert max(errs) < 1e-4, errs


def test_outer_block_sizes(dpp):
    from paper_1905_00165_gb300 import _lib
    n = 520
    K = W.hermitian_kernel(n, seed=9, kind="uniform")
    u = O.uniforms(3, 0, n)
    ref = O.sample_ldl(K, u)
    old = _lib.get_tuning(_lib.DPP_TUNE_OUTER_BLOCK)
    try:
        for nb in (32, 64, 128, 256):
            _lib.set_tuning(_lib.DPP_TUNE_OUTER_BLOCK, nb)
            s = _run(dpp, K, 3)
            r = s.result()
            compare_draw(s.keep.cpu().numpy(), r["logp"], None, ref, u, logp_rtol=MIXED_LOGP_RTOL)
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_OUTER_BLOCK, old)


def _pivot_error_ratios(dpp, K, seed, precision="bf16x6"):
    """|d_mixed - d_fp64| / (2^-22 sqrt(j+1) (K_jj + s_j)) for every pivot of one
    draw, with the mixed path forced onto the FP64 path's decisions."""
    import torch
    n = K.shape[0]
    Kd = torch.from_numpy(np.ascontiguousarray(K)).cuda()
    s64 = dpp.sample_hermitian(Kd, seed=seed, precision="fp64", factor=True)
    keep = s64.keep.cpu().numpy()
    u = torch.from_numpy(O.forced_uniforms(keep)).cuda()
    smx = dpp.sample_hermitian(Kd, precision=precision, uniforms=u)
    torch.cuda.synchronize()
    d64 = s64.pivots.cpu().numpy()
    dmx = smx.pivots.cpu().numpy()
    F = s64.factor.cpu().numpy()
    L = np.tril(F, -1)
    s = (L * L) @ np.abs(d64)
    scale = 2.0 ** -22 * np.sqrt(np.arange(n) + 1.0) * (np.abs(np.diag(K)) + s)
    return np.abs(dmx - d64) / scale


def test_borderline_band_has_margin(dpp):
    """The band tau_j = c 2^-22 sqrt(j+1) (K_jj + s_j) must exceed the mixed
    path's actual pivot error by a wide margin: over every pivot of several
    draws of the workload shapes, the error stays below c / 8."""
    from paper_1905_00165_gb300 import _lib
    c = _lib.get_tuning(_lib.DPP_TUNE_TAU_SAFETY)
    worst = 0.0
    for n, kind, seed in [(2048, "beta", 0), (2048, "projection", 1), (3000, "uniform", 2)]:
        K = W.hermitian_kernel(n, seed=seed, kind=kind)
        r = _pivot_error_ratios(dpp, K, seed)
        worst = max(worst, float(r.max()))
    d = 20
    K, _, _ = W.ust_grid_kernel(d)
    worst = max(worst, float(_pivot_error_ratios(dpp, K, 3).max()))
    print(f"max pivot error / (2^-22 sqrt(j+1)(K_jj+s_j)) = {worst:.3e}, c = {c}")
    assert worst < c / 8.0


@pytest.mark.parametrize("pipeline", [1, 2, 3], ids=["single-helper", "chunked", "split"])
def test_capped_ctas_and_concurrent_streams(dpp, pipeline):
    """The mixed path with each launch capped at 40 CTAs still matches the
    oracle, and four draws issued on four streams at once give the same
    samples, pivots and log P as the same draws one after another."""
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 1100
    K = W.hermitian_kernel(n, seed=17, kind="beta")
    Kd = torch.from_numpy(K).cuda()
    old = _lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS)
    oldp = _lib.get_tuning(_lib.DPP_TUNE_PANEL_PIPELINE)
    _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, 40)
    _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, pipeline)
    try:
        for seed in range(2):
            u = O.uniforms(seed, 0, n)
            ref = O.sample_ldl(K, u)
            s = _run(dpp, K, seed, precision="bf16x6")
            compare_draw(s.keep.cpu().numpy(), s.logp, s.pivots.cpu().numpy(), ref, u,
                         logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)
        seq = []
        for seed in range(4):
            s = dpp.sample_hermitian(Kd, seed=seed, precision="bf16x6")
            torch.cuda.synchronize()
            seq.append((s.keep.clone(), s.pivots.clone(), s.logp))
        streams = [torch.cuda.Stream() for _ in range(4)]
        conc = []
        for seed, st in enumerate(streams):
            with torch.cuda.stream(st):
                conc.append(dpp.sample_hermitian(Kd, seed=seed, precision="bf16x6"))
        torch.cuda.synchronize()
        for (k0, p0, l0), s in zip(seq, conc):
            assert torch.equal(k0, s.keep)
            assert torch.equal(p0, s.pivots)
            assert s.logp == l0
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, old)
        _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, oldp)


def test_chunked_pipeline_small_grid(dpp):
    """The chunked panel pipeline on 8 CTAs: one helper owns every chunk of
    the outer block and each worker has more chunks than shared-memory slots
    (the rest are solved after the panel is published); still the oracle's
    draw."""
    from paper_1905_00165_gb300 import _lib
    n = 3600
    K = W.hermitian_kernel(n, seed=23, kind="beta")
    old = _lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS)
    oldp = _lib.get_tuning(_lib.DPP_TUNE_PANEL_PIPELINE)
    _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, 8)
    _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, 2)
    try:
        u = O.uniforms(2, 0, n)
        ref = O.sample_ldl(K, u)
        s = _run(dpp, K, 2, precision="bf16x6")
        r = s.result()
        assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE) == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                     logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, old)
        _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, oldp)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("precision", ["3xtf32", "bf16x6"])
def test_update_variants_match_oracle(dpp, precision, variant):
    """Every tensor-core update variant (operand ring depth, accumulator drain
    interval): the factor of forced decisions agrees with the oracle's to
    FP32-level accuracy, on every outer-block width (odd numbers of 32-deep
    blocks end a drain group early), and a draw is the oracle's."""
    from paper_1905_00165_gb300 import _lib
    n = 900
    K = W.hermitian_kernel(n, seed=5, kind="beta")
    keep = O.sample_ldl(K, O.uniforms(1, 0, n)).keep
    u = O.forced_uniforms(keep)
    ref = np.tril(O.sample_ldl(K, u).A)
    old = _lib.get_tuning(_lib.DPP_TUNE_UPDATE_VARIANT)
    oldb = _lib.get_tuning(_lib.DPP_TUNE_OUTER_BLOCK)
    _lib.set_tuning(_lib.DPP_TUNE_UPDATE_VARIANT, variant)
    try:
        for nb in (256, 96):
            _lib.set_tuning(_lib.DPP_TUNE_OUTER_BLOCK, nb)
            s = _run(dpp, K, uniforms=u, factor=True, precision=precision)
            err = float(np.max(np.abs(np.tril(s.factor.cpu().numpy()) - ref)))
            assert err < 1e-4, (nb, err)
        _lib.set_tuning(_lib.DPP_TUNE_OUTER_BLOCK, 256)
        uu = O.uniforms(7, 0, n)
        r = O.sample_ldl(K, uu)
        s = _run(dpp, K, seed=7, precision=precision)
        compare_draw(s.keep.cpu().numpy(), s.logp, s.pivots.cpu().numpy(), r, uu,
                     logp_rtol=MIXED_LOGP_RTOL, piv_atol=1e-4)
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_UPDATE_VARIANT, old)
        _lib.set_tuning(_lib.DPP_TUNE_OUTER_BLOCK, oldb)


@pytest.mark.parametrize("panel_ctas", [8, 16])
def test_split_pipeline_small_decision_grid(dpp, panel_ctas):
    """Split pipeline with the decision launch cut to 8 or 16 CTAs
    (DPP_TUNE_PANEL_CTAS): seven or fifteen recompute servers; borderline
    pivots deep into the kernel are still recomputed exactly."""
    from paper_1905_00165_gb300 import _lib
    n = 3000
    K = W.hermitian_kernel(n, seed=5, kind="beta")
    u = O.uniforms(9, 0, n)
    ref = O.sample_ldl(K, u)
    pre = pre_decision_pivots(ref)
    targets = [700, 1279, 2047, 2999]
    for j in targets:
        u[j] = pre[j] - 1e-8 if ref.keep[j] else pre[j] + 1e-8
    ref2 = O.sample_ldl(K, u)
    keys = (_lib.DPP_TUNE_PANEL_PIPELINE, _lib.DPP_TUNE_PANEL_CTAS, _lib.DPP_TUNE_MAX_CTAS)
    old = {k: _lib.get_tuning(k) for k in keys}
    _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, 3)
    _lib.set_tuning(_lib.DPP_TUNE_PANEL_CTAS, panel_ctas)
    _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, 38)
    try:
        s = _run(dpp, K, uniforms=u, precision="bf16x6")
    finally:
        for k, v in old.items():
            _lib.set_tuning(k, v)
    r = s.result()
    assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_RECOMPUTE) == 0, r
    assert r["n_borderline"] >= len(targets), r
    assert np.array_equal(s.keep.cpu().numpy(), ref2.keep)
    gp = s.pivots.cpu().numpy()
    for j in targets:
        assert abs(gp[j] - ref2.pivots[j]) < 1e-10, (j, gp[j], ref2.pivots[j])
