"""The autotuner on the GPU: it times every candidate launch configuration on
the caller's kernel, keeps the fastest in the tuning table, and the draws that
follow (which run with the tuned configuration) are still the oracle's."""
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
    yield m
    m._lib.tune_clear()


@pytest.mark.parametrize("hermitian,precision,n,cands",
                         [(True, "bf16x6", 1100, 13), (False, "3xtf32", 700, 11),
                          (True, "fp64", 300, 2)],
                         ids=["hermitian-mixed", "lu-mixed", "hermitian-fp64"])
def test_autotune_then_draw_matches_oracle(dpp, hermitian, precision, n, cands):
    import torch
    from paper_1905_00165_gb300 import _lib
    _lib.tune_clear()
    K = W.hermitian_kernel(n, seed=60 + n, kind="beta")
    Kd = torch.from_numpy(K).cuda()
    best = dpp.autotune(Kd, hermitian=hermitian, precision=precision, max_streams=2, draws=4)
    op = _lib.DPP_OP_SAMPLE_HERMITIAN if hermitian else _lib.DPP_OP_SAMPLE_LU
    assert best["candidates"] == cands, best
    assert best["streams"] in (1, 2) and best["samples_per_s"] > 0
    assert best["max_ctas"] == (0 if best["streams"] == 1 else
                                torch.cuda.get_device_properties(0).multi_processor_count // 2)
    got = _lib.tune_lookup(op, n, _lib.DPP_R64, _lib.PRECISIONS[precision])
    assert got == best
    # another order of the same power-of-two bucket uses the entry too
    assert _lib.tune_lookup(op, 1 << (n.bit_length() - 1), _lib.DPP_R64,
                            _lib.PRECISIONS[precision]) == best
    assert _lib.tune_lookup(op, 2 * n + 7, _lib.DPP_R64, _lib.PRECISIONS[precision]) is None
    f = dpp.sample_hermitian if hermitian else dpp.sample_lu
    for seed in range(2):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_ldl(K, u) if hermitian else O.sample_lu(K, u)
        s = f(Kd, seed=seed, precision=precision)
        torch.cuda.synchronize()
        r = s.result()
        assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE) == 0, r
        tol = 1e-10 if precision == "fp64" else 1e-6
        compare_draw(s.keep.cpu().numpy(), r["logp"], None, ref, u, logp_rtol=tol)
    _lib.tune_clear()
    assert _lib.tune_lookup(op, n, _lib.DPP_R64, _lib.PRECISIONS[precision]) is None


def test_autotune_batched_then_draw_matches_oracle(dpp):
    """dpp_autotune_batched times 128- and 256-thread CTAs on the caller's
    batch, keeps the faster under the batch's n_max bucket, and the draws that
    follow (with that CTA size) are the oracle's."""
    import torch
    from paper_1905_00165_gb300 import _lib
    _lib.tune_clear()
    sizes = [40, 96, 130, 257, 64, 200, 33, 300]
    Ks = [W.hermitian_kernel(m, seed=70 + i, kind="uniform") for i, m in enumerate(sizes)]
    b = dpp.BatchedSampler([torch.from_numpy(K).cuda() for K in Ks])
    best = b.autotune(draws=2)
    assert best["op"] == _lib.DPP_OP_SAMPLE_BATCHED and best["candidates"] == 2
    assert best["batched_threads"] in (128, 256) and best["samples_per_s"] > 0
    got = _lib.tune_lookup(_lib.DPP_OP_SAMPLE_BATCHED, 300, _lib.DPP_R64, _lib.DPP_PREC_FP32)
    assert got == best
    b.draw(7)
    torch.cuda.synchronize()
    for i, K in enumerate(Ks):
        m = K.shape[0]
        ref = O.sample_ldl(K, O.uniforms(7, i, m))
        res = _lib.decode_result(bytes(b.raw[i * _lib.RESULT_BYTES:(i + 1) * _lib.RESULT_BYTES]
                                       .cpu().numpy().tobytes()))
        assert res["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE) == 0, res
        compare_draw(b.keep[i][:m].cpu().numpy(), res["logp"], None, ref, O.uniforms(7, i, m),
                     logp_rtol=1e-6)
    _lib.tune_clear()
