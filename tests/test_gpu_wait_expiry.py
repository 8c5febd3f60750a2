"""Bounded device waits run out cleanly (failure detection without a GPU fault).

The panel launches hand each decided panel to their other CTAs through a
device flag, and every wait on such a flag is bounded. Here the flag is one
that nothing sets: with DPP_TUNE_FAULT_WITHHOLD the CTA that makes the
decisions never releases its panels, and DPP_TUNE_WAIT_NS shortens the limit
to a few milliseconds. Each call must return, every launch must end, the
draw's status must carry DPP_RES_TIMEOUT, and the next ordinary draw on the
same device must again be the oracle's.
"""
import time

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


def _withheld(dpp, fn):
    """Run fn() with a 5 ms wait limit and the panel release withheld."""
    import torch
    from paper_1905_00165_gb300 import _lib
    old_w = _lib.get_tuning(_lib.DPP_TUNE_WAIT_NS)
    old_p = _lib.get_tuning(_lib.DPP_TUNE_PANEL_PIPELINE)
    _lib.set_tuning(_lib.DPP_TUNE_WAIT_NS, 5e6)
    _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, 2)
    _lib.set_tuning(_lib.DPP_TUNE_FAULT_WITHHOLD, 1)
    try:
        t0 = time.perf_counter()
        s = fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_FAULT_WITHHOLD, 0)
        _lib.set_tuning(_lib.DPP_TUNE_WAIT_NS, old_w)
        _lib.set_tuning(_lib.DPP_TUNE_PANEL_PIPELINE, old_p)
    return s, dt


@pytest.mark.parametrize("precision,hermitian",
                         [("fp64", True), ("fp64", False), ("bf16x6", True), ("3xtf32", False)],
                         ids=["fp64-hermitian", "fp64-lu", "mixed-hermitian-chunked",
                              "mixed-lu"])
def test_withheld_panel_times_out_and_next_draw_is_exact(dpp, precision, hermitian):
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 600
    K = W.hermitian_kernel(n, seed=31, kind="uniform")
    Kd = torch.from_numpy(K).cuda()
    f = dpp.sample_hermitian if hermitian else dpp.sample_lu
    s, dt = _withheld(dpp, lambda: f(Kd, seed=4, precision=precision))
    r = s.result()
    assert r["status"] & _lib.DPP_RES_TIMEOUT, r
    # 19 panels (FP64) or 3 outer blocks (mixed), each ending after its 5 ms
    # limit: far below the default 2 s limit of even one wait
    assert dt < 10.0, dt
    # the library and the device are usable again: the oracle's draw
    u = O.uniforms(4, 0, n)
    ref = O.sample_ldl(K, u) if hermitian else O.sample_lu(K, u)
    s2 = f(Kd, seed=4, precision=precision)
    torch.cuda.synchronize()
    r2 = s2.result()
    assert r2["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE) == 0, r2
    tol = 1e-10 if precision == "fp64" else 1e-6
    compare_draw(s2.keep.cpu().numpy(), r2["logp"], None, ref, u, logp_rtol=tol)


def test_withheld_block_complex_lu_times_out_and_next_draw_is_exact(dpp):
    """The complex LU path: CTA 0 never publishes its outer block, the other
    CTAs' waits run out after 5 ms, and the next draw is the oracle's."""
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 500
    K, _ = W.lu_similarity_kernel(n, seed=19, complex_=True)
    Kd = torch.from_numpy(K).cuda()
    s, dt = _withheld(dpp, lambda: dpp.sample_lu(Kd, seed=2, precision="3xtf32"))
    r = s.result()
    assert r["status"] & _lib.DPP_RES_TIMEOUT, r
    assert dt < 10.0, dt
    u = O.uniforms(2, 0, n)
    ref = O.sample_lu(K, u)
    s2 = dpp.sample_lu(Kd, seed=2, precision="3xtf32")
    torch.cuda.synchronize()
    r2 = s2.result()
    assert r2["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE) == 0, r2
    compare_draw(s2.keep.cpu().numpy(), r2["logp"], None, ref, u, logp_rtol=1e-6)
