"""Parity at n = 16384 in the launch configuration the bench times.

Collected after the other GPU test files (and before the allocation-free
entry's test, which must come last): 3xTF32, each launch capped at a quarter
of the SMs, four draws in flight on four streams, against the FP64 path.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

MIXED_LOGP_RTOL = 1e-6


@pytest.fixture(scope="module")
def dpp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as m
    return m


def _draw(dpp, Kd, seed, precision):
    import torch
    s = dpp.sample_hermitian(Kd, seed=seed, precision=precision)
    torch.cuda.synchronize()
    return s


def test_bench_launch_configuration_n16384(dpp):
    """n = 16384 in the launch configuration the bench times: 3xTF32, each
    launch capped at a quarter of the SMs (so the single-helper panel pipeline
    runs), four draws issued on four streams at once. Every draw equals the
    FP64 path's up to its first pivot within 1e-9 of its uniform, and log P
    agrees to the mixed tolerance."""
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 16384
    Kd = W.hermitian_kernel(n, seed=0, kind="beta", device="cuda",
                            return_torch=True).contiguous()
    seeds = [0, 1, 2, 3]
    refs = [_draw(dpp, Kd, s, "fp64") for s in seeds]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    old = _lib.get_tuning(_lib.DPP_TUNE_MAX_CTAS)
    _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, max(8, sms // 4))
    try:
        streams = [torch.cuda.Stream() for _ in seeds]
        mix = []
        for s, st in zip(seeds, streams):
            with torch.cuda.stream(st):
                mix.append(dpp.sample_hermitian(Kd, seed=s, precision="3xtf32"))
        torch.cuda.synchronize()
    finally:
        _lib.set_tuning(_lib.DPP_TUNE_MAX_CTAS, old)
    for s, ref, m in zip(seeds, refs, mix):
        rr, rm = ref.result(), m.result()
        assert rm["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE
                               | _lib.DPP_RES_RECOMPUTE) == 0, rm
        u = dpp.uniforms(s, 0, n).cpu().numpy()
        kr = ref.keep.cpu().numpy()
        pr = ref.pivots.cpu().numpy()
        pre = np.where(kr == 1, pr, pr + 1.0)
        close = np.flatnonzero(np.abs(u - pre) <= 1e-9)
        j0 = int(close[0]) if len(close) else n
        km = m.keep.cpu().numpy()
        assert np.array_equal(km[:j0], kr[:j0]), int(np.flatnonzero(km[:j0] != kr[:j0])[0])
        if j0 == n:
            assert abs(rm["logp"] - rr["logp"]) <= MIXED_LOGP_RTOL * abs(rr["logp"])
