"""dpp_sample_hermitian_static (no workspace, no device allocation) against
dpp_sample_hermitian at FP64 on the same arguments.

Collected last so that it also runs after every other GPU test has used the
library in the same process; it must pass alone in a fresh process as well.
Each case makes two static calls in a row into preallocated outputs and checks
both against the workspace entry point: keep identical, pivots, log P and the
factor within the parity tolerance (1e-10 relative).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def dpp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as m
    return m


def _outputs(dpp, n, dtype):
    import torch
    fac = dpp.empty_colmajor(n, dtype, "cuda")
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    piv = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    raw = torch.zeros(dpp._lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    return fac, keep, piv, raw


def _colmajor(K):
    return K.t().contiguous().t()


def _check_same(dpp, ref, keep, piv, fac, raw, n):
    import torch
    torch.cuda.synchronize()
    r0 = ref.result()
    r1 = dpp._lib.decode_result(bytes(raw.cpu().numpy().tobytes()))
    assert r1["status"] == r0["status"]
    assert r1["n_kept"] == r0["n_kept"]
    assert torch.equal(keep[:n].cpu(), ref.keep[:n].cpu())
    p0 = ref.pivots[:n].cpu().numpy()
    p1 = piv[:n].cpu().numpy()
    np.testing.assert_allclose(p1, p0, rtol=RTOL, atol=0)
    assert abs(r1["logp"] - r0["logp"]) <= RTOL * max(1.0, abs(r0["logp"]))
    f0 = torch.tril(ref.factor).cpu().numpy()
    f1 = torch.tril(fac).cpu().numpy()
    np.testing.assert_allclose(f1, f0, rtol=RTOL, atol=1e-14)


@pytest.mark.parametrize("n,complex_", [(300, False), (130, True)])
def test_static_matches_workspace_entry_two_calls(dpp, n, complex_):
    import torch
    K = W.hermitian_kernel(n, seed=11 + n, complex_=complex_)
    Kd = _colmajor(torch.from_numpy(K).to("cuda"))
    fac, keep, piv, raw = _outputs(dpp, n, Kd.dtype)
    draws = [(5, 0), (77, 3)]
    refs = [dpp.sample_hermitian(Kd, seed=s, instance=i, precision="fp64", factor=True)
            for s, i in draws]
    for (s, i), ref in zip(draws, refs):
        dpp.sample_hermitian_static(Kd, fac, keep, piv, raw, seed=s, instance=i)
        _check_same(dpp, ref, keep, piv, fac, raw, n)


def test_static_in_place_and_no_device_allocation(dpp):
    import torch
    n = 257
    K = W.hermitian_kernel(n, seed=3, kind="beta")
    Kd = _colmajor(torch.from_numpy(K).to("cuda"))
    ref = dpp.sample_hermitian(Kd, seed=9, instance=1, precision="fp64", factor=True)
    fac, keep, piv, raw = _outputs(dpp, n, Kd.dtype)
    # first call: per-device set-up (symbol lookup) happens here
    dpp.sample_hermitian_static(Kd, fac, keep, piv, raw, seed=9, instance=1)
    _check_same(dpp, ref, keep, piv, fac, raw, n)
    for _ in range(2):
        work = Kd.clone().t().contiguous().t()  # in place: factor_out == K
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        dpp.sample_hermitian_static(work, work, keep, piv, raw, seed=9, instance=1)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0
        _check_same(dpp, ref, keep, piv, work, raw, n)


def test_static_rejects_sizes_above_limit_and_missing_factor(dpp):
    import torch
    L = dpp._lib.load()
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    keep = torch.zeros(64, dtype=torch.uint8, device="cuda")
    raw = torch.zeros(dpp._lib.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    p = buf.data_ptr()
    for dt, nmax in [(dpp._lib.DPP_R64, dpp._lib.DPP_STATIC_MAX_N_R64),
                     (dpp._lib.DPP_C128, dpp._lib.DPP_STATIC_MAX_N_C128)]:
        n = nmax + 1
        st = L.dpp_sample_hermitian_static(p, n, n, dt, 0, 0, None, keep.data_ptr(), p, None,
                                           raw.data_ptr(), None)
        assert st == dpp._lib.DPP_ERR_WORKSPACE
        msg = dpp._lib.last_error()
        assert "limit" in msg and str(dpp._lib.DPP_STATIC_SCRATCH_BYTES) in msg
    st = L.dpp_sample_hermitian_static(p, 4, 4, dpp._lib.DPP_R64, 0, 0, None, keep.data_ptr(),
                                       None, None, raw.data_ptr(), None)
    assert st == dpp._lib.DPP_ERR_INVALID_ARG
    assert "factor_out" in dpp._lib.last_error()
