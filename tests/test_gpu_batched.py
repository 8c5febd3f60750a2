"""Batched persistent-launch sampler against the FP64 oracle: every instance
draws the oracle's set (up to the first borderline decision, |u - d| <= 1e-9)
with log P(Y) within 1e-6 relative (FP32 working precision)."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
from tests._parity import compare_draw, pre_decision_pivots

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[128, 256], ids=["threads128", "threads256"])
def dpp(request):
    """The library, with the batched sampler's CTAs of 128 or 256 threads
    (DPP_TUNE_BATCHED_THREADS)."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as m
    from paper_1905_00165_gb300 import _lib
    old = _lib.get_tuning(_lib.DPP_TUNE_BATCHED_THREADS)
    _lib.set_tuning(_lib.DPP_TUNE_BATCHED_THREADS, request.param)
    yield m
    _lib.set_tuning(_lib.DPP_TUNE_BATCHED_THREADS, old)


def _to_dev(Ks):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(K)).cuda() for K in Ks]


def test_batched_parity_uneven_sizes(dpp):
    import torch
    sizes = [1, 2, 31, 32, 33, 64, 65, 100, 129, 257, 300, 5, 47, 200, 96]
    Ks = [W.hermitian_kernel(m, seed=i + 1, kind=("beta" if i % 2 else "uniform"))
          for i, m in enumerate(sizes)]
    seed = 7
    b = dpp.sample_batched(_to_dev(Ks), seed=seed, want_pivots=True)
    torch.cuda.synchronize()
    res = b.results()
    for i, K in enumerate(Ks):
        n = K.shape[0]
        u = O.uniforms(seed, i, n)  # instance id = index
        ref = O.sample_ldl(K, u)
        r = res[i]
        assert r["status"] & ~4 == 0, (i, r)
        j0, border = compare_draw(b.keep[i][:n].cpu().numpy(), r["logp"],
                                  b.pivots[i][:n].cpu().numpy(), ref, u, logp_rtol=1e-6,
                                  piv_atol=1e-4)
        if not border:
            assert r["n_kept"] == int(ref.keep.sum()), (i, r["n_kept"], int(ref.keep.sum()))


def test_batched_parity_large_instances(dpp):
    """Instances of the batched workload's upper range (n in [512, 1024],
    L-ensembles and Haar kernels, ragged against the 32-wide panels) against
    the oracle, instance by instance."""
    import torch
    sizes = [1024, 512, 777, 1000, 640, 901, 1023, 513]
    Ks = [W.lensemble_kernel(m, seed=300 + i) if i % 2 == 0 else
          W.hermitian_kernel(m, seed=300 + i, kind="beta") for i, m in enumerate(sizes)]
    seed = 13
    b = dpp.sample_batched(_to_dev(Ks), seed=seed, want_pivots=True)
    torch.cuda.synchronize()
    res = b.results()
    for i, K in enumerate(Ks):
        n = K.shape[0]
        u = O.uniforms(seed, i, n)
        ref = O.sample_ldl(K, u)
        r = res[i]
        assert r["status"] & ~4 == 0, (i, r)
        j0, border = compare_draw(b.keep[i][:n].cpu().numpy(), r["logp"],
                                  b.pivots[i][:n].cpu().numpy(), ref, u, logp_rtol=1e-6,
                                  piv_atol=1e-4)
        if not border:
            assert r["n_kept"] == int(ref.keep.sum()), (i, r["n_kept"], int(ref.keep.sum()))


def test_batched_lensembles_and_instances(dpp):
    import torch
    Ks = W.lensemble_batch(24, seed=3, nmin=64, nmax=320)
    inst = [1000 + 3 * i for i in range(len(Ks))]
    b = dpp.sample_batched(_to_dev(Ks), seed=11, instance=inst)
    torch.cuda.synchronize()
    res = b.results()
    for i, K in enumerate(Ks):
        n = K.shape[0]
        u = O.uniforms(11, inst[i], n)
        ref = O.sample_ldl(K, u)
        compare_draw(b.keep[i][:n].cpu().numpy(), res[i]["logp"], None, ref, u, logp_rtol=1e-6)


def test_batched_forced_borderline_recompute(dpp):
    """Uniforms 1e-8 from the oracle pivots (keeping the oracle's decisions)
    force the CTA-local FP64 recompute; every decision must still match."""
    import torch
    sizes = [150, 300, 77]
    Ks = [W.hermitian_kernel(m, seed=50 + m, kind="beta") for m in sizes]
    us = []
    refs = []
    for i, K in enumerate(Ks):
        n = K.shape[0]
        u = O.uniforms(2, i, n)
        ref = O.sample_ldl(K, u)
        pre = pre_decision_pivots(ref)
        for j in range(3, n, max(1, n // 9)):
            u[j] = pre[j] - 1e-8 if ref.keep[j] else pre[j] + 1e-8
        ref2 = O.sample_ldl(K, u)
        assert np.array_equal(ref2.keep, ref.keep)
        us.append(torch.from_numpy(u))
        refs.append(ref2)
    b = dpp.sample_batched(_to_dev(Ks), seed=0, uniforms=us, want_pivots=True)
    torch.cuda.synchronize()
    res = b.results()
    for i, ref in enumerate(refs):
        n = len(ref.keep)
        assert res[i]["n_borderline"] >= 8, res[i]
        assert np.array_equal(b.keep[i][:n].cpu().numpy(), ref.keep)
        assert abs(res[i]["logp"] - ref.logp) <= 1e-6 * abs(ref.logp)


def test_batched_projection_rank_and_empty(dpp):
    import torch
    Ks = [W.hermitian_kernel(m, seed=m, kind="projection") for m in (64, 128, 200, 256)]
    b = dpp.sample_batched(_to_dev(Ks), seed=5)
    torch.cuda.synchronize()
    for i, K in enumerate(Ks):
        assert int(b.keep[i][:K.shape[0]].sum().item()) == K.shape[0] // 4
    e = dpp.sample_batched([], seed=0)
    assert e.batch == 0


def test_batched_adjoint_matches_closed_form(dpp):
    """dK_i of the batched adjoint (each instance's last draw fixed) against the
    oracle's closed form g_i (K_i - 1_{Y_i^c})^{-T}."""
    import torch
    Ks = W.lensemble_batch(6, seed=4, nmin=64, nmax=300)
    b = dpp.sample_batched(_to_dev(Ks), seed=3)
    g = torch.tensor([1.0, -0.5, 2.0, 0.25, 1.5, -1.0], dtype=torch.float64)
    dKs = b.logprob_backward(g)
    torch.cuda.synchronize()
    for i, K in enumerate(Ks):
        n = K.shape[0]
        keep = b.keep[i][:n].cpu().numpy()
        ref = O.logprob_grad(K, keep, float(g[i]))
        got = dKs[i].cpu().numpy()
        err = np.abs(got - ref).max() / max(1.0, np.abs(ref).max())
        assert err < 1e-9, (i, err)


def test_batched_adjoint_fp32_matches_closed_form(dpp):
    """The FP32 form of the batched adjoint (dpp_logprob_backward_batched_fp32)
    against the oracle's FP64 closed form, within FP32 inversion accuracy:
    ||dK - ref||_F <= 3e-5 cond(K - 1_{Y^c}) ||ref||_F."""
    import torch
    Ks = W.lensemble_batch(8, seed=5, nmin=32, nmax=400)
    b = dpp.sample_batched(_to_dev(Ks), seed=4)
    g = torch.tensor([1.0, -0.5, 2.0, 0.25, 1.5, -1.0, 0.75, 3.0], dtype=torch.float64)
    dKs = b.logprob_backward(g, precision="fp32")
    torch.cuda.synchronize()
    for i, K in enumerate(Ks):
        n = K.shape[0]
        keep = b.keep[i][:n].cpu().numpy()
        ref = O.logprob_grad(K, keep, float(g[i]))
        A = O.complement_shift(K, keep)
        cond = np.linalg.cond(A)
        got = dKs[i].cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 3e-5 * cond, (i, err, cond)
        assert np.allclose(got, got.T, atol=0.0)  # both triangles written


def _adjoint_call(dpp, Ks, keeps, g, ws_bytes):
    """dpp_logprob_backward_batched with an explicit workspace size."""
    import ctypes
    import torch
    from paper_1905_00165_gb300 import _lib
    L = dpp.load()
    B = len(Ks)
    ns = [int(K.shape[0]) for K in Ks]
    dKs = [dpp.empty_colmajor(m, torch.float64, "cuda") for m in ns]
    n_h = np.asarray(ns, dtype=np.int64)
    # symmetric K stored row-major: the same as column-major with ld = n
    ld_h = np.asarray([K.stride(0) if m else 1 for K, m in zip(Ks, ns)], dtype=np.int64)
    ldd_h = np.asarray([d.stride(1) if m else 1 for d, m in zip(dKs, ns)], dtype=np.int64)
    P = ctypes.c_void_p * B
    kp = P(*[K.data_ptr() for K in Ks])
    kk = P(*[k.data_ptr() for k in keeps])
    gp = P(*[g.data_ptr() + 8 * i for i in range(B)])
    dp = P(*[d.data_ptr() for d in dKs])
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    st = L.dpp_logprob_backward_batched(
        B, n_h.ctypes.data, ctypes.cast(kp, ctypes.c_void_p), ld_h.ctypes.data,
        ctypes.cast(kk, ctypes.c_void_p), ctypes.cast(gp, ctypes.c_void_p),
        ctypes.cast(dp, ctypes.c_void_p), ldd_h.ctypes.data, ws.data_ptr(), ws_bytes,
        torch.cuda.current_stream().cuda_stream)
    _lib.check(st)
    torch.cuda.synchronize()
    return [d.cpu().numpy() for d in dKs]


def test_batched_adjoint_one_launch_ragged_and_small_grid(dpp):
    """The one-launch adjoint on ragged orders (n = 1, 31, 33, 64, 65, 257, ...)
    against the closed form, with the full workspace and with one that fits
    two CTAs (more instances than CTAs); the single-instance entry point
    against the same closed form."""
    import torch
    from paper_1905_00165_gb300 import _lib
    sizes = [1, 31, 33, 64, 65, 100, 257, 300, 5, 129]
    Ks = [W.hermitian_kernel(m, seed=50 + i, kind="uniform") for i, m in enumerate(sizes)]
    Kd = [torch.from_numpy(np.ascontiguousarray(K)).cuda() for K in Ks]
    keeps_h = [O.sample_ldl(K, O.uniforms(2, i, K.shape[0])).keep for i, K in enumerate(Ks)]
    keeps = [torch.from_numpy(k).cuda() for k in keeps_h]
    g = torch.tensor([1.0, -0.5, 2.0, 0.25, 1.5, -1.0, 0.75, 3.0, -2.0, 0.5],
                     dtype=torch.float64, device="cuda")
    L = dpp.load()
    n_max = max(sizes)
    full = L.dpp_logprob_backward_batched_workspace(len(Ks), n_max)
    ldz = ((n_max + 31) // 32) * 32
    per_cta = 8 * (ldz * ldz + ldz * 32 + (ldz // 32) * 1024 + ldz + 32)
    two = full - (full // per_cta - 2) * per_cta  # room for exactly two CTAs
    assert two <= full
    outs = [_adjoint_call(dpp, Kd, keeps, g, w) for w in (full, two)]
    # and the single-instance entry point (a chain of launches per instance)
    outs.append([dpp.logprob_backward(K, k, grad_logp=g[i:i + 1]).cpu().numpy()
                 for i, (K, k) in enumerate(zip(Kd, keeps))])
    for i, K in enumerate(Ks):
        ref = O.logprob_grad(K, keeps_h[i], float(g[i]))
        scale = max(1.0, np.abs(ref).max())
        for out in outs:
            err = np.abs(out[i] - ref).max() / scale
            assert err < 1e-9, (i, sizes[i], err)
