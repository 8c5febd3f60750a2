"""Parity of the FP64 CUDA path (through the C ABI) with the FP64 oracle.

Decisions must match bit for bit up to the first borderline pivot
(|u_j - d_j| <= 1e-9), and log P(Y) within 1e-10 relative on every draw with
no borderline pivot. Sizes span several 32-wide panels and ragged tails.
"""
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


def _dev(K):
    import torch
    return torch.from_numpy(np.ascontiguousarray(K)).to("cuda")


def _run(dpp, K, seed, inst=0, lu=False, factor=False, uniforms=None):
    import torch
    f = dpp.sample_lu if lu else dpp.sample_hermitian
    s = f(_dev(K), seed=seed, instance=inst, precision="fp64", factor=factor, uniforms=uniforms)
    torch.cuda.synchronize()
    return s


def test_uniforms_bit_identical_to_oracle(dpp):
    for seed, inst in [(0, 0), (1, 0), (12345, 7), (2**40 + 3, 2**33 + 5)]:
        g = dpp.uniforms(seed, inst, 70001).cpu().numpy()
        o = O.uniforms(seed, inst, 70001)
        assert np.array_equal(g.view(np.uint64), o.view(np.uint64))


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 65, 100, 257])
def test_hermitian_real_parity_sizes(dpp, n):
    K = W.hermitian_kernel(n, seed=n, kind="uniform")
    for seed in range(3):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_ldl(K, u)
        s = _run(dpp, K, seed)
        r = s.result()
        assert r["status"] == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u)
        assert r["n_kept"] == int(s.keep.sum().item())


def test_config_n512_256_draws(dpp):
    """K = Q diag(U(0,1)) Q^T, n = 512, Philox seeds 0..255 (all oracle-checked)."""
    n = 512
    K = W.hermitian_kernel(n, seed=0, kind="uniform")
    borderline = 0
    for seed in range(256):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_ldl(K, u)
        s = _run(dpp, K, seed)
        r = s.result()
        assert r["status"] == 0
        _, b = compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u)
        borderline += b
    assert borderline <= 2


def test_exhaustive_n10_every_path(dpp):
    """Forced decisions through explicit uniforms: for all 1024 subsets the GPU
    likelihood equals |det(K - 1_{Y^c})|."""
    import torch
    n = 10
    K = W.hermitian_kernel(n, seed=0, kind="uniform")
    p = O.enumerate_probs(K)
    Kd = _dev(K)
    for mask in range(1 << n):
        keep = np.array([(mask >> j) & 1 for j in range(n)], dtype=np.uint8)
        u = torch.from_numpy(O.forced_uniforms(keep)).cuda()
        s = dpp.sample_hermitian(Kd, uniforms=u)
        r = s.result()
        assert np.array_equal(s.keep.cpu().numpy(), keep)
        assert abs(np.exp(r["logp"]) - p[mask]) < 1e-12


def test_explicit_uniforms_equal_philox(dpp):
    import torch
    n = 200
    K = W.hermitian_kernel(n, seed=3, kind="beta")
    a = _run(dpp, K, seed=9, inst=4)
    u = torch.from_numpy(O.uniforms(9, 4, n)).cuda()
    b = _run(dpp, K, seed=0, uniforms=u)
    assert torch.equal(a.keep, b.keep)
    assert a.logp == b.logp


@pytest.mark.parametrize("n", [33, 130])
def test_hermitian_complex_parity(dpp, n):
    K = W.hermitian_kernel(n, seed=n + 1, kind="beta", complex_=True)
    for seed in range(3):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_ldl(K, u)
        s = _run(dpp, K, seed)
        r = s.result()
        assert r["status"] == 0, r
        compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u)


@pytest.mark.parametrize("n,complex_", [(33, False), (150, False), (70, True)])
def test_lu_parity_and_similarity_twin(dpp, n, complex_):
    K, S = W.lu_similarity_kernel(n, seed=n, complex_=complex_)
    for seed in range(3):
        u = O.uniforms(seed, 0, n)
        ref = O.sample_lu(K, u)
        s = _run(dpp, K, seed, lu=True)
        r = s.result()
        assert r["status"] == 0, r
        j0, _ = compare_draw(s.keep.cpu().numpy(), r["logp"], s.pivots.cpu().numpy(), ref, u,
                             piv_atol=1e-8)
        h = _run(dpp, S, seed)
        if j0 == n:
            assert np.array_equal(h.keep.cpu().numpy(), s.keep.cpu().numpy())
            assert abs(h.logp - r["logp"]) <= 1e-9 * abs(r["logp"])


def test_factor_out_is_oracle_factor(dpp):
    n = 97
    K = W.hermitian_kernel(n, seed=5)
    u = O.uniforms(2, 0, n)
    ref = O.sample_ldl(K, u)
    s = _run(dpp, K, 2, factor=True)
    F = s.factor.cpu().numpy()
    assert np.allclose(np.tril(F), np.tril(ref.A), atol=1e-10)
    K2, _ = W.lu_similarity_kernel(n, seed=6)
    ref2 = O.sample_lu(K2, u)
    s2 = _run(dpp, K2, 2, lu=True, factor=True)
    assert np.allclose(s2.factor.cpu().numpy(), ref2.A, atol=1e-9)


def test_in_place_factorization(dpp):
    import torch
    n = 70
    K = W.hermitian_kernel(n, seed=7)
    Kd = _dev(K).t().contiguous().t()  # column-major storage
    from paper_1905_00165_gb300 import _lib
    L = dpp.load()
    keep = torch.empty(n, dtype=torch.uint8, device="cuda")
    raw = torch.zeros(32, dtype=torch.uint8, device="cuda")
    need = dpp.workspace_size(0, n, 0, 0, 1)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    st = L.dpp_sample_hermitian(Kd.data_ptr(), n, n, 0, 0, 1, 0, None, keep.data_ptr(),
                                Kd.data_ptr(), None, raw.data_ptr(), ws.data_ptr(), need,
                                torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    ref = O.sample_ldl(K, O.uniforms(1, 0, n))
    assert np.array_equal(keep.cpu().numpy(), ref.keep)
    assert np.allclose(np.tril(Kd.cpu().numpy()), np.tril(ref.A), atol=1e-10)


def test_projection_and_spanning_trees(dpp):
    n = 400
    K = W.hermitian_kernel(n, seed=1, kind="projection")
    for seed in range(4):
        assert int(_run(dpp, K, seed).keep.sum().item()) == n // 4
    d = 12
    K, edges, V = W.ust_grid_kernel(d)
    ref = -W.grid_spanning_tree_log_count(d)
    for seed in range(4):
        s = _run(dpp, K, seed)
        keep = s.keep.cpu().numpy().astype(bool)
        assert O.is_spanning_tree(edges[keep], V)
        assert abs(s.logp - ref) < 1e-8 * abs(ref)


def test_empty_and_leading_dimension(dpp):
    import torch
    z = torch.zeros((0, 0), dtype=torch.float64, device="cuda")
    s = dpp.sample_hermitian(z)
    r = s.result()
    assert r["status"] == 0 and r["logp"] == 0.0 and r["n_kept"] == 0
    n = 45
    K = W.hermitian_kernel(n, seed=2)
    cm = torch.zeros((n, 64), dtype=torch.float64, device="cuda")
    cm[:, :n] = torch.from_numpy(K.T.copy()).cuda()
    Kcm = cm.t()[:n, :]  # element (i, j) at i + 64 j
    assert Kcm.stride() == (1, 64)
    s = dpp.sample_hermitian(Kcm, seed=3)
    ref = O.sample_ldl(K, O.uniforms(3, 0, n))
    assert np.array_equal(s.keep.cpu().numpy(), ref.keep)


def test_diagonal_kernel_is_independent_bernoulli(dpp):
    n = 300
    K = W.diagonal_kernel(n, seed=4)
    u = O.uniforms(8, 0, n)
    s = _run(dpp, K, 8)
    assert np.array_equal(s.keep.cpu().numpy(), (u < np.diag(K)).astype(np.uint8))


def test_inadmissible_and_nonfinite_are_reported(dpp):
    from paper_1905_00165_gb300 import _lib
    n = 64
    # a first diagonal entry above one is an out-of-range first pivot
    K2 = W.hermitian_kernel(n, seed=1)
    K2[0, 0] = 1.7
    r2 = _run(dpp, K2, 0).result()
    assert r2["status"] & _lib.DPP_RES_INADMISSIBLE and r2["n_out_of_range"] >= 1
    K3 = W.hermitian_kernel(n, seed=1)
    K3[40, 3] = np.nan
    K3[3, 40] = np.nan
    r3 = _run(dpp, K3, 0).result()
    assert r3["status"] & _lib.DPP_RES_NONFINITE
