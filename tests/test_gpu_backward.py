"""Adjoint of log P(Y) (dK = g (K - 1_{Y^c})^{-H}) through the C ABI, against
the oracle's closed form (a library inverse) and finite differences."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_00165_gb300 as m
    return m


def _kernel(n, herm, cplx, seed):
    if herm:
        return W.hermitian_kernel(n, seed=seed, kind="beta", complex_=cplx)
    K, _ = W.lu_similarity_kernel(n, seed=seed, complex_=cplx)
    return K


@pytest.mark.parametrize("herm", [True, False])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [1, 33, 100, 257])
def test_backward_matches_closed_form(dpp, n, herm, cplx):
    import torch
    K = _kernel(n, herm, cplx, seed=n + 7)
    keep = (O.sample_ldl(K, O.uniforms(3, 0, n)) if herm else O.sample_lu(K, O.uniforms(3, 0, n))).keep
    g = 0.75
    ref = O.logprob_grad(K, keep, g)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).cuda()
    dK = dpp.logprob_backward(Kd, torch.from_numpy(keep).cuda(),
                              torch.tensor(g, dtype=torch.float64, device="cuda"), hermitian=herm)
    got = dK.cpu().numpy()
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(got - ref)) <= 1e-9 * scale, np.max(np.abs(got - ref))


def test_autograd_function_gradcheck(dpp):
    import torch
    n = 12
    K, _ = W.lu_similarity_kernel(n, seed=3)
    keep = torch.from_numpy(O.sample_lu(K, O.uniforms(0, 0, n)).keep).cuda()
    Kt = torch.from_numpy(K).cuda().requires_grad_(True)
    f = lambda X: dpp.DPPLogProb.apply(X, keep, False)
    assert torch.autograd.gradcheck(f, (Kt,), eps=1e-6, atol=1e-6, rtol=1e-5)
    # the forward value is log|det(K - 1_{Y^c})|
    assert abs(float(f(Kt)) - O.subset_logprob(K, keep.cpu().numpy())) < 1e-10


def test_hermitian_symmetric_perturbation_fd(dpp):
    import torch
    n = 40
    K = W.hermitian_kernel(n, seed=4, kind="uniform")
    keep_np = O.sample_ldl(K, O.uniforms(1, 0, n)).keep
    keep = torch.from_numpy(keep_np).cuda()
    Kt = torch.from_numpy(K).cuda().requires_grad_(True)
    lp = dpp.DPPLogProb.apply(Kt, keep, True)
    lp.backward()
    G = Kt.grad.cpu().numpy()
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(10):
        i, j = rng.integers(0, n, 2)
        E = np.zeros_like(K)
        E[i, j] += 1.0
        if i != j:
            E[j, i] += 1.0
        fd = (O.subset_logprob(K + h * E, keep_np) - O.subset_logprob(K - h * E, keep_np)) / (2 * h)
        an = G[i, j] + (G[j, i] if i != j else 0.0)
        assert abs(fd - an) < 1e-6 * max(1.0, abs(fd))
