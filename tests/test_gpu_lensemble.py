"""L-ensemble to marginal kernel on the device (Section 5):
K = L (L + I)^{-1} = I - (L + I)^{-1}, for a batch of kernels in one launch.

Checked against the definition written with numpy's inverse, against the
push-through form Phi (Phi^T Phi + I)^{-1} Phi^T of the workload generator,
and by sampling: the batched sampler on the converted kernels draws the
oracle's sets on the oracle's own conversion of the same L."""
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


def test_conversion_matches_closed_form(dpp):
    import torch
    sizes = [1, 31, 33, 64, 100, 257, 512, 777, 1024]
    Ls = [W.lensemble_L(m, seed=500 + i) for i, m in enumerate(sizes)]
    Ks = dpp.lensemble_to_marginal([torch.from_numpy(L).cuda() for L in Ls])
    torch.cuda.synchronize()
    for i, L in enumerate(Ls):
        n = L.shape[0]
        ref = L @ np.linalg.inv(L + np.eye(n))
        got = Ks[i].cpu().numpy()
        err = np.abs(got - ref).max()
        assert err < 1e-10, (sizes[i], err)
        assert np.array_equal(got, got.T)
        push = W.lensemble_kernel(n, seed=500 + i)
        assert np.abs(got - push).max() < 1e-9, sizes[i]
        lam = np.linalg.eigvalsh(got)
        assert lam.min() > -1e-10 and lam.max() < 1 + 1e-10


def test_converted_kernels_sample_like_the_oracle(dpp):
    import torch
    sizes = [64, 200, 513, 1024]
    Ls = [W.lensemble_L(m, seed=900 + i) for i, m in enumerate(sizes)]
    Ks = dpp.lensemble_to_marginal([torch.from_numpy(L).cuda() for L in Ls])
    b = dpp.sample_batched(Ks, seed=3)
    torch.cuda.synchronize()
    res = b.results()
    for i, L in enumerate(Ls):
        n = L.shape[0]
        Kref = L @ np.linalg.inv(L + np.eye(n))
        Kref = 0.5 * (Kref + Kref.T)
        u = O.uniforms(3, i, n)
        ref = O.sample_ldl(Kref, u)
        # the two conversions differ by rounding (~1e-14): decisions are compared
        # up to the first pivot within 1e-8 of its uniform
        compare_draw(b.keep[i][:n].cpu().numpy(), res[i]["logp"], None, ref, u,
                     logp_rtol=1e-6, gap=1e-8)
