"""Parity at the measured sizes, where the CPU oracle is too slow to run.

* Uniform spanning trees of the 64 x 64 grid (n = 8064, rank 4095) on the mixed
  path: every draw is a spanning tree and log P(Y) = -log(number of spanning
  trees), from Kirchhoff's theorem (Section 4; the same closed form reproduces
  the paper's 40 x 40 likelihood in the oracle pins).
* Projection kernels of order 4096 and rank 1024: |Y| = rank on every draw
  (Section 3), on both paths.
* n = 16384, Beta(1/2, 1/2) spectrum: the mixed path draws the same set as the
  FP64 GPU path (itself oracle-checked at smaller orders) up to the first
  pivot within 1e-9 of its uniform, and log P agrees to the mixed tolerance.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

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


def test_spanning_trees_64x64_grid_mixed(dpp):
    import torch
    from paper_1905_00165_gb300 import _lib
    d = 64
    K, edges, V = W.ust_grid_kernel(d, device="cuda")
    Kd = torch.from_numpy(K).cuda().contiguous()
    ref = -W.grid_spanning_tree_log_count(d)
    assert abs(ref - (-4662.6413)) < 1e-3
    for seed in range(4):
        s = _draw(dpp, Kd, seed, "bf16x6")
        r = s.result()
        assert r["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE) == 0, r
        keep = s.keep.cpu().numpy().astype(bool)
        assert keep.sum() == V - 1
        assert O.is_spanning_tree(edges[keep], V)
        assert abs(r["logp"] - ref) <= MIXED_LOGP_RTOL * abs(ref), (r["logp"], ref)


@pytest.mark.parametrize("precision", ["bf16x6", "fp64"])
def test_projection_rank_4096(dpp, precision):
    n = 4096
    Kd = W.hermitian_kernel(n, seed=1, kind="projection", device="cuda",
                            return_torch=True).contiguous()
    for seed in range(3):
        s = _draw(dpp, Kd, seed, precision)
        assert int(s.keep.sum().item()) == n // 4


def test_mixed_matches_fp64_path_n16384(dpp):
    import torch
    from paper_1905_00165_gb300 import _lib
    n = 16384
    Kd = W.hermitian_kernel(n, seed=0, kind="beta", device="cuda",
                            return_torch=True).contiguous()
    for seed in (0, 1):
        ref = _draw(dpp, Kd, seed, "fp64")
        mix = _draw(dpp, Kd, seed, "bf16x6")
        rr, rm = ref.result(), mix.result()
        assert rm["status"] & (_lib.DPP_RES_TIMEOUT | _lib.DPP_RES_NONFINITE
                               | _lib.DPP_RES_RECOMPUTE) == 0, rm
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

