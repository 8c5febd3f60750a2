"""Comparison helpers for CUDA-vs-oracle parity tests.

A draw is compared decision by decision up to its first borderline pivot: a
pivot whose uniform is within ``gap`` of the oracle's conditional probability
(|u_j - d_j| <= gap) may legitimately be decided either way by arithmetic that
differs only in rounding order, and every later decision depends on it.
"""
import numpy as np

BORDER_GAP = 1e-9  # |u_j - d_j| below which a decision counts as borderline
LOGP_RTOL = 1e-10  # FP64 path: relative log P(Y) tolerance


def pre_decision_pivots(draw) -> np.ndarray:
    """Oracle pivots before their decisions (rejections had 1 subtracted)."""
    piv = np.real(np.asarray(draw.pivots))
    return np.where(draw.keep == 1, piv, piv + 1.0)


def first_borderline(draw, u, gap=BORDER_GAP) -> int:
    """Index of the first borderline decision of an oracle draw (n if none)."""
    pre = pre_decision_pivots(draw)
    idx = np.flatnonzero(np.abs(np.asarray(u) - pre) <= gap)
    return int(idx[0]) if len(idx) else len(pre)


def compare_draw(gpu_keep, gpu_logp, gpu_pivots, draw, u, logp_rtol=LOGP_RTOL,
                 piv_atol=1e-9, gap=BORDER_GAP):
    """Assert parity; returns (n_compared, borderline?)."""
    n = len(draw.keep)
    gpu_keep = np.asarray(gpu_keep)
    j0 = first_borderline(draw, u, gap)
    assert np.array_equal(gpu_keep[:j0], draw.keep[:j0]), (
        "decision mismatch at", int(np.flatnonzero(gpu_keep[:j0] != draw.keep[:j0])[0]))
    if gpu_pivots is not None:
        gp = np.asarray(gpu_pivots)
        op = np.asarray(draw.pivots)
        if np.iscomplexobj(op) and not np.iscomplexobj(gp):
            gp = gp[0::2] + 1j * gp[1::2]
        err = np.abs(gp[:j0] - op[:j0])
        assert np.all(err <= piv_atol), ("pivot error", float(err.max()), int(err.argmax()))
    if j0 == n:
        assert abs(gpu_logp - draw.logp) <= logp_rtol * max(1.0, abs(draw.logp)), (
            gpu_logp, draw.logp)
    return j0, j0 < n
