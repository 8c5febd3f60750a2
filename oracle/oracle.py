"""FP64 CPU oracle for the factorization-based DPP sampler (arXiv:1905.00165).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the library under
``paper_1905_00165_gb300`` never does, and this module imports nothing from it.

Two kinds of function live here:

* ctypes wrappers over ``dpp_oracle.c`` — Algorithm 1 (LU form, real and
  complex), its Hermitian LDL^H specialisation, the greedy maximum-likelihood
  variant, Algorithm 2 (the elementary sampler of projection kernels), and the
  Philox4x32-10 uniforms (the counter-based generator both
  sides implement independently from its published definition);
* closed forms written from their plain definitions with numpy library
  primitives (det, solve, inv):
    - ``subset_logprob``: P(Y) = |det(K - 1_{Y^c})| (Theorem 1 and the proof of
      Prop. 1 that follows Algorithm 1);
    - ``conditional_pivot``: the pivot d_j = K_jj - K_{j,P} (K_P - 1_G)^{-1}
      K_{P,j}, P = [0, j), G = rejected indices of P (Props. 3-5);
    - ``logprob_grad``: d log|det A| / dK = A^{-H}, A = K - 1_{Y^c} (the
      differential of the likelihood of Theorem 1, Y held fixed).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpp_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libdpp_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile dpp_oracle.c with gcc (OpenMP, IEEE FP64, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i64, dp, u8p = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
    lib.oracle_philox4x32_10.argtypes = [dp, dp, dp]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_uniform.restype = ctypes.c_double
    lib.oracle_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, i64, dp]
    lib.oracle_uniforms.restype = None
    for name in ("oracle_dpp_lu_r64", "oracle_dpp_lu_c128",
                 "oracle_dpp_ldl_r64", "oracle_dpp_ldl_c128"):
        f = getattr(lib, name)
        f.argtypes = [i64, dp, i64, dp, u8p, dp, dp]
        f.restype = i64
    lib.oracle_dpp_ldl_greedy_r64.argtypes = [i64, dp, i64, u8p, dp, dp]
    lib.oracle_dpp_ldl_greedy_r64.restype = i64
    lib.oracle_dpp_elementary_r64.argtypes = [i64, dp, i64, i64, dp, dp, dp, dp, dp]
    lib.oracle_dpp_elementary_r64.restype = ctypes.c_int
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


# --------------------------------------------------------------------------
# Philox4x32-10 uniforms
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Raw Philox4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniforms(seed: int, instance: int, n: int) -> np.ndarray:
    """u_j = ((x0 << 21 | x1 >> 11) + 0.5) 2^-53, x = Philox(ctr=(j, inst), key=seed)."""
    u = np.zeros(n, dtype=np.float64)
    _load().oracle_uniforms(seed, instance, n, _ptr(u))
    return u


# --------------------------------------------------------------------------
# Algorithm 1 and its Hermitian specialisation
# --------------------------------------------------------------------------
class Draw:
    """One oracle draw: keep mask, final pivots, log-likelihood, factored A."""

    def __init__(self, keep, pivots, logp, A):
        self.keep = keep
        self.pivots = pivots
        self.logp = logp
        self.A = A

    @property
    def sample(self) -> np.ndarray:
        return np.flatnonzero(self.keep)


def _prep(K: np.ndarray, dtype) -> np.ndarray:
    K = np.asarray(K)
    assert K.ndim == 2 and K.shape[0] == K.shape[1]
    return np.array(K, dtype=dtype, order="F", copy=True)


def sample_lu(K: np.ndarray, u: np.ndarray) -> Draw:
    """Algorithm 1 on a (possibly non-Hermitian) kernel K with uniforms u."""
    cplx = np.iscomplexobj(K)
    A = _prep(K, np.complex128 if cplx else np.float64)
    n = A.shape[0]
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.shape == (n,)
    keep = np.zeros(n, dtype=np.uint8)
    piv = np.zeros(n, dtype=A.dtype)
    lp = np.zeros(1)
    f = _load().oracle_dpp_lu_c128 if cplx else _load().oracle_dpp_lu_r64
    f(n, _ptr(A), n, _ptr(u), _ptr(keep), _ptr(piv), _ptr(lp))
    return Draw(keep, piv, float(lp[0]), A)


def sample_ldl(K: np.ndarray, u: np.ndarray) -> Draw:
    """Hermitian (LDL^H) form of Algorithm 1; reads the lower triangle of K."""
    cplx = np.iscomplexobj(K)
    A = _prep(K, np.complex128 if cplx else np.float64)
    n = A.shape[0]
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.shape == (n,)
    keep = np.zeros(n, dtype=np.uint8)
    piv = np.zeros(n, dtype=np.float64)
    lp = np.zeros(1)
    f = _load().oracle_dpp_ldl_c128 if cplx else _load().oracle_dpp_ldl_r64
    f(n, _ptr(A), n, _ptr(u), _ptr(keep), _ptr(piv), _ptr(lp))
    return Draw(keep, piv, float(lp[0]), A)


def greedy_ldl(K: np.ndarray) -> Draw:
    """Greedy maximum-likelihood variant (keep iff d_j > 1/2), real Hermitian."""
    A = _prep(K, np.float64)
    n = A.shape[0]
    keep = np.zeros(n, dtype=np.uint8)
    piv = np.zeros(n, dtype=np.float64)
    lp = np.zeros(1)
    _load().oracle_dpp_ldl_greedy_r64(n, _ptr(A), n, _ptr(keep), _ptr(piv), _ptr(lp))
    return Draw(keep, piv, float(lp[0]), A)


class ElementaryDraw:
    """One draw of Algorithm 2: the k sampled indices in selection order, the
    Cholesky factor of K_Y in that order, log P(Y) and whether every pivot was
    positive."""

    def __init__(self, n, sample, chol, logp, ok, margin):
        self.n = n
        self.margin = margin
        self.sample = sample
        self.chol = chol
        self.logp = logp
        self.ok = ok

    @property
    def keep(self) -> np.ndarray:
        m = np.zeros(self.n, dtype=np.uint8)
        m[self.sample] = 1
        return m


def sample_elementary(K: np.ndarray, k: int, u: np.ndarray) -> ElementaryDraw:
    """Algorithm 2 (Theorem 2) on a real symmetric projection K of rank k with
    one uniform per step (u[0:k])."""
    A = _prep(K, np.float64)
    n = A.shape[0]
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.shape[0] >= k and 0 <= k <= n
    sample = np.zeros(max(k, 1), dtype=np.int64)
    chol = np.zeros((max(k, 1), max(k, 1)), dtype=np.float64, order="F")
    lp = np.zeros(1)
    margin = np.zeros(max(k, 1))
    rc = _load().oracle_dpp_elementary_r64(n, _ptr(A), n, k, _ptr(u), _ptr(sample), _ptr(chol),
                                           _ptr(lp), _ptr(margin))
    return ElementaryDraw(n, sample[:k].copy(), np.array(chol[:k, :k]), float(lp[0]), rc == 0,
                          margin[:k].copy())


def forced_uniforms(keep: np.ndarray) -> np.ndarray:
    """Uniforms that force the decisions ``keep`` (keep iff u < Re d)."""
    keep = np.asarray(keep).astype(bool)
    return np.where(keep, -1e300, 1e300).astype(np.float64)


# --------------------------------------------------------------------------
# Closed forms (plain definitions, numpy library primitives)
# --------------------------------------------------------------------------
def complement_shift(K: np.ndarray, keep: np.ndarray) -> np.ndarray:
    """A = K - 1_{Y^c}: subtract 1 from the diagonal entries not in Y."""
    keep = np.asarray(keep).astype(bool)
    A = np.array(K, dtype=np.complex128 if np.iscomplexobj(K) else np.float64)
    idx = np.flatnonzero(~keep)
    A[idx, idx] -= 1.0
    return A


def subset_logprob(K: np.ndarray, keep: np.ndarray) -> float:
    """log P(Y) = log|det(K - 1_{Y^c})| (Theorem 1; proof of Prop. 1)."""
    sign, logabs = np.linalg.slogdet(complement_shift(K, keep))
    return float(logabs)


def subset_prob(K: np.ndarray, keep: np.ndarray) -> float:
    return float(abs(np.linalg.det(complement_shift(K, keep))))


def enumerate_probs(K: np.ndarray) -> np.ndarray:
    """P(Y) for all 2^n subsets; index bit j set <=> j in Y."""
    n = K.shape[0]
    probs = np.zeros(1 << n)
    for mask in range(1 << n):
        keep = np.array([(mask >> j) & 1 for j in range(n)], dtype=np.uint8)
        probs[mask] = subset_prob(K, keep)
    return probs


def mask_index(keep: np.ndarray) -> int:
    return int(sum(int(b) << j for j, b in enumerate(np.asarray(keep))))


def conditional_pivot(K: np.ndarray, keep_prefix: np.ndarray, j: int,
                      hermitian: bool = True) -> complex:
    """Pivot d_j given the decisions on [0, j) (Props. 3-5):
    d_j = K_jj - K_{j,P} (K_P - 1_G)^{-1} K_{P,j}, P = [0, j).

    With ``hermitian`` the kernel is read from its lower triangle only.
    Returns the pivot BEFORE the decision at j.
    """
    K = np.asarray(K)
    if hermitian:
        Kl = np.tril(K)
        K = Kl + np.tril(K, -1).conj().T
    if j == 0:
        return K[0, 0]
    A = complement_shift(K[:j, :j], np.asarray(keep_prefix)[:j])
    x = np.linalg.solve(A, K[:j, j])
    return K[j, j] - K[j, :j] @ x


def logprob_grad(K: np.ndarray, keep: np.ndarray, g: float = 1.0) -> np.ndarray:
    """g * d log|det(K - 1_{Y^c})| / dK = g * (K - 1_{Y^c})^{-H}."""
    A = complement_shift(K, keep)
    return g * np.linalg.inv(A).conj().T


def is_spanning_tree(edges: np.ndarray, n_vertices: int) -> bool:
    """Union-find check: |edges| = V - 1 and no cycle."""
    if len(edges) != n_vertices - 1:
        return False
    parent = list(range(n_vertices))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in edges:
        ra, rb = find(int(a)), find(int(b))
        if ra == rb:
            return False
        parent[ra] = rb
    return True
