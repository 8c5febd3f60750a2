"""Seeded synthetic marginal kernels shaped like the paper's workloads.

This module only GENERATES inputs; it holds none of the sampler's arithmetic and
is shared by the CUDA-path tests, the oracle tests and the benchmark. Every
generator is deterministic in its seed (numpy PCG64 Gaussians/uniforms); large
orthogonal factors may be computed with torch on a device, which changes only
rounding, never the distribution.

Kernels (all FP64 / complex128, returned as dense n x n arrays):

* ``hermitian_kernel``: K = Q diag(lam) Q^H with Q Haar-distributed (QR of a
  Gaussian matrix with the R-diagonal phase correction of Mezzadri 2007) and
  lam ~ Uniform(0,1), Beta(1/2,1/2), or {0,1} with exactly ``rank`` ones
  (a projection kernel). Hermitian kernels with spectrum in [0,1] are admissible
  (Macchi; Section 2 of the paper).
* ``ust_grid_kernel``: the transfer-current kernel K = B_r^T (B_r B_r^T)^{-1}
  B_r of the d x d grid graph (unit weights, vertex 0 grounded); DPP(K) is the
  uniform spanning-tree measure (Burton-Pemantle; Figure 1 of the paper).
* ``lu_similarity_kernel``: K = D^{-1} S D with S Hermitian as above and D a
  log-normal diagonal; diagonal similarity preserves every principal minor, so
  DPP(K) = DPP(S) (Prop. 2 of the paper).
* ``aztec_kernel``: the domino tilings of the Aztec diamond of order d as a
  DPP over the 4 d^2 edges of its dual graph: Kasteleyn weights (1 on
  horizontal, i on vertical adjacencies) and Kenyon's local-statistics formula
  K(e, e') = Kast(b, w) Kast^{-1}(w, b') for e = (b, w), e' = (b', w'); a
  complex, non-Hermitian projection of rank d (d + 1) whose draws are uniform
  tilings (Section 1 of the paper, the Aztec diamond figures).
* ``lensemble_kernel``: K = L (L + I)^{-1}, L = Phi Phi^T, Phi with unit-norm
  Gaussian rows scaled by LogUniform(0.1, 10) qualities, formed through the
  push-through identity K = Phi (Phi^T Phi + I)^{-1} Phi^T.
"""
from __future__ import annotations

import math
from typing import List, Optional, Tuple

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def gaussian_matrix(n: int, seed: int, complex_: bool = False) -> np.ndarray:
    rng = _rng(seed)
    if complex_:
        re = rng.standard_normal((n, n))
        im = rng.standard_normal((n, n))
        return (re + 1j * im) / math.sqrt(2.0)
    return rng.standard_normal((n, n))


def _haar_from_gaussian(G, device: Optional[str] = None):
    """Q from QR of G with R-diagonal phase correction (Mezzadri 2007)."""
    if device is not None and device != "cpu":
        import torch
        Gt = torch.from_numpy(G).to(device)
        Q, R = torch.linalg.qr(Gt)
        d = torch.diagonal(R)
        ph = d / d.abs()
        Q = Q * ph.unsqueeze(0)
        return Q
    Q, R = np.linalg.qr(G)
    d = np.diagonal(R)
    return Q * (d / np.abs(d))[None, :]


def spectrum(n: int, kind: str, seed: int, rank: Optional[int] = None) -> np.ndarray:
    rng = _rng(seed + 7919)
    if kind == "uniform":
        return rng.uniform(0.0, 1.0, n)
    if kind == "beta":
        return rng.beta(0.5, 0.5, n)
    if kind == "projection":
        k = n // 4 if rank is None else rank
        lam = np.zeros(n)
        lam[rng.permutation(n)[:k]] = 1.0
        return lam
    raise ValueError(kind)


def hermitian_kernel(n: int, seed: int = 0, kind: str = "uniform",
                     complex_: bool = False, rank: Optional[int] = None,
                     device: Optional[str] = None, return_torch: bool = False):
    """K = Q diag(lam) Q^H, Q Haar (orthogonal or unitary), lam per ``kind``."""
    G = gaussian_matrix(n, seed, complex_)
    lam = spectrum(n, kind, seed, rank)
    Q = _haar_from_gaussian(G, device)
    if device is not None and device != "cpu":
        import torch
        lt = torch.from_numpy(lam).to(Q.device, dtype=Q.real.dtype)
        K = (Q * lt.to(Q.dtype).unsqueeze(0)) @ Q.conj().T
        K = 0.5 * (K + K.conj().T)
        if return_torch:
            return K
        return K.cpu().numpy()
    K = (Q * lam[None, :]) @ Q.conj().T
    return 0.5 * (K + K.conj().T)


def diagonal_kernel(n: int, seed: int = 0) -> np.ndarray:
    return np.diag(_rng(seed).uniform(0.0, 1.0, n))


# --------------------------------------------------------------------------
# Uniform spanning trees of the d x d grid graph
# --------------------------------------------------------------------------
def grid_edges(d: int) -> np.ndarray:
    """Edges of the d x d grid (vertex r*d + c): right edges then down edges."""
    edges = []
    for r in range(d):
        for c in range(d - 1):
            edges.append((r * d + c, r * d + c + 1))
    for r in range(d - 1):
        for c in range(d):
            edges.append((r * d + c, (r + 1) * d + c))
    return np.array(edges, dtype=np.int64)


def ust_grid_kernel(d: int, device: Optional[str] = None) -> Tuple[np.ndarray, np.ndarray, int]:
    """Transfer-current kernel of the d x d grid: (K, edges, n_vertices).

    n = 2 d (d - 1) edges, rank d^2 - 1. Unit weights, vertex 0 grounded.
    """
    edges = grid_edges(d)
    V, E = d * d, len(edges)
    B = np.zeros((V, E))
    B[edges[:, 0], np.arange(E)] = 1.0
    B[edges[:, 1], np.arange(E)] = -1.0
    Br = B[1:, :]
    if device is not None and device != "cpu":
        import torch
        Bt = torch.from_numpy(Br).to(device)
        Lr = Bt @ Bt.T
        X = torch.linalg.solve(Lr, Bt)
        K = Bt.T @ X
        K = 0.5 * (K + K.T)
        return K.cpu().numpy(), edges, V
    Lr = Br @ Br.T
    X = np.linalg.solve(Lr, Br)
    K = Br.T @ X
    return 0.5 * (K + K.T), edges, V


def grid_spanning_tree_log_count(d: int) -> float:
    """log tau(d x d grid) by Kirchhoff: product of the nonzero Laplacian
    eigenvalues (sums of path-graph eigenvalues 2 - 2 cos(pi a / d)) over V."""
    lam = 2.0 - 2.0 * np.cos(np.pi * np.arange(d) / d)
    s = lam[:, None] + lam[None, :]
    s = s.ravel()[1:]  # drop the (0, 0) zero eigenvalue
    return float(np.sum(np.log(s)) - math.log(d * d))


# --------------------------------------------------------------------------
# Domino tilings of the Aztec diamond
# --------------------------------------------------------------------------
def aztec_squares(d: int):
    """Unit squares of the Aztec diamond of order d, by lower-left corner
    (x, y), centre (x + 1/2, y + 1/2) with |x + 1/2| + |y + 1/2| <= d; split by
    checkerboard colour (black: x + y even), each list ordered by (y, x)."""
    sq = [(x, y) for y in range(-d, d) for x in range(-d, d)
          if abs(x + 0.5) + abs(y + 0.5) <= d]
    black = [s for s in sq if (s[0] + s[1]) % 2 == 0]
    white = [s for s in sq if (s[0] + s[1]) % 2 != 0]
    return black, white


def aztec_kasteleyn(d: int):
    """(Kast, edges): the Kasteleyn matrix of the Aztec diamond's dual graph,
    rows black squares, columns white squares, weight 1 for a horizontal
    neighbour and i for a vertical one (every inner face is a 4-cycle with
    two of each, so the alternating product is -1, Kasteleyn's condition);
    edges (black index, white index) ordered by black square, then by the
    directions east, west, north, south. |det Kast| = 2^{d (d + 1) / 2}."""
    black, white = aztec_squares(d)
    wi = {s: i for i, s in enumerate(white)}
    nb = len(black)
    Kast = np.zeros((nb, nb), dtype=np.complex128)
    edges = []
    for b, (x, y) in enumerate(black):
        for dx, dy, wgt in ((1, 0, 1.0), (-1, 0, 1.0), (0, 1, 1j), (0, -1, 1j)):
            w = wi.get((x + dx, y + dy))
            if w is not None:
                Kast[b, w] = wgt
                edges.append((b, w))
    return Kast, np.array(edges, dtype=np.int64)


def aztec_kernel(d: int, device: Optional[str] = None, return_torch: bool = False):
    """(K, edges, n_black): the edge-inclusion kernel of uniform domino
    tilings of the Aztec diamond of order d (n = 4 d^2 edges, complex,
    non-Hermitian, rank d (d + 1)). K[e, e'] = Kast(b, w) Kast^{-1}(w, b');
    every principal minor is an inclusion probability (Kenyon), every draw a
    perfect matching of probability 2^{-d (d + 1) / 2}. The inverse is taken
    with torch on ``device`` when given (a library routine; rounding only);
    ``return_torch`` then returns K on the device with column-major storage."""
    Kast, edges = aztec_kasteleyn(d)
    b, w = edges[:, 0], edges[:, 1]
    wt = Kast[b, w]
    if device is not None and device != "cpu":
        import torch
        KiT = torch.linalg.inv(torch.from_numpy(Kast).to(device)).T
        bi = torch.from_numpy(b).to(device)
        wi_ = torch.from_numpy(w).to(device)
        # K^T[e', e] = Kast^{-1}(w_e, b_e') Kast(b_e, w_e), stored row-major
        Kt = KiT[bi][:, wi_] * torch.from_numpy(wt).to(device)[None, :]
        if return_torch:
            return Kt.t(), edges, Kast.shape[0]
        return Kt.t().cpu().numpy(), edges, Kast.shape[0]
    Ki = np.linalg.inv(Kast)
    K = wt[:, None] * Ki[w][:, b]
    return K, edges, Kast.shape[0]


def aztec_log_tilings(d: int) -> float:
    """log of the number of domino tilings of the Aztec diamond of order d,
    2^{d (d + 1) / 2} (Elkies-Kuperberg-Larsen-Propp)."""
    return d * (d + 1) / 2 * math.log(2.0)


def is_perfect_matching(edges: np.ndarray, keep: np.ndarray, n_black: int) -> bool:
    """The kept edges cover every black and every white square exactly once."""
    k = np.asarray(keep).astype(bool)
    e = edges[k]
    if len(e) != n_black:
        return False
    return len(np.unique(e[:, 0])) == n_black and len(np.unique(e[:, 1])) == n_black


# --------------------------------------------------------------------------
# Non-Hermitian kernels with a known Hermitian twin
# --------------------------------------------------------------------------
def lu_similarity_kernel(n: int, seed: int = 0, sigma: float = 0.5,
                         device: Optional[str] = None, complex_: bool = False):
    """(K, S): S = Q diag(U(0,1)) Q^H, K = D^{-1} S D with D = diag(exp(N(0, sigma^2)))
    (times a uniform phase exp(i theta) when ``complex_``)."""
    S = hermitian_kernel(n, seed, "uniform", device=device, complex_=complex_)
    rng = _rng(seed + 104729)
    dvec = np.exp(sigma * rng.standard_normal(n))
    if complex_:
        dvec = dvec * np.exp(1j * rng.uniform(0.0, 2 * np.pi, n))
    K = S * (dvec[None, :] / dvec[:, None])
    return K, S


# --------------------------------------------------------------------------
# Batched L-ensembles
# --------------------------------------------------------------------------
def lensemble_sizes(batch: int, seed: int = 0, nmin: int = 64, nmax: int = 1024) -> np.ndarray:
    return _rng(seed).integers(nmin, nmax + 1, size=batch)


def lensemble_features(n: int, seed: int, features: int = 64,
                       qmin: float = 0.1, qmax: float = 10.0) -> np.ndarray:
    """Phi (n x features): unit-norm Gaussian rows times LogUniform qualities."""
    rng = _rng(seed)
    G = rng.standard_normal((n, features))
    G /= np.linalg.norm(G, axis=1, keepdims=True)
    q = np.exp(rng.uniform(math.log(qmin), math.log(qmax), n))
    return G * q[:, None]


def lensemble_L(n: int, seed: int, features: int = 64) -> np.ndarray:
    """The L-ensemble kernel L = Phi Phi^T of ``lensemble_kernel``'s Phi."""
    Phi = lensemble_features(n, seed, features)
    L = Phi @ Phi.T
    return 0.5 * (L + L.T)


def lensemble_kernel(n: int, seed: int, features: int = 64,
                     qmin: float = 0.1, qmax: float = 10.0) -> np.ndarray:
    """K = Phi (Phi^T Phi + I)^{-1} Phi^T = L (L + I)^{-1}, L = Phi Phi^T."""
    Phi = lensemble_features(n, seed, features, qmin, qmax)
    M = Phi.T @ Phi + np.eye(features)
    K = Phi @ np.linalg.solve(M, Phi.T)
    return 0.5 * (K + K.T)


def lensemble_batch(batch: int, seed: int = 0, nmin: int = 64, nmax: int = 1024,
                    features: int = 64) -> List[np.ndarray]:
    sizes = lensemble_sizes(batch, seed, nmin, nmax)
    return [lensemble_kernel(int(m), seed * 1000003 + i + 1, features)
            for i, m in enumerate(sizes)]


def lensemble_batch_torch(batch: int, seed: int = 0, nmin: int = 64, nmax: int = 1024,
                          features: int = 64, device: str = "cuda"):
    """The same law as ``lensemble_batch`` built with torch on a device
    (FP64): per kernel, unit-norm Gaussian feature rows scaled by
    LogUniform(0.1, 10) qualities, K = Phi (Phi^T Phi + I)^{-1} Phi^T."""
    import torch
    sizes = lensemble_sizes(batch, seed, nmin, nmax)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    out = []
    eye = torch.eye(features, dtype=torch.float64, device=device)
    for m in sizes:
        m = int(m)
        G = torch.randn(m, features, generator=gen, dtype=torch.float64).to(device)
        G = G / G.norm(dim=1, keepdim=True)
        q = torch.exp(torch.empty(m, dtype=torch.float64).uniform_(math.log(0.1), math.log(10.0),
                                                                   generator=gen)).to(device)
        Phi = G * q[:, None]
        K = Phi @ torch.linalg.solve(Phi.T @ Phi + eye, Phi.T)
        out.append(0.5 * (K + K.T))
    return out


def lensemble_L_batch_torch(batch: int, seed: int = 0, nmin: int = 64, nmax: int = 1024,
                            features: int = 64, device: str = "cuda"):
    """The L-ensemble kernels L_i = Phi_i Phi_i^T of ``lensemble_batch_torch``
    (same sizes, same features), before conversion to marginal kernels."""
    import torch
    sizes = lensemble_sizes(batch, seed, nmin, nmax)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    out = []
    for m in sizes:
        m = int(m)
        G = torch.randn(m, features, generator=gen, dtype=torch.float64).to(device)
        G = G / G.norm(dim=1, keepdim=True)
        q = torch.exp(torch.empty(m, dtype=torch.float64).uniform_(math.log(0.1), math.log(10.0),
                                                                   generator=gen)).to(device)
        Phi = G * q[:, None]
        L = Phi @ Phi.T
        out.append(0.5 * (L + L.T))
    return out
