"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: published
known-answer vectors, the determinant definition of the DPP (Definition and
Theorem 1 of arXiv:1905.00165), exhaustive enumeration, independent library
routines (LAPACK slogdet/solve/inv), textbook special cases (a diagonal kernel
is a product of independent Bernoullis; a projection kernel of rank k always
yields k items), the uniform spanning-tree measure with Kirchhoff's tree count,
and likelihoods the paper prints.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_likelihoods():
    out = {}
    with open(os.path.join(GOLDEN, "paper_likelihoods.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, val, tol, src = line.split()
            out[name] = (float(val), float(tol))
    return out


# ---------------------------------------------------------------------------
# Philox4x32-10 and the uniform recipe
# ---------------------------------------------------------------------------
def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        words = [int(x, 16) for x in r]
        out = O.philox4x32_10(words[0:4], words[4:6])
        assert [int(x) for x in out] == words[6:10]


def test_uniform_recipe_and_histogram():
    u = O.uniforms(seed=12345, instance=7, n=200000)
    assert np.all(u > 0.0) and np.all(u < 1.0)
    # recipe: 53 bits from x0 (all) and x1 (top 21), centred in its cell
    x = O.philox4x32_10([5, 7, 0, 0], [12345, 0])
    bits = (int(x[0]) << 21) | (int(x[1]) >> 11)
    assert u[5] == (bits + 0.5) * 2.0 ** -53
    # chi-squared over 100 equiprobable bins
    counts = np.bincount(np.minimum((u * 100).astype(int), 99), minlength=100)
    e = len(u) / 100
    chi2 = float(np.sum((counts - e) ** 2 / e))
    # 99 dof: the 1e-4 upper quantile is about 160
    assert chi2 < 160.0
    # different seeds/instances give different streams
    assert not np.allclose(O.uniforms(1, 0, 16), O.uniforms(2, 0, 16))
    assert not np.allclose(O.uniforms(1, 0, 16), O.uniforms(1, 1, 16))


# ---------------------------------------------------------------------------
# Exhaustive enumeration (n = 10, the small Hermitian configuration)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def K10():
    return W.hermitian_kernel(10, seed=0, kind="uniform")


def test_enumeration_sums_to_one(K10):
    p = O.enumerate_probs(K10)
    assert abs(p.sum() - 1.0) < 1e-12
    assert np.all(p >= 0)


def test_enumeration_sums_to_one_nonhermitian_and_complex():
    K, S = W.lu_similarity_kernel(8, seed=3)
    assert abs(O.enumerate_probs(K).sum() - 1.0) < 1e-12
    Kc = W.hermitian_kernel(8, seed=4, complex_=True)
    assert abs(O.enumerate_probs(Kc).sum() - 1.0) < 1e-12


@pytest.mark.parametrize("form", ["ldl", "lu"])
def test_every_decision_path_matches_determinant(K10, form):
    """For all 2^10 decision sequences, the product of the factorization's
    branch probabilities equals |det(K - 1_{Y^c})| (Theorem 1), and every
    pivot before its decision lies in [0, 1] (Prop. 1 / admissibility)."""
    n = K10.shape[0]
    p = O.enumerate_probs(K10)
    f = O.sample_ldl if form == "ldl" else O.sample_lu
    for mask in range(1 << n):
        keep = np.array([(mask >> j) & 1 for j in range(n)], dtype=np.uint8)
        d = f(K10, O.forced_uniforms(keep))
        assert np.array_equal(d.keep, keep)
        piv = np.real(d.pivots)
        pre = np.where(keep == 1, piv, piv + 1.0)
        assert np.all(pre > -1e-12) and np.all(pre < 1 + 1e-12)
        branch = np.prod(np.where(keep == 1, pre, 1.0 - pre))
        assert abs(branch - p[mask]) < 1e-12
        assert abs(math.exp(d.logp) - p[mask]) < 1e-12


def test_chi_squared_against_enumeration(K10):
    n = K10.shape[0]
    p = O.enumerate_probs(K10)
    draws = 40000
    counts = np.zeros(1 << n)
    for s in range(draws):
        d = O.sample_ldl(K10, O.uniforms(s, 0, n))
        counts[O.mask_index(d.keep)] += 1
    e = draws * p
    big = e >= 5
    obs = np.concatenate([counts[big], [counts[~big].sum()]])
    exp = np.concatenate([e[big], [e[~big].sum()]])
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    dof = len(obs) - 1
    # Wilson-Hilferty upper quantile at about 1e-4
    z = 3.72
    crit = dof * (1 - 2 / (9 * dof) + z * math.sqrt(2 / (9 * dof))) ** 3
    assert chi2 < crit, (chi2, crit, dof)


def test_marginals_and_pair_marginals():
    """Inclusion frequency -> K_jj and pair frequency -> det K_{ij}
    (the Definition: P[Y subset of sample] = det K_Y)."""
    K = W.hermitian_kernel(12, seed=5, kind="beta")
    n = K.shape[0]
    draws = 20000
    incl = np.zeros(n)
    pair = np.zeros((n, n))
    for s in range(draws):
        k = O.sample_ldl(K, O.uniforms(s, 3, n)).keep.astype(float)
        incl += k
        pair += np.outer(k, k)
    pj = np.diag(K)
    z = (incl / draws - pj) / np.sqrt(pj * (1 - pj) / draws + 1e-300)
    assert np.all(np.abs(z) < 4.5)
    for i in range(n):
        for j in range(i + 1, n):
            pij = K[i, i] * K[j, j] - K[i, j] * K[j, i]
            zz = (pair[i, j] / draws - pij) / math.sqrt(max(pij * (1 - pij), 1e-12) / draws)
            assert abs(zz) < 5.0


# ---------------------------------------------------------------------------
# Likelihood against an independent library routine
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("complex_", [False, True])
def test_logp_equals_slogdet(complex_):
    n = 160
    K = W.hermitian_kernel(n, seed=11, kind="uniform", complex_=complex_)
    for s in range(4):
        d = O.sample_ldl(K, O.uniforms(s, 0, n))
        ref = O.subset_logprob(K, d.keep)
        assert abs(d.logp - ref) <= 1e-10 * abs(ref)
        d2 = O.sample_lu(K, O.uniforms(s, 0, n))
        assert np.array_equal(d.keep, d2.keep)
        assert abs(d2.logp - ref) <= 1e-10 * abs(ref)


def test_conditional_pivot_matches_sampler():
    n = 40
    K = W.hermitian_kernel(n, seed=2, kind="beta")
    d = O.sample_ldl(K, O.uniforms(9, 0, n))
    pre = np.where(d.keep == 1, d.pivots, d.pivots + 1.0)
    for j in range(n):
        cp = O.conditional_pivot(K, d.keep, j)
        assert abs(cp - pre[j]) < 1e-11


# ---------------------------------------------------------------------------
# Textbook special cases
# ---------------------------------------------------------------------------
def test_diagonal_kernel_is_independent_bernoulli():
    n = 300
    K = W.diagonal_kernel(n, seed=1)
    p = np.diag(K)
    for s in range(5):
        u = O.uniforms(s, 0, n)
        d = O.sample_ldl(K, u)
        assert np.array_equal(d.keep, (u < p).astype(np.uint8))
        ref = float(np.sum(np.log(np.where(u < p, p, 1 - p))))
        assert abs(d.logp - ref) < 1e-12 * abs(ref)


@pytest.mark.parametrize("n,k", [(64, 16), (256, 64)])
def test_projection_kernel_cardinality(n, k):
    K = W.hermitian_kernel(n, seed=3, kind="projection", rank=k)
    for s in range(10):
        d = O.sample_ldl(K, O.uniforms(s, 0, n))
        assert int(d.keep.sum()) == k


def test_uniform_spanning_tree_small_grid():
    d = 8
    K, edges, V = W.ust_grid_kernel(d)
    ref = -W.grid_spanning_tree_log_count(d)
    for s in range(20):
        dr = O.sample_ldl(K, O.uniforms(s, 0, K.shape[0]))
        assert O.is_spanning_tree(edges[dr.keep.astype(bool)], V)
        assert abs(dr.logp - ref) < 1e-9 * abs(ref)


def test_grid_tree_count_matches_paper_figure():
    """Kirchhoff's count for the 40 x 40 grid gives the paper's printed
    log-likelihood of its uniform-spanning-tree samples (Fig. 1)."""
    val, tol = _golden_likelihoods()["ust_grid_40"]
    assert abs(-W.grid_spanning_tree_log_count(40) - val) < tol


@pytest.mark.slow
def test_uniform_spanning_tree_grid40_one_draw():
    """One oracle draw on the 40 x 40 grid (n = 3120 edges) is a spanning tree
    with the paper's printed likelihood exp(-1794.24)."""
    val, tol = _golden_likelihoods()["ust_grid_40"]
    K, edges, V = W.ust_grid_kernel(40)
    dr = O.sample_ldl(K, O.uniforms(0, 0, K.shape[0]))
    assert O.is_spanning_tree(edges[dr.keep.astype(bool)], V)
    assert abs(dr.logp - val) < tol


# ---------------------------------------------------------------------------
# Diagonal similarity and LU vs LDL^H
# ---------------------------------------------------------------------------
def test_lu_on_similarity_equals_ldl_on_hermitian_twin():
    """DPP(D^{-1} S D) = DPP(S) (Prop. 2): LU on K and LDL^H on S draw the
    same set with the same likelihood from the same uniforms."""
    n = 96
    K, S = W.lu_similarity_kernel(n, seed=4)
    assert not np.allclose(K, K.T)
    for s in range(10):
        u = O.uniforms(s, 0, n)
        a = O.sample_lu(K, u)
        b = O.sample_ldl(S, u)
        assert np.array_equal(a.keep, b.keep)
        assert abs(a.logp - b.logp) < 1e-10 * abs(b.logp)


def test_complex_hermitian_ldl_equals_lu():
    n = 64
    K = W.hermitian_kernel(n, seed=6, kind="beta", complex_=True)
    for s in range(5):
        u = O.uniforms(s, 1, n)
        a = O.sample_ldl(K, u)
        b = O.sample_lu(K, u)
        assert np.array_equal(a.keep, b.keep)
        assert abs(a.logp - b.logp) < 1e-10 * abs(b.logp)
        assert np.max(np.abs(np.imag(b.pivots))) < 1e-10


def test_returned_factor_is_ldl_of_shifted_kernel():
    """On return A holds the unit-lower L and D of K - 1_{Y^c} (Algorithm 1's
    caption, Hermitian form)."""
    n = 50
    K = W.hermitian_kernel(n, seed=8)
    d = O.sample_ldl(K, O.uniforms(0, 0, n))
    L = np.tril(d.A, -1) + np.eye(n)
    D = np.diag(np.diag(d.A))
    assert np.allclose(L @ D @ L.T, O.complement_shift(K, d.keep), atol=1e-12)


# ---------------------------------------------------------------------------
# Greedy maximum-likelihood variant
# ---------------------------------------------------------------------------
def test_greedy_follows_more_likely_branch():
    n = 30
    K = W.hermitian_kernel(n, seed=12, kind="beta")
    g = O.greedy_ldl(K)
    for j in range(n):
        cp = float(np.real(O.conditional_pivot(K, g.keep, j)))
        assert g.keep[j] == (1 if cp > 0.5 else 0)
    assert abs(g.logp - O.subset_logprob(K, g.keep)) < 1e-10 * abs(g.logp)


# ---------------------------------------------------------------------------
# Adjoint closed form against finite differences
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("complex_", [False, True])
def test_logprob_grad_matches_finite_differences(complex_):
    n = 12
    if complex_:
        K = W.hermitian_kernel(n, seed=13, complex_=True)
    else:
        K, _ = W.lu_similarity_kernel(n, seed=13)
    keep = O.sample_lu(K, O.uniforms(0, 0, n)).keep
    G = O.logprob_grad(K, keep)
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(20):
        i, j = rng.integers(0, n, 2)
        E = np.zeros_like(K)
        E[i, j] = 1.0
        fd = (O.subset_logprob(K + h * E, keep) - O.subset_logprob(K - h * E, keep)) / (2 * h)
        assert abs(fd - np.real(G[i, j])) < 1e-6 * max(1.0, abs(fd))
        if complex_:
            fdi = (O.subset_logprob(K + 1j * h * E, keep)
                   - O.subset_logprob(K - 1j * h * E, keep)) / (2 * h)
            assert abs(fdi - np.imag(G[i, j])) < 1e-6 * max(1.0, abs(fdi))


# ---------------------------------------------------------------------------
# Algorithm 2 (Theorem 2): the elementary sampler of projection kernels
# ---------------------------------------------------------------------------
def _projection(n, k, seed):
    return W.hermitian_kernel(n, seed=seed, kind="projection", rank=k)


def test_elementary_sample_size_likelihood_and_factor():
    """Every draw has exactly k distinct indices (Theorem 2); log P(Y) is
    log det(K_Y) (library slogdet), and the returned factor is the Cholesky
    factor of K_Y in selection order."""
    for n, k, seed in [(40, 1, 1), (40, 10, 2), (120, 30, 3), (64, 64, 4)]:
        K = _projection(n, k, seed)
        for s in range(4):
            d = O.sample_elementary(K, k, O.uniforms(s, 7, k))
            assert d.ok
            assert len(set(d.sample.tolist())) == k and d.sample.min() >= 0 and d.sample.max() < n
            KY = K[np.ix_(d.sample, d.sample)]
            sign, ld = np.linalg.slogdet(KY)
            assert sign > 0 and abs(d.logp - ld) <= 1e-9 * max(1.0, abs(ld))
            assert np.allclose(np.tril(d.chol), d.chol)
            assert np.abs(d.chol @ d.chol.T - KY).max() < 1e-10


def test_elementary_distribution_chi2():
    """n = 8, rank 3: the empirical frequencies of 30 000 draws against
    P(Y) = det(K_Y) for all 56 subsets of size 3 (the DPP of a projection
    kernel has only samples of size k, Theorem 2)."""
    import itertools
    from scipy import stats
    n, k = 8, 3
    K = _projection(n, k, 11)
    subsets = list(itertools.combinations(range(n), k))
    p = np.array([np.linalg.det(K[np.ix_(c, c)]) for c in subsets])
    assert abs(p.sum() - 1.0) < 1e-12
    index = {c: i for i, c in enumerate(subsets)}
    counts = np.zeros(len(subsets))
    draws = 30000
    for s in range(draws):
        d = O.sample_elementary(K, k, O.uniforms(s, 0, k))
        counts[index[tuple(sorted(d.sample.tolist()))]] += 1
    keep = p * draws >= 5
    chi2 = ((counts[keep] - draws * p[keep]) ** 2 / (draws * p[keep])).sum()
    pval = stats.chi2.sf(chi2, keep.sum() - 1)
    assert pval > 1e-3, (chi2, pval)


def test_elementary_inclusion_marginals():
    """Inclusion frequencies approach diag(K) (P[i in Y] = K_ii)."""
    n, k = 30, 9
    K = _projection(n, k, 5)
    draws = 8000
    freq = np.zeros(n)
    for s in range(draws):
        freq[O.sample_elementary(K, k, O.uniforms(s, 3, k)).sample] += 1
    freq /= draws
    se = np.sqrt(np.diag(K) * (1 - np.diag(K)) / draws) + 1e-3
    assert np.all(np.abs(freq - np.diag(K)) < 5 * se)


def test_elementary_edge_cases():
    """k = 0 draws nothing; the identity (rank n) keeps every index with
    probability one."""
    K = _projection(10, 3, 6)
    d = O.sample_elementary(K, 0, np.zeros(1))
    assert d.sample.size == 0 and d.logp == 0.0
    n = 12
    d = O.sample_elementary(np.eye(n), n, O.uniforms(1, 0, n))
    assert sorted(d.sample.tolist()) == list(range(n)) and abs(d.logp) < 1e-12


def test_complex_lu_logp_on_nonhermitian_kernel():
    """The complex LU form on a non-Hermitian K = D^{-1} S D (D with complex
    phases): log P equals log|det(K - 1_{Y^c})| (LAPACK slogdet), and the
    decisions equal those of the Hermitian LDL^H form on S (Prop. 2)."""
    n = 60
    K, S = W.lu_similarity_kernel(n, seed=12, complex_=True)
    assert np.abs(K - K.conj().T).max() > 1e-3  # genuinely non-Hermitian
    for seed in range(3):
        u = O.uniforms(seed, 4, n)
        d = O.sample_lu(K, u)
        assert abs(d.logp - O.subset_logprob(K, d.keep)) <= 1e-10 * max(1.0, abs(d.logp))
        h = O.sample_ldl(S, u)
        assert np.array_equal(d.keep, h.keep)
        assert abs(d.logp - h.logp) <= 1e-10 * max(1.0, abs(h.logp))


# ---------------------------------------------------------------------------
# Domino tilings of the Aztec diamond (complex, non-Hermitian; Figs. 3 and 4)
# ---------------------------------------------------------------------------
def _count_perfect_matchings(edges, n_black):
    """Brute force: perfect matchings of the bipartite graph, black by black."""
    adj = [[] for _ in range(n_black)]
    for b, w in edges:
        adj[int(b)].append(int(w))

    def rec(b, used):
        if b == n_black:
            return 1
        return sum(rec(b + 1, used | (1 << w)) for w in adj[b] if not used >> w & 1)

    return rec(0, 0)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_aztec_kasteleyn_counts_tilings(d):
    """The number of tilings by brute force is 2^{d(d+1)/2}, and so is
    |det Kast| (Kasteleyn's theorem pins the weights)."""
    Kast, edges = W.aztec_kasteleyn(d)
    assert len(edges) == 4 * d * d
    count = _count_perfect_matchings(edges, Kast.shape[0])
    assert count == 2 ** (d * (d + 1) // 2)
    assert abs(np.linalg.slogdet(Kast)[1] - W.aztec_log_tilings(d)) < 1e-12


def test_aztec_kernel_enumeration_order2():
    """Order 2 (n = 16): P(Y) = |det(K - 1_{Y^c})| over all 2^16 subsets sums
    to one and is 1/8 on exactly the 8 tilings, 0 elsewhere."""
    K, edges, nb = W.aztec_kernel(2)
    assert np.abs(K - K.conj().T).max() > 1e-3  # genuinely non-Hermitian
    probs = O.enumerate_probs(K)
    assert abs(probs.sum() - 1.0) < 1e-12
    support = np.flatnonzero(probs > 1e-9)
    assert len(support) == 8
    for mask in support:
        keep = np.array([(mask >> j) & 1 for j in range(16)], dtype=np.uint8)
        assert W.is_perfect_matching(edges, keep, nb)
        assert abs(probs[mask] - 0.125) < 1e-12


@pytest.mark.parametrize("d", [2, 5, 8])
def test_aztec_oracle_draws_are_uniform_tilings(d):
    """Every LU draw of the Kenyon kernel is a tiling with log P equal to
    -log(#tilings) = -(d(d+1)/2) ln 2."""
    K, edges, nb = W.aztec_kernel(d)
    n = K.shape[0]
    for seed in range(4):
        dr = O.sample_lu(K, O.uniforms(seed, 0, n))
        assert W.is_perfect_matching(edges, dr.keep, nb)
        assert abs(dr.logp + W.aztec_log_tilings(d)) <= 1e-9 * W.aztec_log_tilings(d)


def test_aztec_order10_likelihood_matches_paper():
    """Fig. 3: both samples of the order-10 diamond have likelihood
    exp(-38.1231)."""
    val, tol = _golden_likelihoods()["aztec_10"]
    K, edges, nb = W.aztec_kernel(10)
    for seed in range(2):
        dr = O.sample_lu(K, O.uniforms(seed, 0, K.shape[0]))
        assert W.is_perfect_matching(edges, dr.keep, nb)
        assert abs(dr.logp - val) <= tol
    val80, tol80 = _golden_likelihoods()["aztec_80"]
    assert abs(-W.aztec_log_tilings(80) - val80) <= tol80
