"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every check uses a published
known-answer vector, a closed form, a brute-force enumeration, a library
routine computing a textbook quantity, or a theorem the paper relies on.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_graphs():
    rng = np.random.default_rng(7)
    out = [synth.grid(4, 3), synth.complete(5), synth.cycle(7), synth.grid(5, 5)]
    for i in range(3):
        n = 9 + i
        s = rng.integers(0, n, 3 * n)
        d = rng.integers(0, n, 3 * n)
        g = synth.from_edges(n, s, d, name=f"rand{i}")
        out.append(g)
    return out


def tiny_graphs():
    """Graphs small enough to enumerate every spanning tree."""
    k23 = synth.from_edges(5, [0, 0, 0, 1, 1, 1], [2, 3, 4, 2, 3, 4], name="K23")
    diamond = synth.from_edges(4, [0, 0, 1, 1, 2], [1, 2, 2, 3, 3], name="diamond")
    house = synth.from_edges(6, [0, 1, 2, 3, 0, 2, 4, 1], [1, 2, 3, 0, 4, 4, 5, 5], name="house6")
    return [synth.complete(4), synth.cycle(5), k23, diamond, synth.grid(3, 3), house,
            synth.grid(2, 4)]


# ----------------------------------------------------------------- Philox

def test_philox_known_answers(orc):
    """Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11)."""
    rows = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            out = orc.philox4x32_10(w[0:4], w[4:6])
            assert list(out) == w[6:10]
            rows += 1
    assert rows == 3


def test_successor_index_is_uniform(orc):
    """floor(x * deg / 2^64) of the 64-bit Philox word is uniform over the
    neighbours (chi-square, 60k draws of one vertex over stack depths)."""
    g = synth.from_edges(8, [0] * 7, list(range(1, 8)))  # star, centre degree 7
    counts = np.zeros(8, dtype=np.int64)
    for d in range(60000):
        counts[orc.successor(g, 0, d, 3, 0, 12345)] += 1
    assert counts[0] == 0
    p = stats.chisquare(counts[1:]).pvalue
    assert p > 1e-4, counts


def test_successor_depends_on_every_key_word(orc):
    g = synth.complete(64)
    base = orc.successor(g, 5, 0, 0, 0, 1)
    seen = {base}
    for args in [(5, 1, 0, 0, 1), (5, 0, 1, 0, 1), (5, 0, 0, 1, 1), (5, 0, 0, 0, 2), (5, 0, 0, 0, 1 << 40)]:
        seen.add(orc.successor(g, *args))
    assert len(seen) >= 4


# -------------------------------------------------------------------- BFS

@pytest.mark.parametrize("gi", range(7))
def test_bfs_against_all_pairs_shortest_paths(orc, gi):
    g = small_graphs()[gi]
    A = csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    D = shortest_path(A, unweighted=True)
    for u in [0, g.n // 2, g.n - 1]:
        ecc, dist, par = orc.bfs(g, u)
        assert np.array_equal(dist, D[u].astype(np.int32))
        assert ecc == int(D[u].max())
        for v in range(g.n):
            if v == u:
                assert par[v] == -1
                continue
            nb = g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]
            closer = [w for w in nb if D[u, w] == D[u, v] - 1]
            assert par[v] == min(closer)


def test_bfs_reports_disconnected(orc):
    g = synth.from_edges(4, [0, 2], [1, 3], lcc=False)
    ecc, _, _ = orc.bfs(g, 0)
    assert ecc == -1


# ----------------------------------------------------------------- Wilson

def _is_spanning_tree(g, nxt, u):
    n = g.n
    if nxt[u] != -1:
        return False
    for v in range(n):
        if v == u:
            continue
        nb = g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]
        if nxt[v] not in nb:
            return False
        w, steps = v, 0
        while w != u:
            w = nxt[w]
            steps += 1
            if steps > n:
                return False
    return True


@pytest.mark.parametrize("gi", range(7))
def test_wilson_equals_cycle_popping(orc, gi):
    """Wilson's cycle-popping theorem (cited in Appendix A.2): with per-vertex
    stacks, loop-erased walks and explicit popping in another order give the
    same tree and pop the same number of entries at every vertex."""
    g = small_graphs()[gi]
    for u in [0, g.n - 1]:
        for t in range(40):
            a, pa, steps = orc.wilson(g, u, t, 99)
            b, pb, draws = orc.cycle_pop(g, u, t, 99)
            assert np.array_equal(a, b)
            assert np.array_equal(pa, pb)
            assert steps == draws
            assert _is_spanning_tree(g, a, u)


def test_wilson_equals_cycle_popping_rmat(orc):
    g = synth.rmat(10, 8, seed=3)
    u = synth.max_degree_vertex(g)
    for t in range(20):
        a, pa, _ = orc.wilson(g, u, t, 5)
        b, pb, _ = orc.cycle_pop(g, u, t, 5)
        assert np.array_equal(a, b) and np.array_equal(pa, pb)


@pytest.mark.parametrize("gi", range(7))
def test_matrix_tree_theorem(orc, gi):
    """Enumerated spanning trees = det of a Laplacian minor (Kirchhoff)."""
    g = tiny_graphs()[gi]
    trees = orc.spanning_trees(g)
    assert len(trees) == round(orc.matrix_tree_count(g))


def test_known_tree_counts(orc):
    """Textbook counts: K4 has 16 = 4^2 spanning trees (Cayley), C5 has 5,
    K_{2,3} has 12 = 2^2 * 3^1, the 3x3 grid has 192."""
    g = tiny_graphs()
    assert len(orc.spanning_trees(g[0])) == 16
    assert len(orc.spanning_trees(g[1])) == 5
    assert len(orc.spanning_trees(g[2])) == 12
    assert len(orc.spanning_trees(g[4])) == 192


@pytest.mark.parametrize("gi,u", [(0, 0), (2, 0), (3, 1), (5, 2)])
def test_wilson_samples_uniformly(orc, gi, u):
    """Proposition (Wilson): the sampled tree is uniform over all spanning
    trees (chi-square over the enumerated trees)."""
    g = tiny_graphs()[gi]
    trees = orc.spanning_trees(g)
    index = {t: i for i, t in enumerate(trees)}
    counts = np.zeros(len(trees), dtype=np.int64)
    N = 400 * len(trees)
    for t in range(N):
        nxt, _, _ = orc.wilson(g, u, t, 2024)
        counts[index[orc.tree_edges_of(nxt)]] += 1
    p = stats.chisquare(counts).pvalue
    assert p > 1e-4, (p, counts)


def test_wilson_mean_steps_is_mean_hitting_time(orc):
    """Lemma (Appendix A.2): expected walk steps = sum_v deg(v) r(u, v)."""
    g = synth.grid(6, 6)
    u = 14
    Lp = orc.dense_pinv(g)
    r = orc.effective_resistance(Lp, u)
    expect = float((g.degrees() * r).sum())
    steps = np.array([orc.wilson(g, u, t, 11)[2] for t in range(4000)], dtype=np.float64)
    se = steps.std() / math.sqrt(steps.shape[0])
    assert abs(steps.mean() - expect) < 5 * se, (steps.mean(), expect, se)


# --------------------------------------------------------- DFS, Algorithm 2

def test_dfs_times_are_nested_intervals(orc):
    g = synth.grid(5, 4)
    nxt, _, _ = orc.wilson(g, 7, 3, 1)
    alpha, omega = orc.dfs_times(nxt, 7)
    assert sorted(np.concatenate([alpha, omega]).tolist()) == list(range(2 * g.n))
    for v in range(g.n):
        # v is inside its parent's interval
        if nxt[v] >= 0:
            p = nxt[v]
            assert alpha[p] < alpha[v] and omega[v] < omega[p]


@pytest.mark.parametrize("gi", range(7))
def test_aggregate_kirchhoff_exact(orc, gi):
    """Theorem 1 (Kirchhoff) with Eq. (N-values-in-path): averaging the
    per-tree +-1 counts over ALL spanning trees gives r(u, v) exactly."""
    g = tiny_graphs()[gi]
    trees = orc.spanning_trees(g)
    Lp = orc.dense_pinv(g)
    for u in range(g.n):
        _, _, par = orc.bfs(g, u)
        R = np.zeros(g.n, dtype=np.int64)
        for tr in trees:
            nxt = orc.root_tree(tr, g.n, u)
            orc.aggregate(nxt, par, u, R)
        r = orc.effective_resistance(Lp, u)
        np.testing.assert_allclose(R / len(trees), r, rtol=0, atol=1e-12)
        assert R[u] == 0


@pytest.mark.parametrize("maker", [lambda: synth.path(9), lambda: synth.star(8),
                                   lambda: synth.from_edges(10, [0, 0, 1, 1, 2, 4, 4, 6, 6],
                                                            [1, 2, 3, 4, 5, 6, 7, 8, 9])])
def test_aggregate_on_trees_counts_distances(orc, maker):
    """If G is a tree every UST is G, so R[v] = tau * dist(u, v) exactly."""
    g = maker()
    for u in [0, g.n - 1, g.n // 2]:
        ecc, dist, par = orc.bfs(g, u)
        R, _ = orc.sample_aggregate(g, u, par, 0, 17, seed=4)
        assert np.array_equal(R, 17 * dist.astype(np.int64))


def test_strict_reading_would_lose_last_edge(orc):
    """The inclusive subtree test is needed: on the single edge u-b the only
    tree contains (u, b) and r(u, b) = 1; v = b lies in its own subtree."""
    g = synth.path(2)
    _, _, par = orc.bfs(g, 0)
    R, _ = orc.sample_aggregate(g, 0, par, 0, 5, seed=0)
    assert R.tolist() == [0, 5]


def test_sample_aggregate_threads_match_sequential(orc):
    g = synth.grid(7, 6)
    _, _, par = orc.bfs(g, 20)
    R1, s1 = orc.sample_aggregate(g, 20, par, 3, 70, seed=8, threads=1)
    R4, s4 = orc.sample_aggregate(g, 20, par, 3, 70, seed=8, threads=4)
    assert np.array_equal(R1, R4) and s1 == s4
    # tree ranges compose: [3, 40) + [40, 70) = [3, 70)
    Ra, _ = orc.sample_aggregate(g, 20, par, 3, 40, seed=8)
    Rb, _ = orc.sample_aggregate(g, 20, par, 40, 70, seed=8)
    assert np.array_equal(Ra + Rb, R1)


# ------------------------------------------------------------- solve, combine

@pytest.mark.parametrize("gi", range(7))
def test_cg_column_matches_dense_pinv(orc, gi):
    """x solves L x = e_u - 1/n with x _|_ 1, i.e. x = L^+[:, u] (Section 3.1,
    step 1), against the dense closed form (L + J/n)^{-1} - J/n."""
    g = small_graphs()[gi]
    Lp = orc.dense_pinv(g)
    for u in [0, g.n - 1]:
        x, it, rr, ok = orc.cg(g, u, tol=1e-13)
        assert ok and rr <= 1e-13
        np.testing.assert_allclose(x, Lp[:, u], rtol=0, atol=1e-11)
        assert abs(x.sum()) < 1e-10


def test_dense_pinv_closed_forms(orc):
    """Textbook effective resistances: cycle C_n has r = k(n-k)/n, K_n has
    r = 2/n, a star has r(centre, leaf) = 1; L^+ rows sum to zero."""
    n = 11
    Lp = orc.dense_pinv(synth.cycle(n))
    r = orc.effective_resistance(Lp, 0)
    k = np.arange(n)
    np.testing.assert_allclose(r, k * (n - k) / n, atol=1e-12)
    Lp = orc.dense_pinv(synth.complete(9))
    r = orc.effective_resistance(Lp, 3)
    np.testing.assert_allclose(np.delete(r, 3), 2.0 / 9, atol=1e-12)
    Lp = orc.dense_pinv(synth.star(7))
    r = orc.effective_resistance(Lp, 0)
    np.testing.assert_allclose(r[1:], 1.0, atol=1e-12)
    np.testing.assert_allclose(Lp.sum(axis=1), 0.0, atol=1e-12)


def test_combine_recovers_dense_diagonal_from_exact_counts(orc):
    """Eq. (diag-comp): with R[v] = tau r(u, v) exact (a tree graph) and the
    exact column, the combination is the dense diagonal of L^+."""
    g = synth.from_edges(10, [0, 0, 1, 1, 2, 4, 4, 6, 6], [1, 2, 3, 4, 5, 6, 7, 8, 9])
    u = 4
    _, dist, par = orc.bfs(g, u)
    R, _ = orc.sample_aggregate(g, u, par, 0, 13, seed=1)
    x, _, _, _ = orc.cg(g, u)
    d = orc.combine(R, 13, x, u)
    np.testing.assert_allclose(d, np.diag(orc.dense_pinv(g)), atol=1e-12)


def test_tau_satisfies_union_bound(orc):
    """Proof of Theorem 2: tau = ecc^2 * ceil(...) is the smallest multiple of
    ecc^2 for which Hoeffding's bound per edge, 2 exp(-2 (eps'/ecc)^2 tau), is
    at most delta / m, with eps' = (1 - kappa) eps."""
    for ecc, m, n, eps in [(8, 10 ** 7, 10 ** 6, 0.3), (48, 4512, 2304, 0.3), (5, 908998, 46589, 0.9),
                           (3, 100, 50, 0.5)]:
        delta = 1.0 / n
        t = orc.tau(ecc, m, eps, delta, 0.3)
        e1 = (1 - 0.3) * eps / ecc
        assert t % (ecc * ecc) == 0
        assert 2 * math.exp(-2 * e1 * e1 * t) <= delta / m * (1 + 1e-12)
        t_less = t - ecc * ecc
        assert 2 * math.exp(-2 * e1 * e1 * t_less) > delta / m


# ---------------------------------------------------------------- estimate

def test_estimate_within_clt_and_hoeffding(orc):
    """R/tau estimates r(u, v) (Section 3.2); the error stays inside the
    Hoeffding guarantee and inside 5 standard errors of the per-tree counts."""
    g = synth.grid(8, 8)
    u = 27
    ecc, dist, par = orc.bfs(g, u)
    tau = 3000
    per = np.zeros((tau, g.n), dtype=np.int64)
    for t in range(tau):
        nxt, _, _ = orc.wilson(g, u, t, 77)
        per[t] = orc.aggregate(nxt, par, u)
    Lp = orc.dense_pinv(g)
    r = orc.effective_resistance(Lp, u)
    est = per.mean(axis=0)
    se = per.std(axis=0) / math.sqrt(tau)
    err = np.abs(est - r)
    assert np.all(err <= 5 * se + 1e-12), np.max(err / (se + 1e-30))
    hoeff = ecc * math.sqrt(math.log(2 * g.m * g.n) / (2 * tau))
    assert err.max() <= hoeff
    # the full pipeline of Algorithm 1 against the dense diagonal
    d, R, x, _ = orc.diag(g, u, tau, seed=77)
    assert np.array_equal(R, per.sum(axis=0))
    np.testing.assert_allclose(d[u], Lp[u, u], atol=1e-10)
    assert np.max(np.abs(d - np.diag(Lp))) <= 5 * se.max() + 1e-9


def test_estimate_closed_form_cycle(orc):
    """On C_n every spanning tree drops one edge; R/tau -> k(n-k)/n."""
    n = 9
    g = synth.cycle(n)
    _, _, par = orc.bfs(g, 0)
    tau = 9000
    R, _ = orc.sample_aggregate(g, 0, par, 0, tau, seed=3)
    k = np.arange(n)
    # per-tree count for vertex k is in {k - (n - k), k} ... bounded by n
    np.testing.assert_allclose(R / tau, k * (n - k) / n, atol=5 * n / math.sqrt(tau))


# ---------------------------------------------------------------- centralities

def test_farness_from_diagonal_equals_sum_of_resistances():
    """Eq. elec-farness: sum_w r(v, w) = n L+[v,v] + tr(L+), checked against
    effective resistances summed pair by pair from the dense pseudoinverse."""
    import oracle
    for g in small_graphs():
        Lp = oracle.dense_pinv(g)
        d = np.diag(Lp)
        R = d[:, None] + d[None, :] - 2 * Lp  # Eq. eff-res, every pair
        c = oracle.centralities(d)
        np.testing.assert_allclose(c["farness"], R.sum(axis=1), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(c["closeness"], (g.n - 1) / R.sum(axis=1), rtol=1e-12)
        # Kirchhoff index: the sum of r over unordered pairs (Klein and Randic)
        assert math.isclose(c["kirchhoff"], R.sum() / 2, rel_tol=1e-12)


def test_centralities_closed_forms():
    import oracle
    for n in (5, 8, 13):
        c = oracle.centralities(np.diag(oracle.dense_pinv(synth.complete(n))))
        np.testing.assert_allclose(c["closeness"], n / 2, rtol=1e-12)      # r = 2/n to the n-1 others
        assert math.isclose(c["kirchhoff"], n - 1, rel_tol=1e-12)
        np.testing.assert_allclose(c["nrwb"], 1 / n + 1 / (2 * (n - 1)), rtol=1e-12)
        c = oracle.centralities(np.diag(oracle.dense_pinv(synth.cycle(n))))
        np.testing.assert_allclose(c["closeness"], 6 / (n + 1), rtol=1e-12)  # sum_k k(n-k)/n = (n^2-1)/6
        assert math.isclose(c["kirchhoff"], n * (n * n - 1) / 12, rel_tol=1e-12)
        c = oracle.centralities(np.diag(oracle.dense_pinv(synth.star(n))))
        assert math.isclose(c["kirchhoff"], (n - 1) ** 2, rel_tol=1e-12)   # n-1 pairs at 1, the rest at 2


def test_nrwb_equals_ratio_of_sums_over_inverse_of_L_plus_P():
    """The NRWB lemma against its derivation, computed straight from
    M^{-1} = (L + J/n)^{-1}: 1/n + (sum_t M_tt - M_tv) / ((n-1) sum_t (M_tt + M_vv - 2 M_tv))."""
    import oracle
    for g in small_graphs() + [synth.star(6), synth.path(7)]:
        n = g.n
        L = oracle.laplacian(g)
        M1 = np.linalg.inv(L + np.ones((n, n)) / n)
        ref = np.empty(n)
        for v in range(n):
            t = np.arange(n) != v
            num = np.sum(M1[t, t] - M1[t, v])
            den = np.sum(M1[t, t] + M1[v, v] - 2 * M1[t, v])
            ref[v] = 1.0 / n + num / ((n - 1) * den)
        c = oracle.centralities(np.diag(oracle.dense_pinv(g)))
        np.testing.assert_allclose(c["nrwb"], ref, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- edge counts

def _undirected(g, arc_values):
    """Sum of both arcs of every undirected edge, keyed by (a, b), a < b."""
    rp, ci = g.row_ptr, g.col_idx
    out = {}
    for v in range(g.n):
        for k in range(rp[v], rp[v + 1]):
            w = int(ci[k])
            key = (min(v, w), max(v, w))
            out[key] = out.get(key, 0) + arc_values[k]
    return out


def test_edge_frequency_over_all_spanning_trees_is_effective_resistance():
    """Kirchhoff: the fraction of all spanning trees that contain e equals
    r(e). The oracle's arc extraction applied to every enumerated tree (rooted
    at each pivot) reproduces the dense-pinv resistances exactly."""
    import oracle
    for g in tiny_graphs():
        Lp = oracle.dense_pinv(g)
        trees = oracle.spanning_trees(g)
        for u in (0, g.n - 1):
            counts = np.zeros(g.nnz, dtype=np.int64)
            for te in trees:
                np.add.at(counts, oracle.tree_arcs(g, oracle.root_tree(te, g.n, u), u), 1)
            assert counts.sum() == len(trees) * (g.n - 1)
            for (a, b), c in _undirected(g, counts).items():
                r = Lp[a, a] + Lp[b, b] - 2 * Lp[a, b]
                assert abs(c / len(trees) - r) <= 1e-12, (g.name, a, b)


def test_sampled_edge_frequencies_match_resistances():
    """Sampled trees: every tree has n-1 arcs, bridges are in every tree, and
    edge frequencies are within 5 standard errors of r(e)."""
    import oracle
    g = synth.from_edges(8, [0, 1, 2, 0, 3, 4, 5, 6, 5], [1, 2, 0, 3, 4, 5, 6, 7, 7], name="two-blocks")
    T = 3000
    counts = oracle.edge_counts(g, 0, 0, T, seed=4)
    assert counts.sum() == T * (g.n - 1)
    Lp = oracle.dense_pinv(g)
    for (a, b), c in _undirected(g, counts).items():
        r = Lp[a, a] + Lp[b, b] - 2 * Lp[a, b]
        f = c / T
        if abs(r - 1.0) < 1e-12:
            assert c == T  # a bridge is in every spanning tree
        sigma = math.sqrt(max(r * (1 - r), 1e-12) / T)
        assert abs(f - r) <= 5 * sigma + 1e-12, (a, b, f, r)


# ---------------------------------------------------------------- pivot selection

def _exact_ecc(g):
    A = csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    return shortest_path(A, unweighted=True).max(axis=1).astype(np.int64)


def test_double_sweep_bounds_are_lower_bounds_and_exact_on_trees():
    import oracle
    for g in small_graphs() + [synth.grid(9, 7), synth.rmat(8, 4, seed=3)]:
        ecc = _exact_ecc(g)
        piv, bound = oracle.select_pivot(g, sweeps=10)
        assert bound <= ecc[piv]                        # a lower bound
        assert bound <= ecc.min()                       # the least bound never exceeds the radius
    rng = np.random.default_rng(5)
    for n in (9, 17, 40):
        parent = [int(rng.integers(0, v)) for v in range(1, n)]  # a random tree
        t = synth.from_edges(n, list(range(1, n)), parent, name=f"tree{n}")
        ecc = _exact_ecc(t)
        piv, bound = oracle.select_pivot(t, sweeps=3)
        # on a tree the second and third sources are the two ends of a diameter,
        # and ecc(x) = max(dist(x, a), dist(x, b)) for those ends: the bound is exact
        assert bound == ecc[piv] == ecc.min()
    piv, bound = oracle.select_pivot(synth.path(21), sweeps=2)
    assert (piv, bound) == (10, 10)
    # 9x9 grid: the sweeps alternate between opposite corners, so the bound of
    # the centre (8, the radius) is shared by other vertices; it is a bound,
    # not the eccentricity, and the least bound equals the radius here
    g = synth.grid(9, 9)
    piv, bound = oracle.select_pivot(g, sweeps=10)
    assert bound == 8 and _exact_ecc(g)[piv] >= 8


# --------------------------------------------- biconnected-component variant

def _block_example():
    """Triangle {0,1,2}, triangle {2,3,4}, square {4,5,6,7}, bridge {7,8}:
    cut vertices 2, 4 and 7, 3 * 3 * 4 * 1 = 36 spanning trees."""
    src = [0, 1, 0, 2, 3, 2, 4, 5, 6, 4, 7]
    dst = [1, 2, 2, 3, 4, 4, 5, 6, 7, 7, 8]
    return synth.from_edges(9, src, dst, lcc=False)


def _same_partition(a, b) -> bool:
    m1, m2 = {}, {}
    for x, y in zip(a, b):
        if m1.setdefault(x, y) != y or m2.setdefault(y, x) != x:
            return False
    return True


def test_blocks_textbook_cases(orc):
    """Every edge of a tree is a bridge (its own block); a cycle, a grid and a
    complete graph are one block; the example has its four blocks."""
    for g, nb in [(synth.path(7), 6), (synth.star(6), 5), (synth.ba(60, 1, seed=3), 59), (synth.cycle(9), 1),
                  (synth.grid(5, 4), 1), (synth.complete(6), 1)]:
        ab = orc.blocks(g)
        assert len(set(ab.tolist())) == nb
        src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        rev = {(int(a), int(b)): int(x) for a, b, x in zip(src, g.col_idx, ab)}
        assert all(rev[(b, a)] == x for (a, b), x in rev.items())  # both arcs of an edge agree
    ab = orc.blocks(_block_example())
    sizes = sorted(np.bincount(ab).tolist())
    assert sizes == [2, 6, 6, 8]  # arcs per block: bridge, two triangles, square


def test_blocks_match_networkx(orc):
    """The oracle's Hopcroft-Tarjan blocks equal networkx's biconnected
    components (an independent implementation) on sparse random graphs."""
    nx = pytest.importorskip("networkx")
    graphs = [synth.er(400, 2.2, seed=s) for s in range(4)] + [synth.ba(300, 2, seed=5), synth.rmat(10, 4, seed=3),
                                                               _block_example()]
    for g in graphs:
        G = nx.Graph()
        G.add_edges_from(map(tuple, g.edges().tolist()))
        ref = {}
        for b, es in enumerate(nx.biconnected_component_edges(G)):
            for a, c in es:
                ref[(a, c)] = ref[(c, a)] = b
        src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        want = [ref[(int(a), int(c))] for a, c in zip(src, g.col_idx)]
        assert _same_partition(orc.blocks(g).tolist(), want)


def test_parent_block_walks_sample_uniform_trees_toward_u(orc):
    """Appendix D's biconnected-component variant in the form that was measured
    (and not built): every vertex v != u walks only inside its parent block.
    Every cycle lies in one block, so each block pops its cycles on its own and
    yields a uniform tree of the block rooted at its vertex nearest u; their
    union is uniform over the spanning trees of G and already oriented toward
    u. Brute force: chi-square over all 36 spanning trees, and every sample a
    tree of G rooted at u."""
    g = _block_example()
    u = 5
    w = orc.parent_block_graph(g, u)
    assert w.nnz < g.nnz  # the cut vertices 2, 4 and 7 lose their other blocks
    assert w.row_ptr[u + 1] == w.row_ptr[u]  # the root draws nothing
    trees = orc.spanning_trees(g)
    assert len(trees) == 3 * 3 * 4 * 1
    index = {t: i for i, t in enumerate(trees)}
    counts = np.zeros(len(trees), dtype=np.int64)
    for t in range(400 * len(trees)):
        nxt, _, _ = orc.cycle_pop(w, u, t, 99)
        edges = orc.tree_edges_of(nxt)
        assert np.array_equal(orc.root_tree(edges, g.n, u), nxt)
        counts[index[edges]] += 1
    assert stats.chisquare(counts).pvalue > 1e-4, counts
