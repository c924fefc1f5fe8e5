"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work (B_u, sampled trees, pop counts, R) must match bit for bit.
Floating point: the column x = L^+[:, u] within 1e-8 of an FP64 reference
(dense pseudoinverse or FP64 CG at 1e-13); the diagonal within 1e-12
relative of the oracle's combination applied to the same R and x.
"""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))
COL_TOL = 1e-8     # column vs FP64 reference, absolute, scaled by max(1, |x|_inf)
DIAG_RTOL = 1e-12  # diag vs oracle combine on the same (R, x)


@pytest.fixture(scope="module")
def pkg():
    import paper_2006_13679_gb300 as p
    p.build()
    return p


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.lib()
    return oracle


def make(pkg, g, u, **kw):
    return pkg.UST(g.row_ptr, g.col_idx, u, **kw)


GRAPHS = {
    "grid48": lambda: (synth.grid(48, 48), 24 * 48 + 24),
    "rmat12": lambda: (lambda g: (g, synth.max_degree_vertex(g)))(synth.rmat(12, 16, seed=5)),
    "ba3000": lambda: (lambda g: (g, synth.max_degree_vertex(g)))(synth.ba(3000, 4, seed=2)),
    "er2000": lambda: (lambda g: (g, synth.max_degree_vertex(g)))(synth.er(2000, 6.0, seed=3)),
    "path50": lambda: (synth.path(50), 17),
    "k2": lambda: (synth.path(2), 1),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_bfs_tree(pkg, orc, name):
    g, u = GRAPHS[name]()
    with make(pkg, g, u) as h:
        par, dist = h.bfs()
        ecc, d_ref, p_ref = orc.bfs(g, u)
        assert np.array_equal(dist, d_ref)
        assert np.array_equal(par, p_ref)
        info = h.info()
        assert info["ecc"] == ecc
        assert info["farness"] == int(d_ref.astype(np.int64).sum())


@pytest.mark.parametrize("name", ["grid48", "rmat12", "ba3000", "er2000"])
def test_sampled_trees_bit_exact(pkg, orc, name):
    """Every sampled tree and every per-vertex pop count equals the
    sequential loop-erased-walk tree on the same stacks."""
    g, u = GRAPHS[name]()
    seed = 0x1234_5678_9ABC_DEF0
    with make(pkg, g, u) as h:
        nxt, pops = h.sample_trees(3, 40, seed, with_pops=True)
        for i in range(40):
            ref, ref_pops, _ = orc.wilson(g, u, 3 + i, seed)
            assert np.array_equal(nxt[i], ref), (name, i)
            assert np.array_equal(pops[i], ref_pops), (name, i)


def test_counts_grid48_full(pkg, orc):
    """48x48 grid, pivot 1176, 1000 trees, seed 0: R bit-exact."""
    g, u = GRAPHS["grid48"]()
    with make(pkg, g, u) as h:
        h.sample_aggregate(1000, 0)
        R = h.counts()
        _, _, par = orc.bfs(g, u)
        R_ref, steps = orc.sample_aggregate(g, u, par, 0, 1000, 0, threads=THREADS)
        assert np.array_equal(R, R_ref)
        info = h.info()
        assert info["trees"] == 1000 and info["draws"] == steps


def test_counts_rmat16_full(pkg, orc):
    """R-MAT scale 16, edge factor 16, LCC, max-degree pivot, 4096 trees, in
    the sampler's default launch configuration: R bit-exact."""
    g, u, T, _ = synth.workload("rmat16")
    with make(pkg, g, u) as h:
        h.sample_aggregate(T, 0)
        R = h.counts()
        _, _, par = orc.bfs(g, u)
        R_ref, steps = orc.sample_aggregate(g, u, par, 0, T, 0, threads=THREADS)
        assert np.array_equal(R, R_ref)
        assert h.info()["draws"] == steps


def test_calls_continue_tree_ids(pkg, orc):
    g = synth.grid(7, 5)
    u = 17
    with make(pkg, g, u) as a, make(pkg, g, u) as b:
        a.sample_aggregate(37, 9)
        for k in (1, 5, 31):
            b.sample_aggregate(k, 9)
        assert np.array_equal(a.counts(), b.counts())
        assert a.info()["trees"] == b.info()["trees"] == 37
        assert a.num_trees() == b.num_trees() == 37
        _, _, par = orc.bfs(g, u)
        R_ref, _ = orc.sample_aggregate(g, u, par, 0, 37, 9)
        assert np.array_equal(a.counts(), R_ref)
        # a tree range that does not start at 0
        assert np.array_equal(a.tree_range_counts(5, 36, 9), orc.sample_aggregate(g, u, par, 5, 36, 9)[0])


@pytest.mark.parametrize("maker,u", [(lambda: synth.path(2), 0), (lambda: synth.path(31), 0),
                                     (lambda: synth.star(20), 0), (lambda: synth.star(20), 7),
                                     (lambda: synth.complete(9), 4), (lambda: synth.cycle(13), 12),
                                     (lambda: synth.grid(1, 40), 39)])
def test_edge_graphs(pkg, orc, maker, u):
    g = maker()
    with make(pkg, g, u) as h:
        h.sample_aggregate(301, 77)
        _, dist, par = orc.bfs(g, u)
        R_ref, _ = orc.sample_aggregate(g, u, par, 0, 301, 77)
        assert np.array_equal(h.counts(), R_ref)
        if g.m == g.n - 1:  # a tree: every UST is G itself
            assert np.array_equal(h.counts(), 301 * dist.astype(np.int64))


@pytest.mark.parametrize("bt,cps", [(64, 0), (128, 0), (256, 1), (256, 8), (512, 2), (1024, 1)])
def test_launch_configurations_agree(pkg, orc, bt, cps):
    g, u = GRAPHS["rmat12"]()
    with make(pkg, g, u, block_threads=bt, ctas_per_sm=cps) as h:
        h.sample_aggregate(500, 3)
        _, _, par = orc.bfs(g, u)
        R_ref, _ = orc.sample_aggregate(g, u, par, 0, 500, 3, threads=THREADS)
        assert np.array_equal(h.counts(), R_ref)


def test_column_and_diag_grid48(pkg, orc):
    g, u = GRAPHS["grid48"]()
    Lp = orc.dense_pinv(g)
    with make(pkg, g, u) as h:
        h.sample_aggregate(1000, 0)
        x = h.column()
        assert np.max(np.abs(x - Lp[:, u])) <= COL_TOL * max(1.0, np.max(np.abs(Lp[:, u])))
        assert abs(x.sum()) < 1e-9
        info = h.info()
        assert info["cg_relres"] <= 1e-9
        d = h.diag()
        R = h.counts()
        ref = orc.combine(R, 1000, x, u)
        np.testing.assert_allclose(d, ref, rtol=DIAG_RTOL, atol=0)
        # within the Hoeffding guarantee of tau = 1000 trees (Theorem 2)
        ecc = info["ecc"]
        eps_tau = ecc * np.sqrt(np.log(2 * g.m * g.n) / (2 * 1000)) / (1 - 0.3)
        assert np.max(np.abs(d - np.diag(Lp))) <= eps_tau


def test_column_rmat16_against_fp64_cg(pkg, orc):
    g, u, T, _ = synth.workload("rmat16")
    with make(pkg, g, u) as h:
        x = h.column()
        x_ref, _, rr, ok = orc.cg(g, u, tol=1e-13)
        assert ok
        assert np.max(np.abs(x - x_ref)) <= COL_TOL * max(1.0, np.max(np.abs(x_ref)))
        assert h.info()["cg_relres"] <= 1e-9


def test_diag_tops_up_to_tau(pkg, orc):
    g = synth.grid(10, 10)
    u = 55
    with make(pkg, g, u) as h:
        h.sample_aggregate(10, 4)
        tau = h.tau(2.0)
        ecc, _, _ = orc.bfs(g, u)
        assert tau == orc.tau(ecc, g.m, 2.0, 1.0 / g.n, 0.3)
        d = h.diag(2.0)
        assert h.info()["trees"] == tau
        np.testing.assert_allclose(d, orc.combine(h.counts(), tau, h.column(), u), rtol=DIAG_RTOL, atol=0)
        Lp = orc.dense_pinv(g)
        assert np.max(np.abs(d - np.diag(Lp))) <= 2.0


def test_error_paths(pkg):
    from paper_2006_13679_gb300 import UstError, UST_ENOTCONNECTED, UST_EINVAL, UST_ESTATE, UST_ETIMEOUT
    g = synth.from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5], lcc=False)
    with pytest.raises(UstError) as e:
        make(pkg, g, 0)
    assert e.value.code == UST_ENOTCONNECTED
    rp = np.array([0, 1, 2, 2], dtype=np.int32)  # arc 0->1, 1->2 without reverses
    ci = np.array([1, 2], dtype=np.int32)
    with pytest.raises(UstError) as e:
        pkg.UST(rp, ci, 0)
    assert e.value.code in (UST_EINVAL, UST_ENOTCONNECTED)
    g, u = GRAPHS["grid48"]()
    with make(pkg, g, u) as h:
        with pytest.raises(UstError) as e:
            h.diag()
        assert e.value.code == UST_ESTATE
    with make(pkg, g, u, max_pop_rounds=1) as h:
        with pytest.raises(UstError) as e:
            h.sample_aggregate(8, 0)
        assert e.value.code == UST_ETIMEOUT
        assert h.info()["trees"] == 0
        assert not h.counts().any()


def test_device_pointers(pkg, orc):
    import torch
    g, u = GRAPHS["rmat12"]()
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    st = torch.cuda.Stream()
    with pkg.UST(rp, ci, u, stream=st) as h:
        h.sample_aggregate(200, 1)
        R = torch.empty(g.n, dtype=torch.int64, device="cuda")
        h.counts(R)
        d = torch.empty(g.n, dtype=torch.float64, device="cuda")
        h.diag(0.0, d)
        st.synchronize()
        _, _, par = orc.bfs(g, u)
        R_ref, _ = orc.sample_aggregate(g, u, par, 0, 200, 1)
        assert np.array_equal(R.cpu().numpy(), R_ref)
        x = h.column()
        np.testing.assert_allclose(d.cpu().numpy(), orc.combine(R_ref, 200, x, u), rtol=DIAG_RTOL, atol=0)


def test_repeat_runs_are_identical(pkg):
    g, u = GRAPHS["ba3000"]()
    with make(pkg, g, u) as a, make(pkg, g, u) as b:
        a.sample_aggregate(300, 11)
        b.sample_aggregate(300, 11)
        assert np.array_equal(a.counts(), b.counts())
        assert np.array_equal(a.diag(), b.diag())


@pytest.mark.parametrize("maker", [lambda: synth.ba(70000, 3, seed=9), lambda: synth.rmat(17, 8, seed=2)])
def test_counts_above_shared_memory_limit(pkg, orc, maker):
    """Graphs with more than 65,535 vertices keep their per-tree counters in
    global memory instead of shared memory: R bit-exact as well."""
    g = maker()
    assert g.n > 0xFFFF
    u = synth.max_degree_vertex(g)
    with make(pkg, g, u) as h:
        h.sample_aggregate(300, 21)
        _, _, par = orc.bfs(g, u)
        R_ref, steps = orc.sample_aggregate(g, u, par, 0, 300, 21, threads=THREADS)
        assert np.array_equal(h.counts(), R_ref)
        assert h.info()["draws"] == steps
        nxt, pops = h.sample_trees(100, 3, 21, with_pops=True)
        for i in range(3):
            ref, ref_pops, _ = orc.wilson(g, u, 100 + i, 21)
            assert np.array_equal(nxt[i], ref) and np.array_equal(pops[i], ref_pops)


@pytest.mark.parametrize("bt,cps", [(512, 1), (512, 2), (1024, 1)])
def test_large_sampler_shapes_agree(pkg, orc, bt, cps):
    """The large-graph sampler at every shape the launch tuner may pick: R
    and the draws bit-exact."""
    g = synth.rmat(17, 8, seed=2)
    u = synth.max_degree_vertex(g)
    with make(pkg, g, u, block_threads=bt, ctas_per_sm=cps) as h:
        h.sample_aggregate(300, 13)
        _, _, par = orc.bfs(g, u)
        R_ref, steps = orc.sample_aggregate(g, u, par, 0, 300, 13, threads=THREADS)
        assert np.array_equal(h.counts(), R_ref)
        assert h.info()["draws"] == steps


@pytest.mark.parametrize("maker,bt", [
    (lambda: synth.ba(57345, 3, seed=4), 0),     # the first tail word in use
    (lambda: synth.er(60000, 10.0, seed=6), 0),
    (lambda: synth.er(60000, 10.0, seed=6), 256),
    (lambda: synth.ba(65535, 2, seed=8), 0),     # the largest graph with 16-bit ids
])
def test_counts_with_shared_words_in_a_global_tail(pkg, orc, maker, bt):
    """Graphs between 56k and 65,535 vertices run the shared-memory sampler
    with its last words in a per-CTA global tail: R, the draws and sampled
    trees with their pop counts bit-exact."""
    g = maker()
    assert 56 * 1024 < g.n <= 0xFFFF
    u = synth.max_degree_vertex(g)
    with make(pkg, g, u, block_threads=bt) as h:
        h.sample_aggregate(200, 23)
        _, _, par = orc.bfs(g, u)
        R_ref, steps = orc.sample_aggregate(g, u, par, 0, 200, 23, threads=THREADS)
        assert np.array_equal(h.counts(), R_ref)
        assert h.info()["draws"] == steps
        nxt, pops = h.sample_trees(50, 3, 23, with_pops=True)
        for i in range(3):
            ref, ref_pops, _ = orc.wilson(g, u, 50 + i, 23)
            assert np.array_equal(nxt[i], ref) and np.array_equal(pops[i], ref_pops)


def test_all_fp64_solve_matches(pkg, orc):
    """The all-FP64 form of the column solve (the reference form the mixed
    precision solve is compared with) reaches the same column."""
    g, u, T, _ = synth.workload("rmat16")
    with make(pkg, g, u, solve_fp64=True) as h:
        x = h.column()
        x_ref, _, _, ok = orc.cg(g, u, tol=1e-13)
        assert ok and h.info()["cg_relres"] <= 1e-9
        assert np.max(np.abs(x - x_ref)) <= COL_TOL * max(1.0, np.max(np.abs(x_ref)))


def test_one_tree_per_launch_equals_batched(pkg, orc):
    g, u = GRAPHS["rmat12"]()
    with make(pkg, g, u) as a, make(pkg, g, u) as b:
        a.sample_aggregate(64, 5)
        for _ in range(64):
            b.sample_aggregate(1, 5)
        assert np.array_equal(a.counts(), b.counts())


def test_sharded_tree_ranges_equal_one_run(pkg, orc):
    """Two ranks' tree ranges under one seed, summed and installed with
    ust_set_counts, give the counts and diagonal of one context that sampled
    all the trees (the multi-GPU path, emulated in one process)."""
    from paper_2006_13679_gb300 import parallel
    g, u = synth.rmat(12, 16, seed=5), None
    u = synth.max_degree_vertex(g)
    T = 300
    with pkg.UST(g.row_ptr, g.col_idx, u) as h1, pkg.UST(g.row_ptr, g.col_idx, u) as h2:
        h1.sample_aggregate(2 * T, 5)
        R = sum(h2.tree_range_counts(*parallel.tree_range(r, 2, T), 5) for r in range(2))
        h2.set_counts(R, 2 * T)
        assert np.array_equal(h2.counts(), h1.counts())
        assert h2.info()["trees"] == 2 * T
        np.testing.assert_array_equal(h2.diag(), h1.diag())
        with pytest.raises(pkg.UstError):
            h2.set_counts(R, 0)


@pytest.mark.parametrize("case,rp,ci,code", [
    ("row_ptr not monotone", [0, 2, 1, 4], [1, 2, 0, 0], "EINVAL"),
    ("row_ptr end != nnz", [0, 1, 2, 2], [1, 0, 0], "EINVAL"),
    ("column out of range", [0, 1, 2], [1, 2], "EINVAL"),
    ("self-loop", [0, 2, 3], [0, 1, 0], "EINVAL"),
    ("unsorted row", [0, 2, 3, 4], [2, 1, 0, 0], "EINVAL"),
    ("duplicate arc", [0, 2, 4], [1, 1, 0, 0], "EINVAL"),
    ("asymmetric", [0, 2, 4, 5], [1, 2, 0, 2, 0], "EINVAL"),
    ("isolated vertex", [0, 1, 2, 2], [1, 0], "ENOTCONNECTED"),
])
def test_input_checks_on_device(pkg, case, rp, ci, code):
    """ust_init checks the CSR on the device: every malformed input is
    rejected with its error code and nothing else runs on it."""
    rp = np.array(rp, dtype=np.int32)
    ci = np.array(ci, dtype=np.int32)
    with pytest.raises(pkg.UstError) as e:
        pkg.UST(rp, ci, 0)
    assert e.value.code == getattr(pkg, "UST_" + code), case


def test_batch_input_checks_name_the_graph(pkg):
    good = synth.grid(4, 4)
    bad_rp = np.array([0, 2, 4, 5], dtype=np.int32)
    bad_ci = np.array([1, 2, 0, 2, 0], dtype=np.int32)  # 1 -> 2 without 2 -> 1
    with pytest.raises(pkg.UstError) as e:
        pkg.USTBatch([(good.row_ptr, good.col_idx), (bad_rp, bad_ci)], [0, 0])
    assert e.value.code == pkg.UST_EINVAL
    assert "graph 1" in str(e.value)


@pytest.mark.parametrize("name", ["grid48", "rmat12"])
def test_centralities_from_the_diagonal(pkg, orc, name):
    """ust_centralities: closeness, NRWB and Kirchhoff index of the estimated
    diagonal equal the oracle's formulas applied to the same diagonal."""
    g, u = GRAPHS[name]()
    with make(pkg, g, u) as h:
        h.sample_aggregate(400, 3)
        d = h.diag()
        c = h.centralities()
    ref = orc.centralities(d)
    np.testing.assert_allclose(c["closeness"], ref["closeness"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(c["nrwb"], ref["nrwb"], rtol=1e-12, atol=0)
    assert abs(c["kirchhoff"] - ref["kirchhoff"]) <= 1e-12 * abs(ref["kirchhoff"])


@pytest.mark.parametrize("name,trees", [("grid48", 120), ("rmat12", 200), ("ba70000", 6)])
def test_edge_counts_bit_exact(pkg, orc, name, trees):
    """ust_track_edges: per-arc tree counts equal the oracle's, in both the
    shared-memory and the global-memory sampler."""
    if name == "ba70000":
        g = synth.ba(70000, 3, seed=9)
        u = synth.max_degree_vertex(g)
    else:
        g, u = GRAPHS[name]()
    with make(pkg, g, u) as h:
        h.track_edges(True)
        h.sample_aggregate(trees // 2, 13)
        h.sample_aggregate(trees - trees // 2, 13)
        got = h.edge_counts()
        assert got.sum() == trees * (g.n - 1)
        assert np.array_equal(got, orc.edge_counts(g, u, 0, trees, 13))
        if name == "grid48":
            with pytest.raises(pkg.UstError):
                h2 = make(pkg, g, u, max_pop_rounds=1)
                h2.track_edges(True)
                try:
                    h2.sample_aggregate(4, 0)
                finally:
                    assert not h2.edge_counts().any()  # a failed call leaves the counts unchanged
                    h2.close()
            h.reset(u)
            assert not h.edge_counts().any()


@pytest.mark.parametrize("name", ["grid48", "rmat12", "ba3000", "er2000", "path50"])
def test_select_pivot_equals_oracle(pkg, orc, name):
    """ust_select_pivot: the same pivot and eccentricity bound as the oracle's
    double sweeps (integer results, equal exactly)."""
    g, _ = GRAPHS[name]()
    for sweeps, start in ((10, -1), (3, 0)):
        assert pkg.select_pivot(g.row_ptr, g.col_idx, sweeps, start) == orc.select_pivot(g, sweeps, start)


def test_select_pivot_rejects_disconnected(pkg):
    g = synth.from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5], lcc=False)
    with pytest.raises(pkg.UstError) as e:
        pkg.select_pivot(g.row_ptr, g.col_idx)
    assert e.value.code == pkg.UST_ENOTCONNECTED


# ------------------------------------------- biconnected-component variant

def _block_example():
    src = [0, 1, 0, 2, 3, 2, 4, 5, 6, 4, 7]
    dst = [1, 2, 2, 3, 4, 4, 5, 6, 7, 7, 8]
    return synth.from_edges(9, src, dst, lcc=False)


BLOCK_GRAPHS = {
    "example": lambda: (_block_example(), 5),
    "tree": lambda: (lambda g: (g, synth.max_degree_vertex(g)))(synth.ba(500, 1, seed=4)),
    "er_sparse": lambda: (lambda g: (g, synth.max_degree_vertex(g)))(synth.er(3000, 2.5, seed=7)),
    "rmat12": GRAPHS["rmat12"],
    "ba3000": GRAPHS["ba3000"],
}


@pytest.mark.parametrize("name", sorted(BLOCK_GRAPHS))
def test_block_variant_bit_exact(pkg, orc, name):
    """wilson_blocks: the device's Tarjan-Vishkin rows give the same trees,
    counts and draws as the oracle's Hopcroft-Tarjan rows."""
    g, u = BLOCK_GRAPHS[name]()
    w = orc.parent_block_graph(g, u)
    _, _, par = orc.bfs(g, u)
    with make(pkg, g, u, wilson_blocks=True) as h:
        h.sample_aggregate(300, 31)
        R_ref, steps = orc.sample_aggregate(w, u, par, 0, 300, 31, threads=THREADS)
        assert np.array_equal(h.counts(), R_ref)
        assert h.info()["draws"] == steps
        nxt, pops = h.sample_trees(10, 3, 31, with_pops=True)
        for i in range(3):
            ref, ref_pops, _ = orc.wilson(w, u, 10 + i, 31)
            assert np.array_equal(nxt[i], ref) and np.array_equal(pops[i], ref_pops)


def test_block_variant_on_one_block_equals_plain_wilson(pkg, orc):
    """A grid is one block: the restricted rows are the full rows (the root's
    is unused), so the trees are plain Wilson's."""
    g, u = synth.grid(12, 12), 78
    with make(pkg, g, u, wilson_blocks=True) as a, make(pkg, g, u) as b:
        a.sample_aggregate(200, 5)
        b.sample_aggregate(200, 5)
        assert np.array_equal(a.counts(), b.counts())


def test_block_variant_reset_and_edge_counts(pkg, orc):
    """ust_reset rebuilds the rows for the new pivot; arc counts are reported
    per arc of the input graph."""
    g = synth.er(2000, 3.0, seed=11)
    u0, u1 = synth.max_degree_vertex(g), 17
    with make(pkg, g, u0, wilson_blocks=True) as h:
        h.sample_aggregate(50, 2)
        h.reset(u1)
        h.track_edges(True)
        h.sample_aggregate(120, 9)
        w = orc.parent_block_graph(g, u1)
        _, _, par = orc.bfs(g, u1)
        R_ref, _ = orc.sample_aggregate(w, u1, par, 0, 120, 9, threads=THREADS)
        assert np.array_equal(h.counts(), R_ref)
        assert np.array_equal(h.edge_counts(), orc.edge_counts(g, u1, 0, 120, 9, walk=w))


def test_block_variant_rmat16_full(pkg, orc):
    """The bench workload (R-MAT16, 4096 trees) with the variant."""
    g, u, T, _ = synth.workload("rmat16")
    w = orc.parent_block_graph(g, u)
    _, _, par = orc.bfs(g, u)
    with make(pkg, g, u, wilson_blocks=True) as h:
        h.sample_aggregate(T, 0)
        R_ref, steps = orc.sample_aggregate(w, u, par, 0, T, 0, threads=THREADS)
        assert np.array_equal(h.counts(), R_ref)
        assert h.info()["draws"] == steps


def test_block_variant_rejected_for_batches(pkg):
    gs = [synth.grid(4, 4), synth.cycle(10)]
    with pytest.raises(pkg.UstError) as ei:
        pkg.USTBatch([(g.row_ptr, g.col_idx) for g in gs], [0, 0], wilson_blocks=True)
    assert ei.value.code == pkg.UST_EINVAL


def _with_pendants(g, u, k, seed):
    """g plus k new vertices of degree 1, each joined to a random vertex of g
    (the first three to the pivot u), and a path of two new vertices hanging
    from vertex 0: the vertex at its end is pendant, its neighbour is not."""
    rng = np.random.default_rng(seed)
    deg = np.diff(g.row_ptr)
    src = [np.repeat(np.arange(g.n), deg), np.arange(g.n, g.n + k), [g.n + k, g.n + k + 1]]
    tgt = rng.integers(0, g.n, k)
    tgt[:3] = u
    dst = [g.col_idx, tgt, [0, g.n + k]]
    return synth.from_edges(g.n + k + 2, np.concatenate(src), np.concatenate(dst), lcc=False)


def test_pendant_vertices_left_out_of_the_trees(pkg, orc):
    """Above 65,535 vertices the sampler builds its trees on the vertices of
    degree 2 and more (and the pivot) and derives the counts of degree-1
    vertices from their neighbours': R and the draw count bit-exact with the
    oracle's Wilson on the whole graph, here with a quarter of the vertices
    pendant, three of them at the pivot; sampled trees (every vertex) too."""
    base = synth.rmat(17, 8, seed=2)
    u = synth.max_degree_vertex(base)
    g = _with_pendants(base, u, 40000, seed=3)
    assert g.n > 0xFFFF and (np.diff(g.row_ptr) == 1).sum() > 40000
    _, _, par = orc.bfs(g, u)
    with make(pkg, g, u) as h:
        h.sample_aggregate(300, 17)
        R_ref, steps = orc.sample_aggregate(g, u, par, 0, 300, 17, threads=THREADS)
        assert np.array_equal(h.counts(), R_ref)
        assert h.info()["draws"] == steps
        nxt, pops = h.sample_trees(7, 2, 17, with_pops=True)
        for i in range(2):
            ref, ref_pops, _ = orc.wilson(g, u, 7 + i, 17)
            assert np.array_equal(nxt[i], ref) and np.array_equal(pops[i], ref_pops)


def test_pendant_pivot_keeps_every_vertex(pkg, orc):
    """After ust_reset to a pivot of degree 1 the trees take every vertex (the
    pivot is no pendant vertex of its own trees); back at a hub the pendant
    vertices are left out again. R bit-exact both times."""
    base = synth.rmat(17, 8, seed=2)
    u = synth.max_degree_vertex(base)
    g = _with_pendants(base, u, 20000, seed=5)
    leaf = g.n - 1  # the end of the hanging path
    with make(pkg, g, u) as h:
        for pivot in (leaf, u):
            h.reset(pivot)
            h.sample_aggregate(200, 29)
            _, _, par = orc.bfs(g, pivot)
            R_ref, steps = orc.sample_aggregate(g, pivot, par, 0, 200, 29, threads=THREADS)
            assert np.array_equal(h.counts(), R_ref), pivot
            assert h.info()["draws"] == steps
