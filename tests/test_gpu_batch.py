"""Batches of graphs (ust_init_batch): every graph's counts, column and
diagonal equal those of a single-graph context for the same graph, pivot and
graph id, and the counts equal the oracle's."""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))


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


def small_batch():
    gs = [synth.grid(20, 15), synth.ba(3000, 4, seed=1), synth.er(2500, 8.0, seed=2), synth.path(40),
          synth.rmat(11, 8, seed=3), synth.ba(60000, 3, seed=4)]  # the last exceeds the shared-memory sampler
    return gs, [synth.max_degree_vertex(g) for g in gs]


def test_batch_equals_single_graph_contexts(pkg, orc):
    gs, piv = small_batch()
    base = 11
    with pkg.USTBatch([(g.row_ptr, g.col_idx) for g in gs], piv, graph_id=base) as b:
        assert b.count == len(gs) and b.n == sum(g.n for g in gs)
        b.sample_aggregate(40, 9)
        b.sample_aggregate(60, 9)  # tree ids continue per graph
        R = b.split(b.counts())
        x = b.split(b.column())
        d = b.split(b.diag())
        for i, g in enumerate(gs):
            info = b.graph_info(i)
            assert info["n"] == g.n and info["trees"] == 100 and info["pivot"] == piv[i]
            with pkg.UST(g.row_ptr, g.col_idx, piv[i], graph_id=base + i) as h:
                h.sample_aggregate(100, 9)
                assert np.array_equal(R[i], h.counts()), i
                # both columns meet cg_tol = 1e-9; the two solver forms agree far inside the 1e-8 bar
                scale = max(1.0, float(np.max(np.abs(x[i]))))
                assert np.max(np.abs(x[i] - h.column())) <= 1e-9 * scale, i
            x_ref, _, _, ok = orc.cg(g, piv[i], tol=1e-12, max_iter=50000)
            assert ok
            assert np.max(np.abs(x[i] - x_ref)) <= 1e-8 * max(1.0, float(np.max(np.abs(x_ref)))), i
            ecc, _, par = orc.bfs(g, piv[i])
            assert info["ecc"] == ecc
            R_ref, _ = orc.sample_aggregate(g, piv[i], par, 0, 100, 9, graph=base + i, threads=THREADS)
            assert np.array_equal(R[i], R_ref), i
            np.testing.assert_allclose(d[i], orc.combine(R[i], 100, x[i], piv[i]), rtol=1e-12, atol=0)


def test_batch_tops_up_each_graph_to_its_tau(pkg, orc):
    gs = [synth.grid(6, 6), synth.cycle(30), synth.complete(12)]
    piv = [14, 0, 3]
    with pkg.USTBatch([(g.row_ptr, g.col_idx) for g in gs], piv) as b:
        b.diag(1.5)
        for i, g in enumerate(gs):
            ecc, _, _ = orc.bfs(g, piv[i])
            assert b.graph_info(i)["trees"] == orc.tau(ecc, g.m, 1.5, 1.0 / g.n, 0.3)


def test_batch_rejects_disconnected_graph(pkg):
    gs = [synth.grid(5, 5), synth.from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5], lcc=False)]
    with pytest.raises(pkg.UstError) as e:
        pkg.USTBatch([(g.row_ptr, g.col_idx) for g in gs], [0, 0])
    assert e.value.code == pkg.UST_ENOTCONNECTED


def test_batch_of_256_uneven_graphs(pkg, orc):
    """The batch workload: 256 BA/ER largest components with n in [1k, 64k]
    and average degree in [8, 32], max-degree pivots, 1024 trees each; counts
    of sampled graphs against the oracle."""
    specs = synth.batch_specs(256)
    gs = [synth.batch_graph(s) for s in specs]
    piv = [synth.max_degree_vertex(g) for g in gs]
    with pkg.USTBatch([(g.row_ptr, g.col_idx) for g in gs], piv, skip_validation=True) as b:
        b.sample_aggregate(1024, 0)
        R = b.split(b.counts())
        d = b.split(b.diag())
        x = b.split(b.column())
        for i in [0, 1, 127, 255, int(np.argmax([g.n for g in gs]))]:
            g = gs[i]
            _, _, par = orc.bfs(g, piv[i])
            R_ref, _ = orc.sample_aggregate(g, piv[i], par, 0, 1024, 0, graph=i, threads=THREADS)
            assert np.array_equal(R[i], R_ref), i
            x_ref, _, _, ok = orc.cg(g, piv[i], tol=1e-12, max_iter=50000)
            assert ok
            assert np.max(np.abs(x[i] - x_ref)) <= 1e-8 * max(1.0, float(np.max(np.abs(x_ref)))), i
            np.testing.assert_allclose(d[i], orc.combine(R[i], 1024, x[i], piv[i]), rtol=1e-12, atol=0)


def test_batch_centralities(pkg, orc):
    gs = [synth.grid(6, 6), synth.ba(2000, 4, seed=3), synth.cycle(40)]
    piv = [14, synth.max_degree_vertex(gs[1]), 0]
    with pkg.USTBatch([(g.row_ptr, g.col_idx) for g in gs], piv) as b:
        b.sample_aggregate(300, 4)
        d = b.split(b.diag())
        c = b.centralities()
        cl, nr = b.split(c["closeness"]), b.split(c["nrwb"])
        for i in range(len(gs)):
            ref = orc.centralities(d[i])
            np.testing.assert_allclose(cl[i], ref["closeness"], rtol=1e-12, atol=0)
            np.testing.assert_allclose(nr[i], ref["nrwb"], rtol=1e-12, atol=0)
            assert abs(c["kirchhoff"][i] - ref["kirchhoff"]) <= 1e-12 * abs(ref["kirchhoff"])


def test_batch_edge_counts(pkg, orc):
    gs = [synth.grid(6, 6), synth.ba(2000, 4, seed=3), synth.er(1500, 6.0, seed=5)]
    piv = [14, synth.max_degree_vertex(gs[1]), synth.max_degree_vertex(gs[2])]
    with pkg.USTBatch([(g.row_ptr, g.col_idx) for g in gs], piv, graph_id=5) as b:
        b.track_edges(True)
        b.sample_aggregate(40, 6)
        got = b.edge_counts()
        off = 0
        for i, g in enumerate(gs):
            assert np.array_equal(got[off:off + g.nnz], orc.edge_counts(g, piv[i], 0, 40, 6, graph=5 + i)), i
            off += g.nnz


def test_tuned_and_fixed_launch_shapes_give_equal_counts(pkg, orc):
    """The launch-shape tuner (ust_opts.autotune) changes only the speed of a
    launch: a batch tuned at creation (the default for batches) and one on the
    fixed shape table give identical counts, and a tuned single graph gives
    the oracle's counts."""
    gs, piv = small_batch()
    graphs = [(g.row_ptr, g.col_idx) for g in gs]
    with pkg.USTBatch(graphs, piv, autotune=1) as a, pkg.USTBatch(graphs, piv, autotune=-1) as b:
        a.sample_aggregate(50, 3)
        b.sample_aggregate(50, 3)
        assert np.array_equal(a.counts(), b.counts())
        shapes = {(a.graph_info(i)["sample_threads"], a.graph_info(i)["sample_ctas"]) for i in range(len(gs))}
        assert all(bt in (64, 128, 256, 512, 1024) and ctas > 0 for bt, ctas in shapes)
    g = synth.er(9000, 10.0, seed=7)
    u = synth.max_degree_vertex(g)
    with pkg.UST(g.row_ptr, g.col_idx, u, autotune=1) as h:
        h.sample_aggregate(200, 5)
        _, _, par = orc.bfs(g, u)
        R_ref, _ = orc.sample_aggregate(g, u, par, 0, 200, 5, threads=THREADS)
        assert np.array_equal(h.counts(), R_ref)
