"""Parity at full size on the large workloads, on outputs the oracle can
compute one by one.

- random hyperbolic graph, n = 2^20, average degree 20, exponent 3,
  temperature 0, largest component, max-degree pivot, tau from eps = 0.3
- R-MAT scale 22, edge factor 16, largest component, max-degree pivot,
  tau from eps = 0.3

Checked: B_u bit-exact, tau(0.3), single trees spread over [0, tau)
bit-exact with their pop counts, the counts of the last 2 x 152 tree ids
below tau bit-exact (every CTA of the 152-SM launch samples at least two
trees), the column against FP64 CG within 1e-8, and the diagonal
combination within 1e-12 of the oracle's on the same counts and column.
"""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))
SEED = 0x5EED
RANGE_TREES = 2 * 152  # two trees for every CTA of a one-CTA-per-SM launch on 152 SMs


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


@pytest.mark.parametrize("name", ["hyperbolic20", "rmat22"])
def test_large_workload(pkg, orc, name):
    g, u, _, eps = synth.workload(name)
    with pkg.UST(g.row_ptr, g.col_idx, u) as h:
        par, dist = h.bfs()
        ecc, d_ref, p_ref = orc.bfs(g, u)
        assert np.array_equal(dist, d_ref) and np.array_equal(par, p_ref)
        tau = h.tau(eps)
        assert tau == orc.tau(ecc, g.m, eps, 1.0 / g.n, 0.3)
        for t in [0, 1, tau // 2, tau - 1]:
            nxt, pops = h.sample_trees(t, 1, SEED, with_pops=True)
            ref, ref_pops, _ = orc.wilson(g, u, t, SEED)
            assert np.array_equal(nxt[0], ref), (name, t)
            assert np.array_equal(pops[0], ref_pops), (name, t)
        t0 = tau - RANGE_TREES
        R = h.tree_range_counts(t0, tau, SEED)
        R_ref, _ = orc.sample_aggregate(g, u, p_ref, t0, tau, SEED, threads=THREADS)
        assert np.array_equal(R, R_ref)
        x = h.column()
        x_ref, _, _, ok = orc.cg(g, u, tol=1e-12, max_iter=20000)
        assert ok
        assert np.max(np.abs(x - x_ref)) <= 1e-8 * max(1.0, np.max(np.abs(x_ref)))
        h.sample_aggregate(64, SEED)
        d = h.diag()
        np.testing.assert_allclose(d, orc.combine(h.counts(), 64, x, u), rtol=1e-12, atol=0)
