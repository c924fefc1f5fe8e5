"""The labelling rules behind the device's walk rows for the biconnected-
component variant, modelled step by step in plain Python and checked against
the oracle's Hopcroft-Tarjan blocks on random sparse graphs and every kind of
pivot. The model follows the kernels' order: subtree sizes and preorder
numbers level by level over B_u, lo/hi reach over non-tree edges, then the two
union rules of Tarjan and Vishkin over tree edges. (The kernels themselves are
checked bit-exact against the oracle in the GPU tests.)"""
import numpy as np
import pytest

import synth


def _model_parent_block_rows(orc, g, u):
    ecc, dist, par = orc.bfs(g, u)
    n, rp, ci = g.n, g.row_ptr, g.col_idx
    levels = [np.nonzero(dist == d)[0] for d in range(ecc + 1)]
    nd = np.ones(n, dtype=np.int64)
    for d in range(ecc, 0, -1):
        np.add.at(nd, par[levels[d]], nd[levels[d]])
    pre = np.zeros(n, dtype=np.int64)
    cur = np.zeros(n, dtype=np.int64)
    cur[u] = 1
    for d in range(1, ecc + 1):
        for v in levels[d]:  # any child order gives a preorder
            pre[v] = cur[par[v]]
            cur[par[v]] += nd[v]
            cur[v] = pre[v] + 1

    def tree(v, w):
        return par[w] == v or par[v] == w

    lo, hi = pre.copy(), pre.copy()
    for v in range(n):
        for w in ci[rp[v]:rp[v + 1]]:
            if not tree(v, w):
                lo[v], hi[v] = min(lo[v], pre[w]), max(hi[v], pre[w])
    for d in range(ecc, 0, -1):
        for v in levels[d]:
            lo[par[v]], hi[par[v]] = min(lo[par[v]], lo[v]), max(hi[par[v]], hi[v])
    uf = list(range(n))

    def find(x):
        while uf[x] != x:
            x = uf[x]
        return x

    def union(a, b):
        a, b = find(a), find(b)
        if a != b:
            uf[max(a, b)] = min(a, b)

    for v in range(n):  # (1) non-tree edges between unrelated subtrees
        for w in ci[rp[v]:rp[v + 1]]:
            if not tree(v, w) and pre[v] < pre[w] and pre[w] >= pre[v] + nd[v]:
                union(v, int(w))
    for v in range(n):  # (2) a subtree that reaches outside its parent's subtree
        p = par[v]
        if v != u and p != u and (lo[v] < pre[p] or hi[v] >= pre[p] + nd[p]):
            union(v, int(p))
    lab = [find(v) for v in range(n)]

    def block(v, w):
        if par[w] == v:
            return lab[w]
        if par[v] == w:
            return lab[v]
        return lab[v] if pre[v] > pre[w] else lab[w]

    row_ptr, col_idx = [0], []
    for v in range(n):
        if v != u:
            col_idx += [int(w) for w in ci[rp[v]:rp[v + 1]] if block(v, int(w)) == lab[v]]
        row_ptr.append(len(col_idx))
    return np.array(row_ptr), np.array(col_idx, dtype=np.int64)


def _cases():
    rng = np.random.default_rng(7)
    out = []
    for s in range(12):
        out.append(("er", synth.er(int(rng.integers(20, 300)), float(rng.uniform(1.6, 3.5)), seed=s)))
        out.append(("ba", synth.ba(int(rng.integers(20, 200)), int(rng.integers(1, 3)), seed=s)))
    out += [("rmat", synth.rmat(9, 4, seed=3)), ("grid", synth.grid(6, 4)), ("path", synth.path(8)),
            ("star", synth.star(7)), ("cycle", synth.cycle(7))]
    return out


@pytest.mark.parametrize("k", range(len(_cases())))
def test_tarjan_vishkin_rows_equal_oracle_rows(orc, k):
    _, g = _cases()[k]
    for u in sorted({0, g.n // 2, g.n - 1, synth.max_degree_vertex(g)}):
        rp, ci = _model_parent_block_rows(orc, g, u)
        w = orc.parent_block_graph(g, u)
        assert np.array_equal(rp, w.row_ptr) and np.array_equal(ci, w.col_idx), u
