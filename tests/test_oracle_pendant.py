"""Pins, on the oracle, the two facts that let the large-graph sampler leave
pendant vertices (degree 1, not the pivot, next to a vertex of degree 2 or
more) out of its trees.

1. Cycle popping on the stacks of the whole graph gives, on the other (core)
   vertices, the tree that Wilson's walks give when every stack entry naming a
   pendant vertex is skipped: such an entry and the pendant vertex, whose every
   entry names the same neighbour, form a 2-cycle, and the popping order does
   not matter (Wilson's cycle-popping theorem, Appendix A.2). Checked against
   the oracle's own Wilson on the whole graph, tree by tree, with the draw
   count: the whole graph's draws are the core's, plus one pop of the pendant
   vertex per skipped entry, plus every pendant vertex's first draw.
2. Algorithm 2 gives a pendant vertex v with neighbour w the count
   1 + count(w) in every tree (P(v) is P(w) with the edge (w, v) in front,
   which every tree uses downwards, and v lies in a subtree exactly when w
   does), so over T trees R[v] = T + R[w].
"""
import numpy as np

import oracle
import synth


def _graph():
    """A 6x6 grid with seven pendant vertices: three at the pivot 14, three at
    other grid vertices, and the end of a two-vertex path hanging from vertex
    35 (the path's first vertex has degree 2 and stays in the core)."""
    g = synth.grid(6, 6)
    deg = np.diff(g.row_ptr)
    src = [np.repeat(np.arange(g.n), deg), np.arange(36, 43), [43]]
    dst = [g.col_idx, [14, 14, 14, 0, 7, 21, 35], [42]]
    h = synth.from_edges(44, np.concatenate(src), np.concatenate(dst), lcc=False)
    return h, 14


def _pendant(g, u):
    deg = np.diff(g.row_ptr)
    out = {}
    for v in range(g.n):
        if v != u and deg[v] == 1:
            w = int(g.col_idx[g.row_ptr[v]])
            if deg[w] >= 2:
                out[v] = w
    return out


def _core_wilson(g, u, tree, seed, pend):
    """Wilson's walks on the core, skipping the stack entries that name a
    pendant vertex. Returns (parent of every core vertex, entries the core
    consumed, entries skipped)."""
    n = g.n
    depth = np.zeros(n, dtype=np.int64)
    nxt = np.full(n, -2, dtype=np.int64)
    in_tree = np.zeros(n, dtype=bool)
    in_tree[u] = True
    nxt[u] = -1
    consumed = skipped = 0

    def step(x):
        nonlocal consumed, skipped
        while True:
            y = oracle.successor(g, x, int(depth[x]), tree, 0, seed)
            depth[x] += 1
            consumed += 1
            if y in pend:
                skipped += 1
                continue
            return y

    for s in range(n):
        if s in pend or in_tree[s]:
            continue
        x = s
        while not in_tree[x]:
            nxt[x] = step(x)
            x = nxt[x]
        x = s
        while not in_tree[x]:
            in_tree[x] = True
            x = nxt[x]
    return nxt, consumed, skipped


def test_core_tree_with_pendant_entries_skipped_equals_wilson_on_the_whole_graph():
    g, u = _graph()
    pend = _pendant(g, u)
    assert len(pend) == 7  # 36..41 and 43 (42 has degree 2)
    core = np.array([v for v in range(g.n) if v not in pend])
    for tree in range(12):
        nxt_full, _, steps = oracle.wilson(g, u, tree, 5)
        nxt_core, consumed, skipped = _core_wilson(g, u, tree, 5, pend)
        assert np.array_equal(nxt_core[core], nxt_full[core]), tree
        for v, w in pend.items():
            assert nxt_full[v] == w
        assert steps == consumed + skipped + len(pend), tree


def test_pendant_counts_follow_from_the_neighbour():
    g, u = _graph()
    pend = _pendant(g, u)
    _, _, par = oracle.bfs(g, u)
    T = 300
    R, _ = oracle.sample_aggregate(g, u, par, 0, T, 11)
    for v, w in pend.items():
        assert R[v] == T + R[w], (v, w)
    # per tree as well
    for tree in range(5):
        nxt, _, _ = oracle.wilson(g, u, tree, 11)
        c = oracle.aggregate(nxt, par, u)
        for v, w in pend.items():
            assert c[v] == 1 + c[w]
