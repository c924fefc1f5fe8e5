"""The samplers' relabelling (csrc/ust_relabel.cu), modelled step by step in
Python on the CPU.

The device builds a Cuthill-McKee order level by level of the BFS from the
pivot: vertex w on level d+1 is discovered by its level-d neighbour of least
new id, m(w), and level d+1 takes the next ids in order of (m(w), degree,
input id), sorted by a stable LSD radix sort whose scatter ranks equal digits
inside a tile by warp match masks and per-warp counts. The pendant vertices
(degree 1, not the pivot, neighbour of degree 2 or more) then move behind the
others, keeping their order.

Checked here: the model of the radix scatter sorts stably (against numpy's
stable argsort), the level-by-level order equals the textbook queue form of
Cuthill-McKee (a vertex's unvisited neighbours appended by increasing degree
when it leaves the queue), and the result is a permutation with the pivot
first and the pendant vertices last.
"""
import numpy as np
import pytest

import oracle
import synth

T, C, B = 256, 8, 256  # threads, chunks per thread, bins (8-bit digits)
TILE = T * C


def _scatter_pass(keys, vals, shift):
    """One pass of the device's histogram, exclusive scan and stable scatter."""
    count = len(keys)
    tiles = (count + TILE - 1) // TILE
    digit = (keys >> shift) & (B - 1)
    hist = np.zeros((B, tiles), dtype=np.int64)
    for b in range(tiles):
        hist[:, b] = np.bincount(digit[b * TILE:(b + 1) * TILE], minlength=B)
    offs = np.concatenate([[0], np.cumsum(hist.reshape(-1))])[:-1].reshape(B, tiles)
    okeys = np.full(count, -1, dtype=np.int64)
    ovals = np.full(count, -1, dtype=np.int64)
    for b in range(tiles):
        base = offs[:, b].copy()
        for c in range(C):
            lo = b * TILE + c * T
            if lo >= count:
                break
            d = digit[lo:min(lo + T, count)]
            # rank among equal digits before it: earlier warps, then earlier lanes
            ranks = np.zeros(len(d), dtype=np.int64)
            seen = {}
            for t, dig in enumerate(d):
                ranks[t] = seen.get(dig, 0)
                seen[dig] = ranks[t] + 1
            for t, dig in enumerate(d):
                r = base[dig] + ranks[t]
                assert 0 <= r < count and okeys[r] == -1
                okeys[r] = keys[lo + t]
                ovals[r] = vals[lo + t]
            for dig, cnt in seen.items():
                base[dig] += cnt
    return okeys, ovals


def _radix_sort(keys, vals, bits):
    for shift in range(0, bits, 8):
        keys, vals = _scatter_pass(keys, vals, shift)
    return keys, vals


@pytest.mark.parametrize("count,hi", [(1, 3), (300, 4), (2048, 1000), (2049, 7), (5000, 1 << 20)])
def test_radix_scatter_is_stable(count, hi):
    rng = np.random.default_rng(count)
    keys = rng.integers(0, hi, count).astype(np.int64)
    vals = np.arange(count, dtype=np.int64)
    bits = max(1, int(hi - 1).bit_length())
    k, v = _radix_sort(keys.copy(), vals.copy(), bits)
    assert np.array_equal(v, np.argsort(keys, kind="stable"))
    assert np.array_equal(k, np.sort(keys, kind="stable"))


def _device_order(g, u):
    """The device's construction: levels, then (m(w), degree, id) per level by
    the radix-sort model, then the stable pendant partition."""
    n = g.n
    deg = np.diff(g.row_ptr)
    _, dist, _ = oracle.bfs(g, u)
    ecc = int(dist.max())
    lv_keys, lv = _radix_sort(dist.astype(np.int64), np.arange(n, dtype=np.int64), max(1, ecc.bit_length()))
    first = np.searchsorted(lv_keys, np.arange(ecc + 2))
    newid = np.full(n, -1, dtype=np.int64)
    orig = np.full(n, -1, dtype=np.int64)
    orig[0], newid[u] = u, 0
    for d in range(ecc):
        seg = lv[first[d + 1]:first[d + 2]]
        keys = np.empty(len(seg), dtype=np.int64)
        for i, w in enumerate(seg):
            nb = g.col_idx[g.row_ptr[w]:g.row_ptr[w + 1]]
            m = min(int(newid[x]) for x in nb if dist[x] == d)
            keys[i] = ((m - first[d]) << 32) | int(deg[w])
        size = first[d + 1] - first[d]
        _, vals = _radix_sort(keys, seg.copy(), 32 + max(1, int(size - 1).bit_length()))
        orig[first[d + 1]:first[d + 2]] = vals
        newid[vals] = np.arange(first[d + 1], first[d + 2])
    pend = np.array([v != u and deg[v] == 1 and deg[g.col_idx[g.row_ptr[v]]] >= 2 for v in orig], dtype=np.int64)
    _, orig = _radix_sort(pend, orig.copy(), 1)
    return orig, int(pend.sum())


def _queue_cm(g, u):
    """Textbook Cuthill-McKee: breadth-first from u, each vertex's unvisited
    neighbours appended by increasing degree (ties: smaller id)."""
    deg = np.diff(g.row_ptr)
    seen = np.zeros(g.n, dtype=bool)
    order = [u]
    seen[u] = True
    head = 0
    while head < len(order):
        x = order[head]
        head += 1
        nb = [int(w) for w in g.col_idx[g.row_ptr[x]:g.row_ptr[x + 1]] if not seen[w]]
        nb.sort(key=lambda w: (deg[w], w))
        for w in nb:
            seen[w] = True
        order.extend(nb)
    return np.array(order, dtype=np.int64)


@pytest.mark.parametrize("maker,u", [
    (lambda: synth.grid(7, 9), 31),
    (lambda: synth.rmat(10, 8, seed=4), None),
    (lambda: synth.ba(600, 2, seed=1), None),
    (lambda: synth.star(12), 0),
    (lambda: synth.path(40), 17),
])
def test_level_order_is_cuthill_mckee_with_pendant_vertices_last(maker, u):
    g = maker()
    if u is None:
        u = synth.max_degree_vertex(g)
    orig, npend = _device_order(g, u)
    assert sorted(orig.tolist()) == list(range(g.n))  # a permutation
    assert orig[0] == u
    deg = np.diff(g.row_ptr)
    is_pend = np.array([v != u and deg[v] == 1 and deg[g.col_idx[g.row_ptr[v]]] >= 2 for v in range(g.n)])
    assert npend == int(is_pend.sum())
    assert not is_pend[orig[:g.n - npend]].any() and is_pend[orig[g.n - npend:]].all()
    cm = _queue_cm(g, u)
    # both parts keep the Cuthill-McKee order
    assert np.array_equal(orig[:g.n - npend], cm[~is_pend[cm]])
    assert np.array_equal(orig[g.n - npend:], cm[is_pend[cm]])
