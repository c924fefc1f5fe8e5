"""Seeded synthetic graphs in int32 CSR form.

Every generator returns a :class:`Graph` that is simple (no self-loops, no
duplicate arcs), undirected (both arcs of every edge are stored), has sorted
adjacency rows and is connected (the largest connected component is kept and
relabelled 0..n-1 in increasing order of the original ids).

Randomness comes from numpy's Philox bit generator keyed by the seed, so a
graph is a pure function of its parameters.

The workloads stand in for the paper's synthetic studies: random hyperbolic
graphs with average degree 20 and power-law exponent 3 (Section 5.4 and
Appendix E, Figure "hyperbolic scaling") and R-MAT graphs with Graph500
parameters (Appendix E, R-MAT scaling). The paper's real-world KONECT graphs
are not available; these seeded graphs replace them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.sparse import coo_matrix, csr_matrix
from scipy.sparse.csgraph import connected_components


@dataclasses.dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col_idx: np.ndarray  # int32[2m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.col_idx.shape[0] // 2)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def edges(self) -> np.ndarray:
        """Undirected edge list (a < b), shape [m, 2]."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        dst = self.col_idx.astype(np.int64)
        keep = src < dst
        return np.stack([src[keep], dst[keep]], axis=1)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed) & ((1 << 64) - 1)))


def from_edges(n: int, src, dst, name: str = "", lcc: bool = True) -> Graph:
    """Symmetrise, drop self-loops, deduplicate, keep the largest component."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    s2 = np.concatenate([src, dst])
    d2 = np.concatenate([dst, src])
    a = coo_matrix((np.ones(s2.shape[0], dtype=np.int8), (s2, d2)), shape=(n, n)).tocsr()
    a.sum_duplicates()
    a.data[:] = 1
    if lcc:
        ncomp, lab = connected_components(a, directed=False)
        if ncomp > 1:
            big = np.argmax(np.bincount(lab))
            ids = np.nonzero(lab == big)[0]
            a = a[ids][:, ids]
    a = csr_matrix(a)
    a.sort_indices()
    return Graph(n=a.shape[0], row_ptr=a.indptr.astype(np.int32),
                 col_idx=a.indices.astype(np.int32), name=name)


def max_degree_vertex(g: Graph) -> int:
    """Pivot rule of the workloads: maximum degree, smallest id on ties."""
    return int(np.argmax(g.degrees()))


def grid(w: int, h: int) -> Graph:
    """w x h 4-neighbour grid; vertex (row, col) has id row*w + col."""
    idx = np.arange(w * h, dtype=np.int64).reshape(h, w)
    src = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    dst = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return from_edges(w * h, src, dst, name=f"grid{w}x{h}")


def cycle(n: int) -> Graph:
    v = np.arange(n)
    return from_edges(n, v, (v + 1) % n, name=f"C{n}")


def path(n: int) -> Graph:
    v = np.arange(n - 1)
    return from_edges(n, v, v + 1, name=f"P{n}")


def star(n: int) -> Graph:
    """Vertex 0 is the centre, 1..n-1 are leaves."""
    v = np.arange(1, n)
    return from_edges(n, np.zeros_like(v), v, name=f"S{n}")


def complete(n: int) -> Graph:
    a, b = np.triu_indices(n, 1)
    return from_edges(n, a, b, name=f"K{n}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, chunk: int = 1 << 22) -> Graph:
    """R-MAT with Graph500 quadrant probabilities (a, b, c, d = 1-a-b-c).

    edge_factor * 2^scale edge draws; each level picks a quadrant: a -> (0,0),
    b -> (0,1), c -> (1,0), d -> (1,1) as (source bit, target bit). No noise
    and no vertex permutation. Then symmetrise, deduplicate, drop self-loops,
    keep the largest connected component.
    """
    n = 1 << scale
    total = edge_factor * n
    rng = _rng(seed)
    srcs, dsts = [], []
    done = 0
    while done < total:
        k = min(chunk, total - done)
        s = np.zeros(k, dtype=np.int64)
        d = np.zeros(k, dtype=np.int64)
        for _ in range(scale):
            r = rng.random(k)
            sb = r >= (a + b)
            db = ((r >= a) & (r < a + b)) | (r >= a + b + c)
            s = (s << 1) | sb
            d = (d << 1) | db
        srcs.append(s)
        dsts.append(d)
        done += k
    return from_edges(n, np.concatenate(srcs), np.concatenate(dsts),
                      name=f"rmat{scale}_ef{edge_factor}")


def er(n: int, avg_deg: float, seed: int) -> Graph:
    """Erdos-Renyi G(n, p) with p = avg_deg / (n - 1), largest component."""
    rng = _rng(seed)
    pairs = n * (n - 1) // 2
    p = avg_deg / (n - 1)
    k = int(rng.binomial(pairs, p))
    s = rng.integers(0, n, size=int(k * 1.02) + 16)
    d = rng.integers(0, n, size=s.shape[0])
    keep = s != d
    s, d = s[keep], d[keep]
    lo, hi = np.minimum(s, d), np.maximum(s, d)
    key = np.unique(lo * n + hi)
    key = key[rng.permutation(key.shape[0])[:k]]
    return from_edges(n, key // n, key % n, name=f"er{n}")


def ba(n: int, k: int, seed: int) -> Graph:
    """Barabasi-Albert preferential attachment, k edges per new vertex.

    The seed graph is a clique on vertices 0..k. Vertex i > k adds k edge
    slots; each slot's target is the endpoint stored at a uniformly drawn
    position among all endpoints of earlier slots, which is a
    degree-proportional choice. A drawn position holds either a source (the
    vertex that owns the slot, known) or a target; a target position is
    resolved by following that slot's own draw, so the whole endpoint list is
    resolved with vectorised pointer chasing instead of a loop over vertices.
    Duplicate edges are merged.
    """
    rng = _rng(seed)
    k = max(1, int(k))
    seed_a, seed_b = np.triu_indices(k + 1, 1)
    m0 = int(seed_a.shape[0])
    new = np.arange(k + 1, n, dtype=np.int64)
    slots = int(new.shape[0]) * k
    owner = np.repeat(new, k)
    src_all = np.concatenate([seed_a, owner])
    limit = 2 * (m0 + (np.arange(slots) // k) * k)  # endpoints before this vertex
    draw = (rng.random(slots) * limit).astype(np.int64)
    target = np.full(slots, -1, dtype=np.int64)
    ptr = draw.copy()
    todo = np.arange(slots)
    while todo.shape[0]:
        p = ptr[todo]
        e = p // 2
        even = (p % 2) == 0
        val = np.full(todo.shape[0], -1, dtype=np.int64)
        val[even] = src_all[e[even]]
        seed_t = (~even) & (e < m0)
        val[seed_t] = seed_b[e[seed_t]]
        later = (~even) & (e >= m0)
        ls = e[later] - m0
        val[later] = target[ls]
        target[todo] = val
        pending = val < 0
        nxt = todo[pending]
        ptr[nxt] = draw[(e - m0)[pending]]
        todo = nxt
    s = np.concatenate([seed_a, owner])
    d = np.concatenate([seed_b, target])
    return from_edges(n, s, d, name=f"ba{n}_k{k}")


def _hyperbolic_expected_degree(n: int, alpha: float, R: float, grid_pts: int = 1500) -> float:
    """Expected average degree of the threshold random hyperbolic graph."""
    r = (np.arange(grid_pts) + 0.5) / grid_pts * R
    dens = alpha * np.sinh(alpha * r) / (np.cosh(alpha * R) - 1.0) * (R / grid_pts)
    ri = r[:, None]
    rj = r[None, :]
    num = np.cosh(ri) * np.cosh(rj) - np.cosh(R)
    den = np.sinh(ri) * np.sinh(rj)
    cosang = np.clip(num / den, -1.0, 1.0)
    theta = np.arccos(cosang)  # connect iff angular gap <= theta
    prob = theta / math.pi
    return float((n - 1) * dens @ prob @ dens)


def hyperbolic(n: int, avg_deg: float = 20.0, gamma: float = 3.0, seed: int = 1,
               bands: int = 32) -> Graph:
    """Threshold (temperature 0) random hyperbolic graph, largest component.

    alpha = (gamma - 1) / 2. The disk radius R is fitted by bisection so that
    the expected average degree equals avg_deg. Neighbour search sorts points
    by angle inside radial bands and checks the exact distance only for
    points inside each band's angular window.
    """
    alpha = (gamma - 1.0) / 2.0
    lo, hi = 1.0, 4.0 * math.log(n) + 20.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if _hyperbolic_expected_degree(n, alpha, mid) > avg_deg:
            lo = mid
        else:
            hi = mid
    R = 0.5 * (lo + hi)
    rng = _rng(seed)
    theta = rng.random(n) * 2.0 * math.pi
    u = rng.random(n)
    # inverse CDF of density alpha sinh(alpha r) / (cosh(alpha R) - 1)
    r = np.arccosh(1.0 + u * (np.cosh(alpha * R) - 1.0)) / alpha
    edges_s, edges_d = [], []
    # band boundaries: geometric in the outer region where most points live
    bnd = np.linspace(0.0, R, bands + 1)
    band_of = np.minimum((r / R * bands).astype(np.int64), bands - 1)
    coshr, sinhr = np.cosh(r), np.sinh(r)
    coshR = math.cosh(R)
    for bi in range(bands):
        members = np.nonzero(band_of == bi)[0]
        if members.shape[0] == 0:
            continue
        order = np.argsort(theta[members])
        mem = members[order]
        th = theta[mem]
        th_ext = np.concatenate([th - 2 * math.pi, th, th + 2 * math.pi])
        mem_ext = np.concatenate([mem, mem, mem])
        rb = max(bnd[bi], 1e-9)
        # queries: all points in bands <= bi (each unordered pair visited once
        # from the lower band, ties inside a band resolved by id below)
        q = np.nonzero(band_of <= bi)[0]
        num = coshr[q] * math.cosh(rb) - coshR
        den = sinhr[q] * math.sinh(rb)
        with np.errstate(divide="ignore", invalid="ignore"):
            c = np.where(den > 0, num / den, -1.0)
        dmax = np.arccos(np.clip(c, -1.0, 1.0))
        left = np.searchsorted(th_ext, theta[q] - dmax, side="left")
        right = np.searchsorted(th_ext, theta[q] + dmax, side="right")
        right = np.minimum(right, left + mem.shape[0])
        cnt = right - left
        tot = int(cnt.sum())
        if tot == 0:
            continue
        step = 1 << 24
        qi_all = np.repeat(np.arange(q.shape[0]), cnt)
        off = np.arange(tot) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        for s0 in range(0, tot, step):
            qi = qi_all[s0:s0 + step]
            cand = mem_ext[left[qi] + off[s0:s0 + step]]
            a = q[qi]
            ok = (cand != a) & ((band_of[a] < bi) | (a < cand))
            a, cand = a[ok], cand[ok]
            dth = np.abs(theta[a] - theta[cand])
            dth = np.minimum(dth, 2 * math.pi - dth)
            cd = coshr[a] * coshr[cand] - sinhr[a] * sinhr[cand] * np.cos(dth)
            hit = cd <= coshR
            edges_s.append(a[hit])
            edges_d.append(cand[hit])
    s = np.concatenate(edges_s) if edges_s else np.zeros(0, np.int64)
    d = np.concatenate(edges_d) if edges_d else np.zeros(0, np.int64)
    return from_edges(n, s, d, name=f"hyperbolic{n}")


def workload(name: str):
    """Named workloads: returns (graph, pivot, n_trees or None, eps or None).

    grid48      48x48 grid, pivot (24, 24) = 1176, 1000 trees
    rmat16      R-MAT scale 16, edge factor 16, LCC, max-degree pivot, 4096 trees
    rmat17      R-MAT scale 17, edge factor 16, LCC, max-degree pivot, 1024 trees
                (the smallest R-MAT above 65,535 vertices: a profiling case
                of the large-graph sampler)
    rmat19      R-MAT scale 19, edge factor 16, LCC, max-degree pivot, 1024 trees
                (per-tree state far larger than L2, as for scale 22)
    hyperbolic20  threshold RHG n = 2^20, avg degree 20, gamma 3, eps 0.3
    rmat22      R-MAT scale 22, edge factor 16, LCC, max-degree pivot, eps 0.3
    """
    if name == "grid48":
        return grid(48, 48), 24 * 48 + 24, 1000, None
    if name == "rmat16":
        g = rmat(16, 16, seed=1)
        return g, max_degree_vertex(g), 4096, None
    if name == "rmat17":
        g = rmat(17, 16, seed=1)
        return g, max_degree_vertex(g), 1024, None
    if name == "rmat19":
        g = rmat(19, 16, seed=1)
        return g, max_degree_vertex(g), 1024, None
    if name == "rmat22":
        g = rmat(22, 16, seed=1)
        return g, max_degree_vertex(g), None, 0.3
    if name == "hyperbolic20":
        g = hyperbolic(1 << 20, 20.0, 3.0, seed=1)
        return g, max_degree_vertex(g), None, 0.3
    raise KeyError(name)


def batch_specs(count: int = 256, seed: int = 0):
    """Parameters of the uneven batch: (kind, n, avg_deg, seed) per graph.

    Even index: Barabasi-Albert with k = avg/2; odd index: Erdos-Renyi with
    p = avg/(n-1); n ~ U[1000, 64000], avg ~ U[8, 32]; generator seed = index.
    """
    rng = _rng(seed)
    ns = rng.integers(1000, 64001, size=count)
    avgs = rng.uniform(8.0, 32.0, size=count)
    return [("ba" if i % 2 == 0 else "er", int(ns[i]), float(avgs[i]), i) for i in range(count)]


def batch_graph(spec) -> Graph:
    kind, n, avg, s = spec
    if kind == "ba":
        return ba(n, max(1, int(round(avg / 2))), seed=s)
    return er(n, avg, seed=s)
