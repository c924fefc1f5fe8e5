"""CPU oracle for the UST approximation of diag(L^+) (arXiv 2006.13679).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package. The product
path (the CUDA library and its binding) never loads it, and it shares no code
with that path.

Two layers:

* ``ust_oracle.c`` (built into ``liboracle.so`` with gcc, loaded through
  ctypes): Philox4x32-10, BFS, Wilson's loop-erased walks, explicit cycle
  popping, DFS timestamps, Algorithm 2, the Algorithm 1 sampling loop, FP64
  Jacobi-PCG, the diagonal combination and tau.
* numpy/scipy helpers in this file: the dense closed form
  L^+ = (L + J/n)^{-1} - J/n (Section 2.1), effective resistances from it
  (Eq. eff-res), brute-force spanning-tree enumeration and the matrix-tree
  count, which pin the C layer in the tests; the centralities that
  depend only on the diagonal (closeness, NRWB, Kirchhoff index); and, for
  the biconnected-component variant of Appendix D, the blocks (Hopcroft and
  Tarjan's search) and the parent-block rows the walks draw from.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ust_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fvisibility=hidden", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.orc_successor.argtypes = [_i32p, _i32p, ctypes.c_int32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
            L.orc_successor.restype = ctypes.c_int32
            L.orc_bfs.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _i32p, _i32p]
            L.orc_bfs.restype = ctypes.c_int32
            for fn in (L.orc_wilson, L.orc_cycle_pop):
                fn.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, ctypes.c_uint32,
                               ctypes.c_uint32, ctypes.c_uint64, _i32p, _i32p]
                fn.restype = ctypes.c_int64
            L.orc_dfs_times.argtypes = [ctypes.c_int32, _i32p, ctypes.c_int32, _i32p, _i32p]
            L.orc_aggregate.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _i32p, _i32p, _i64p]
            L.orc_sample_aggregate.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _i32p,
                                               ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32,
                                               ctypes.c_uint64, _i64p, ctypes.c_int32]
            L.orc_sample_aggregate.restype = ctypes.c_int64
            L.orc_max_threads.restype = ctypes.c_int32
            L.orc_cg.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, ctypes.c_double,
                                 ctypes.c_int32, _f64p, _i32p, _f64p]
            L.orc_cg.restype = ctypes.c_int32
            L.orc_combine.argtypes = [ctypes.c_int32, _i64p, ctypes.c_int64, _f64p, ctypes.c_int32, _f64p]
            L.orc_tau.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double]
            L.orc_tau.restype = ctypes.c_int64
            _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    return rp, ci


# ---------------------------------------------------------------- C layer

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def successor(g, v: int, depth: int, tree: int, graph: int, seed: int) -> int:
    rp, ci = _csr(g)
    return int(lib().orc_successor(_p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), v, depth,
                                   tree, graph, seed))


def bfs(g, u: int):
    """Returns (ecc, dist[n], parent[n]); ecc = -1 if g is disconnected."""
    rp, ci = _csr(g)
    dist = np.zeros(g.n, dtype=np.int32)
    par = np.zeros(g.n, dtype=np.int32)
    ecc = lib().orc_bfs(g.n, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), u,
                        _p(dist, ctypes.c_int32), _p(par, ctypes.c_int32))
    return int(ecc), dist, par


def wilson(g, u: int, tree: int, seed: int, graph: int = 0):
    """Wilson LERW tree: returns (next[n] with next[u] = -1, pops[n], steps)."""
    rp, ci = _csr(g)
    nxt = np.zeros(g.n, dtype=np.int32)
    pops = np.zeros(g.n, dtype=np.int32)
    steps = lib().orc_wilson(g.n, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), u, tree, graph,
                             seed, _p(nxt, ctypes.c_int32), _p(pops, ctypes.c_int32))
    return nxt, pops, int(steps)


def cycle_pop(g, u: int, tree: int, seed: int, graph: int = 0):
    rp, ci = _csr(g)
    nxt = np.zeros(g.n, dtype=np.int32)
    pops = np.zeros(g.n, dtype=np.int32)
    draws = lib().orc_cycle_pop(g.n, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), u, tree, graph,
                                seed, _p(nxt, ctypes.c_int32), _p(pops, ctypes.c_int32))
    return nxt, pops, int(draws)


def dfs_times(nxt: np.ndarray, u: int):
    n = nxt.shape[0]
    nx = np.ascontiguousarray(nxt, dtype=np.int32)
    alpha = np.zeros(n, dtype=np.int32)
    omega = np.zeros(n, dtype=np.int32)
    lib().orc_dfs_times(n, _p(nx, ctypes.c_int32), u, _p(alpha, ctypes.c_int32), _p(omega, ctypes.c_int32))
    return alpha, omega


def aggregate(nxt: np.ndarray, bfs_parent: np.ndarray, u: int, R: np.ndarray | None = None) -> np.ndarray:
    """Algorithm 2 for one tree (next[] rooted at u); returns R (int64)."""
    n = nxt.shape[0]
    if R is None:
        R = np.zeros(n, dtype=np.int64)
    alpha, omega = dfs_times(nxt, u)
    nx = np.ascontiguousarray(nxt, dtype=np.int32)
    bp = np.ascontiguousarray(bfs_parent, dtype=np.int32)
    lib().orc_aggregate(n, _p(nx, ctypes.c_int32), _p(bp, ctypes.c_int32), u,
                        _p(alpha, ctypes.c_int32), _p(omega, ctypes.c_int32), _p(R, ctypes.c_int64))
    return R


def sample_aggregate(g, u: int, bfs_parent: np.ndarray, t0: int, t1: int, seed: int,
                     graph: int = 0, threads: int = 1):
    """Trees [t0, t1): returns (R int64[n], total walk steps)."""
    rp, ci = _csr(g)
    R = np.zeros(g.n, dtype=np.int64)
    bp = np.ascontiguousarray(bfs_parent, dtype=np.int32)
    steps = lib().orc_sample_aggregate(g.n, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), u,
                                       _p(bp, ctypes.c_int32), t0, t1, graph, seed,
                                       _p(R, ctypes.c_int64), threads)
    return R, int(steps)


def max_threads() -> int:
    return int(lib().orc_max_threads())


def cg(g, u: int, tol: float = 1e-13, max_iter: int = 100000):
    """FP64 Jacobi-PCG column x = L^+[:, u]; returns (x, iters, relres, ok)."""
    rp, ci = _csr(g)
    x = np.zeros(g.n, dtype=np.float64)
    it = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1, dtype=np.float64)
    rc = lib().orc_cg(g.n, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), u, tol, max_iter,
                      _p(x, ctypes.c_double), _p(it, ctypes.c_int32), _p(rr, ctypes.c_double))
    return x, int(it[0]), float(rr[0]), rc == 0


def combine(R: np.ndarray, tau: int, x: np.ndarray, u: int) -> np.ndarray:
    n = R.shape[0]
    Rc = np.ascontiguousarray(R, dtype=np.int64)
    xc = np.ascontiguousarray(x, dtype=np.float64)
    d = np.zeros(n, dtype=np.float64)
    lib().orc_combine(n, _p(Rc, ctypes.c_int64), tau, _p(xc, ctypes.c_double), u, _p(d, ctypes.c_double))
    return d


def select_pivot(g, sweeps: int = 10, start: int = -1):
    """Pivot of low eccentricity (Appendix D, choice of u): BFS from a first
    source (start, or the vertex of largest degree), then from the vertex
    farthest from the previous source, `sweeps` times; each vertex keeps the
    largest distance seen, a lower bound on its eccentricity. Returns the
    vertex of least bound and the bound. Ties: smallest vertex id."""
    deg = np.diff(np.asarray(g.row_ptr, dtype=np.int64))
    s = int(np.argmax(deg)) if start < 0 else int(start)
    lb = np.zeros(g.n, dtype=np.int64)
    for _ in range(sweeps):
        _, dist, _ = bfs(g, s)
        if (dist < 0).any():
            raise ValueError("graph is not connected")
        lb = np.maximum(lb, dist)
        s = int(np.argmax(dist))
    piv = int(np.argmin(lb))
    return piv, int(lb[piv])


def tree_arcs(g, nxt, u: int) -> np.ndarray:
    """CSR positions of a rooted tree's arcs v -> next[v], v != u (rows are
    sorted, so the position is found by binary search in row v)."""
    rp, ci = _csr(g)
    out = np.empty(g.n - 1, dtype=np.int64)
    k = 0
    for v in range(g.n):
        if v == u:
            continue
        row = ci[rp[v]:rp[v + 1]]
        j = int(np.searchsorted(row, nxt[v]))
        assert j < row.shape[0] and row[j] == nxt[v], "tree arc not in the graph"
        out[k] = rp[v] + j
        k += 1
    return out


def edge_counts(g, u: int, t0: int, t1: int, seed: int, graph: int = 0, walk=None) -> np.ndarray:
    """Per CSR arc v -> w of g, the number of trees t0 .. t1-1 (Wilson's
    loop-erased walks, Appendix A.2) in which w is v's parent: sampling USTs
    and counting the trees each edge appears in (appendix on Kirchhoff edge
    centrality). walk: the rows the walks draw from (parent_block_graph for
    the biconnected-component variant), default g."""
    counts = np.zeros(g.nnz, dtype=np.int64)
    for t in range(t0, t1):
        nxt, _, _ = wilson(g if walk is None else walk, u, t, seed, graph)
        np.add.at(counts, tree_arcs(g, nxt, u), 1)
    return counts


# ------------------------------------------- biconnected-component variant

class CSR:
    """Rows of a (possibly directed) sampling graph: n, row_ptr, col_idx."""

    def __init__(self, n: int, row_ptr: np.ndarray, col_idx: np.ndarray):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])


def blocks(g) -> np.ndarray:
    """Block (biconnected component) id of every CSR arc of g; both arcs of an
    edge get the same id. Hopcroft and Tarjan's depth-first search with an
    edge stack: every tree or back edge is pushed once; when the search
    leaves a tree edge (p, v) with low(v) >= disc(p), p separates v's subtree
    and the edges above (p, v) on the stack, (p, v) included, form one
    block. Appendix D samples the UST block by block (Hayashi et al.)."""
    rp, ci = _csr(g)
    n = g.n
    disc = np.full(n, -1, dtype=np.int64)
    low = np.zeros(n, dtype=np.int64)
    arc_block = np.full(ci.shape[0], -1, dtype=np.int64)
    clock, nb = 0, 0
    estack = []
    for s in range(n):
        if disc[s] >= 0:
            continue
        disc[s] = low[s] = clock
        clock += 1
        frames = [[s, -1, int(rp[s]), -1]]  # vertex, parent, next arc, tree arc into the vertex
        while frames:
            fr = frames[-1]
            v, p, it, tarc = fr
            if it < rp[v + 1]:
                fr[2] = it + 1
                w = int(ci[it])
                if disc[w] < 0:
                    estack.append(it)
                    disc[w] = low[w] = clock
                    clock += 1
                    frames.append([w, v, int(rp[w]), it])
                elif w != p and disc[w] < disc[v]:  # back edge to an ancestor
                    estack.append(it)
                    low[v] = min(low[v], disc[w])
            else:
                frames.pop()
                if p >= 0:
                    low[p] = min(low[p], low[v])
                    if low[v] >= disc[p]:
                        while True:
                            a = estack.pop()
                            arc_block[a] = nb
                            if a == tarc:
                                break
                        nb += 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp.astype(np.int64)))
    for a in np.nonzero(arc_block < 0)[0]:  # the reverse arcs take their edge's block
        v, w = int(src[a]), int(ci[a])
        row = ci[rp[w]:rp[w + 1]]
        arc_block[a] = arc_block[rp[w] + int(np.searchsorted(row, v))]
    return arc_block


def parent_block_graph(g, u: int, bfs_parent=None) -> CSR:
    """Sampling rows of the biconnected-component variant (Appendix D): every
    v != u keeps, in CSR order, its neighbours inside its parent block, the
    block of the edge (v, bfs_parent(v)); u's row is empty (the root never
    draws). Every cycle lies in one block, so Wilson on these rows samples
    each block's tree on its own, rooted at the block's vertex nearest u, and
    the union is a uniform spanning tree of g directed toward u."""
    rp, ci = _csr(g)
    if bfs_parent is None:
        _, _, bfs_parent = bfs(g, u)
    ab = blocks(g)
    deg = np.diff(rp.astype(np.int64))
    pb = np.full(g.n, -2, dtype=np.int64)
    for v in range(g.n):
        if v == u:
            continue
        row = ci[rp[v]:rp[v + 1]]
        pb[v] = ab[rp[v] + int(np.searchsorted(row, bfs_parent[v]))]
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    keep = ab == pb[src]
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(src[keep], minlength=g.n))])
    return CSR(g.n, row_ptr, ci[keep])


def centralities(diag) -> dict:
    """Centralities from a diagonal of L^+, written out from the paper:
    electrical farness f(v) = n L+[v,v] + tr(L+) (Section 3.1, Eq.
    elec-farness), electrical closeness (n - 1) / f(v) (Section 2,
    electrical closeness), normalized random-walk betweenness
    1/n + tr(L+) / ((n - 1) f(v)) (the NRWB lemma of Section 3.3, derived in
    the appendix) and the Kirchhoff index n tr(L+) (appendix on the Kirchhoff
    index). The NRWB form is the lemma's: the definition as printed sums
    per-target ratios, the derivation takes the ratio of the summed
    numerators and denominators, and the method computes the latter."""
    d = np.asarray(diag, dtype=np.float64)
    n = d.shape[0]
    tr = float(d.sum())
    f = n * d + tr
    return {"farness": f, "closeness": (n - 1) / f, "nrwb": 1.0 / n + tr / ((n - 1) * f), "kirchhoff": n * tr}


def tau(ecc: int, m: int, eps: float, delta: float, kappa: float = 0.3) -> int:
    return int(lib().orc_tau(ecc, m, eps, delta, kappa))


def diag(g, u: int, n_trees: int, seed: int, threads: int = 1):
    """Whole Algorithm 1 with a fixed tree count: (diag, R, x, ecc)."""
    ecc, _, par = bfs(g, u)
    R, _ = sample_aggregate(g, u, par, 0, n_trees, seed, threads=threads)
    x, _, _, _ = cg(g, u)
    return combine(R, n_trees, x, u), R, x, ecc


# ------------------------------------------------------- dense and brute force

def laplacian(g) -> np.ndarray:
    n = g.n
    L = np.zeros((n, n), dtype=np.float64)
    src = np.repeat(np.arange(n), g.degrees())
    L[src, g.col_idx.astype(np.int64)] = -1.0
    L[np.arange(n), np.arange(n)] = g.degrees().astype(np.float64)
    return L


def dense_pinv(g) -> np.ndarray:
    """L^+ = (L + J/n)^{-1} - J/n (Section 2.1)."""
    n = g.n
    L = laplacian(g)
    J = np.full((n, n), 1.0 / n)
    return np.linalg.inv(L + J) - J


def effective_resistance(Lp: np.ndarray, u: int) -> np.ndarray:
    """r(u, v) = L^+[u,u] - 2 L^+[u,v] + L^+[v,v] (Eq. eff-res), for all v."""
    d = np.diag(Lp)
    return d[u] - 2.0 * Lp[u, :] + d


def matrix_tree_count(g) -> float:
    """Number of spanning trees: determinant of L with one row/column removed."""
    L = laplacian(g)
    return float(np.linalg.det(L[1:, 1:]))


def spanning_trees(g):
    """All spanning trees of a tiny graph by brute force over (n-1)-edge subsets.

    Each tree is returned as a frozenset of edges (a, b), a < b.
    """
    edges = [tuple(map(int, e)) for e in g.edges()]
    n = g.n
    out = []
    for comb in itertools.combinations(edges, n - 1):
        parent = list(range(n))

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x

        ok = True
        for a, b in comb:
            ra, rb = find(a), find(b)
            if ra == rb:
                ok = False
                break
            parent[ra] = rb
        if ok:
            out.append(frozenset(comb))
    return out


def root_tree(tree_edges, n: int, u: int) -> np.ndarray:
    """Parent array of a spanning tree rooted at u (next[u] = -1)."""
    adj = [[] for _ in range(n)]
    for a, b in tree_edges:
        adj[a].append(b)
        adj[b].append(a)
    nxt = np.full(n, -2, dtype=np.int32)
    nxt[u] = -1
    stack = [u]
    while stack:
        v = stack.pop()
        for w in adj[v]:
            if nxt[w] == -2:
                nxt[w] = v
                stack.append(w)
    return nxt


def tree_edges_of(nxt: np.ndarray) -> frozenset:
    return frozenset((min(int(v), int(p)), max(int(v), int(p))) for v, p in enumerate(nxt) if p >= 0)
