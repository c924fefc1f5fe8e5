"""GB300 (sm_103a) UST approximation of diag(L^+) (arXiv 2006.13679).

The computation lives in libust.so (CUDA, C ABI in include/ust.h). This
package builds it (``build()``) and wraps it: ``UST`` mirrors the C calls
one to one and only marshals arguments. Host arguments are numpy arrays;
device arguments are torch CUDA tensors (PyTorch supplies device memory and
streams only).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding
from ._binding import (UST_EINVAL, UST_ENOMEM, UST_ENOTCONNECTED, UST_ENOTCONVERGED, UST_ESTATE,
                       UST_ETIMEOUT, UST_OK, UstError, check, load)
from ._build import LIB as LIB_PATH

__all__ = ["UST", "USTBatch", "select_pivot", "probe_random_access", "build", "load", "UstError", "LIB_PATH", "UST_OK", "UST_EINVAL", "UST_ENOTCONNECTED",
           "UST_ENOMEM", "UST_ETIMEOUT", "UST_ENOTCONVERGED", "UST_ESTATE"]


def build(force: bool = False) -> str:
    """Compiles libust.so for sm_103a with nvcc (in-tree) and loads it."""
    from . import _build
    path = _build.build(force=force)
    load()
    return path


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, on_device) for a numpy array or a contiguous torch tensor (a
    CPU tensor, pinned or not, is a host buffer; a CUDA tensor a device one)."""
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor arguments must be contiguous")
        if x.element_size() != np.dtype(dtype).itemsize:
            raise TypeError(f"expected {np.dtype(dtype).name} elements")
        return ctypes.c_void_p(x.data_ptr()), (1 if x.is_cuda else 0)
    a = np.ascontiguousarray(x)
    if a.dtype != dtype:
        raise TypeError(f"expected {np.dtype(dtype).name}, got {a.dtype}")
    return ctypes.c_void_p(a.ctypes.data), 0


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def select_pivot(row_ptr, col_idx, sweeps: int = 10, start: int = -1, stream=None) -> tuple[int, int]:
    """``ust_select_pivot``: (pivot, eccentricity lower bound) by double sweeps."""
    L = load()
    rp = row_ptr if _is_torch(row_ptr) else np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = col_idx if _is_torch(col_idx) else np.ascontiguousarray(col_idx, dtype=np.int32)
    prp, dev = _ptr(rp, np.int32)
    pci, _ = _ptr(ci, np.int32)
    g = _binding.ust_csr(n=int(rp.shape[0]) - 1, nnz=int(ci.shape[0]), row_ptr=prp.value, col_idx=pci.value,
                         on_device=dev)
    sh = _stream_handle(stream)
    piv, bound = ctypes.c_int32(), ctypes.c_int32()
    check(L.ust_select_pivot(ctypes.byref(g), int(sweeps), int(start), sh, ctypes.byref(piv), ctypes.byref(bound)))
    return int(piv.value), int(bound.value)


def probe_random_access(nbytes: int, mode: int = 0, reps: int = 3, stream=None) -> float:
    """``ust_probe_random_access``: random 4-byte accesses per second over a
    device array of ``nbytes`` (mode 0 loads through L2, mode 1 atomics)."""
    out = ctypes.c_double()
    rc = load().ust_probe_random_access(int(nbytes), int(mode), int(reps), _stream_handle(stream), ctypes.byref(out))
    if rc != 0:
        raise UstError(rc, "random-access probe failed")
    return float(out.value)


class UST:
    """One graph and pivot: ``ust_init`` ... ``ust_free``.

    row_ptr, col_idx: int32 CSR (numpy on the host or torch CUDA tensors),
    symmetric, sorted rows, no self-loops, connected. pivot: the vertex u.
    wilson_blocks: sample with the biconnected-component variant (every
    vertex walks inside its parent block; ``ust_opts.wilson_blocks``).
    """

    def __init__(self, row_ptr, col_idx, pivot: int, *, delta: float = 0.0, kappa: float = 0.3,
                 cg_tol: float = 1e-9, max_pop_rounds: int = 0, max_cg_iters: int = 0, graph_id: int = 0,
                 block_threads: int = 0, ctas_per_sm: int = 0, stream=None, skip_validation: bool = False,
                 solve_fp64: bool = False, wilson_blocks: bool = False, autotune: int = 0):
        L = load()
        self._keep = []
        rp = row_ptr if _is_torch(row_ptr) else np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = col_idx if _is_torch(col_idx) else np.ascontiguousarray(col_idx, dtype=np.int32)
        self._keep += [rp, ci]
        prp, dev_rp = _ptr(rp, np.int32)
        pci, dev_ci = _ptr(ci, np.int32)
        if dev_rp != dev_ci:
            raise ValueError("row_ptr and col_idx must both be host or both be device arrays")
        n = int(rp.shape[0]) - 1
        g = _binding.ust_csr(n=n, nnz=int(ci.shape[0]), row_ptr=prp.value, col_idx=pci.value, on_device=dev_rp)
        o = _binding.default_opts()
        o.delta, o.kappa, o.cg_tol = delta, kappa, cg_tol
        o.max_pop_rounds, o.max_cg_iters = max_pop_rounds, max_cg_iters
        o.skip_validation = int(bool(skip_validation))
        o.graph_id, o.block_threads, o.ctas_per_sm = graph_id, block_threads, ctas_per_sm
        o.solve_fp64 = int(bool(solve_fp64))
        o.wilson_blocks = int(bool(wilson_blocks))
        o.autotune = int(autotune)
        sh = _stream_handle(stream)
        o.stream = sh.value if sh is not None else None
        h = ctypes.c_void_p()
        rc = L.ust_init(ctypes.byref(g), int(pivot), ctypes.byref(o), ctypes.byref(h))
        check(rc, None)
        self._h = h
        self.n = n
        self.pivot = int(pivot)

    # -- lifecycle
    def close(self) -> None:
        if getattr(self, "_h", None):
            load().ust_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def reset(self, pivot: int) -> None:
        check(load().ust_reset(self._h, int(pivot)), self._h)
        self.pivot = int(pivot)

    def sample_aggregate(self, n_trees: int, seed: int) -> None:
        check(load().ust_sample_aggregate(self._h, int(n_trees), int(seed) & (2 ** 64 - 1)), self._h)

    def tau(self, eps: float) -> int:
        return int(load().ust_tau(self._h, float(eps)))

    def num_trees(self) -> int:
        """``ust_num_trees``: trees aggregated in R so far."""
        return int(load().ust_num_trees(self._h))

    def _out(self, out, dtype, count):
        if out is None:
            out = np.empty(count, dtype=dtype)
        p, dev = _ptr(out, dtype)
        return out, p, dev

    def diag(self, eps: float = 0.0, out=None):
        out, p, dev = self._out(out, np.float64, self.n)
        check(load().ust_diag(self._h, float(eps), p, dev), self._h)
        return out

    def centralities(self, eps: float = 0.0) -> dict:
        """Electrical closeness, normalized random-walk betweenness (n each)
        and Kirchhoff index (one per graph) from the diagonal estimate."""
        count = getattr(self, "count", 1)
        cl = np.empty(self.n, dtype=np.float64)
        nr = np.empty(self.n, dtype=np.float64)
        kf = np.empty(count, dtype=np.float64)
        check(load().ust_centralities(self._h, float(eps), ctypes.c_void_p(cl.ctypes.data),
                                      ctypes.c_void_p(nr.ctypes.data), ctypes.c_void_p(kf.ctypes.data), 0), self._h)
        return {"closeness": cl, "nrwb": nr, "kirchhoff": kf if count > 1 else float(kf[0])}

    def track_edges(self, on: bool = True) -> None:
        """Counts, per CSR arc v -> w, the sampled trees in which w is v's parent."""
        check(load().ust_track_edges(self._h, int(bool(on))), self._h)

    def edge_counts(self, out=None):
        nnz = getattr(self, "nnz", None) or int(self.info()["nnz"])
        out, ptr, dev = self._out(out, np.int64, nnz)
        check(load().ust_get_edge_counts(self._h, ptr, dev), self._h)
        return out

    def counts(self, out=None):
        out, p, dev = self._out(out, np.int64, self.n)
        check(load().ust_get_counts(self._h, p, dev), self._h)
        return out

    def column(self, out=None):
        out, p, dev = self._out(out, np.float64, self.n)
        check(load().ust_get_column(self._h, p, dev), self._h)
        return out

    def bfs(self):
        par = np.empty(self.n, dtype=np.int32)
        dist = np.empty(self.n, dtype=np.int32)
        check(load().ust_get_bfs(self._h, ctypes.c_void_p(par.ctypes.data), ctypes.c_void_p(dist.ctypes.data)),
              self._h)
        return par, dist

    def tree_range_counts(self, t0: int, t1: int, seed: int, out=None):
        out, p, dev = self._out(out, np.int64, self.n)
        check(load().ust_tree_range_counts(self._h, int(t0), int(t1), int(seed) & (2 ** 64 - 1), p, dev), self._h)
        return out

    def set_counts(self, R, trees: int) -> None:
        """Installs exact counts of `trees` trees (e.g. summed over GPUs) as R."""
        R = R if _is_torch(R) else np.ascontiguousarray(R, dtype=np.int64)
        ptr, dev = _ptr(R, np.int64)
        check(load().ust_set_counts(self._h, ptr, int(trees), dev), self._h)

    def sample_trees(self, t0: int, count: int, seed: int, with_pops: bool = False):
        nxt = np.empty((count, self.n), dtype=np.int32)
        pops = np.empty((count, self.n), dtype=np.int32) if with_pops else None
        check(load().ust_sample_trees(self._h, int(t0), int(count), int(seed) & (2 ** 64 - 1),
                                      ctypes.c_void_p(nxt.ctypes.data),
                                      ctypes.c_void_p(pops.ctypes.data) if with_pops else None), self._h)
        return (nxt, pops) if with_pops else nxt

    def info(self) -> dict:
        i = _binding.ust_info()
        check(load().ust_get_info(self._h, ctypes.byref(i)), self._h)
        return i.as_dict()


class USTBatch:
    """A batch of graphs in one context: ``ust_init_batch`` ... ``ust_free``.

    graphs: list of (row_ptr, col_idx) int32 CSR arrays (numpy, host);
    pivots: one pivot per graph. Per-vertex outputs are the graphs' values one
    after another; ``offsets()`` gives where each graph starts. Graph g draws
    with fourth Philox counter word graph_id + g.
    """

    def __init__(self, graphs, pivots, *, delta: float = 0.0, kappa: float = 0.3, cg_tol: float = 1e-9,
                 max_pop_rounds: int = 0, max_cg_iters: int = 0, graph_id: int = 0, block_threads: int = 0,
                 ctas_per_sm: int = 0, stream=None, skip_validation: bool = False, solve_fp64: bool = False,
                 wilson_blocks: bool = False, autotune: int = 0):
        L = load()
        self._keep = []
        csrs = (_binding.ust_csr * len(graphs))()
        for i, (rp, ci) in enumerate(graphs):
            rp = np.ascontiguousarray(rp, dtype=np.int32)
            ci = np.ascontiguousarray(ci, dtype=np.int32)
            self._keep += [rp, ci]
            csrs[i] = _binding.ust_csr(n=int(rp.shape[0]) - 1, nnz=int(ci.shape[0]), row_ptr=rp.ctypes.data,
                                       col_idx=ci.ctypes.data, on_device=0)
        piv = np.ascontiguousarray(pivots, dtype=np.int32)
        self._keep.append(piv)
        o = _binding.default_opts()
        o.delta, o.kappa, o.cg_tol = delta, kappa, cg_tol
        o.max_pop_rounds, o.max_cg_iters = max_pop_rounds, max_cg_iters
        o.skip_validation = int(bool(skip_validation))
        o.graph_id, o.block_threads, o.ctas_per_sm = graph_id, block_threads, ctas_per_sm
        o.solve_fp64 = int(bool(solve_fp64))
        o.wilson_blocks = int(bool(wilson_blocks))  # single-graph contexts only: UST_EINVAL here
        o.autotune = int(autotune)
        sh = _stream_handle(stream)
        o.stream = sh.value if sh is not None else None
        h = ctypes.c_void_p()
        rc = L.ust_init_batch(csrs, piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(graphs),
                              ctypes.byref(o), ctypes.byref(h))
        check(rc, None)
        self._h = h
        self.count = len(graphs)
        self._off = np.empty(self.count + 1, dtype=np.int64)
        check(L.ust_batch_offsets(h, ctypes.c_void_p(self._off.ctypes.data)), h)
        self.n = int(self._off[-1])

    def reset(self) -> None:
        """Recomputes every graph's B_u (same pivots) and clears counts and columns."""
        check(load().ust_reset(self._h, -1), self._h)

    close = UST.close
    __del__ = UST.__del__
    __enter__ = UST.__enter__
    __exit__ = UST.__exit__
    sample_aggregate = UST.sample_aggregate
    set_counts = UST.set_counts
    tau = UST.tau
    num_trees = UST.num_trees
    _out = UST._out
    diag = UST.diag
    centralities = UST.centralities
    track_edges = UST.track_edges
    edge_counts = UST.edge_counts
    counts = UST.counts
    column = UST.column
    info = UST.info

    def offsets(self) -> np.ndarray:
        return self._off.copy()

    def graph_info(self, g: int) -> dict:
        i = _binding.ust_info()
        check(load().ust_batch_graph_info(self._h, int(g), ctypes.byref(i)), self._h)
        return i.as_dict()

    def split(self, values) -> list:
        """Per-graph views of a concatenated per-vertex output."""
        return [values[self._off[g]:self._off[g + 1]] for g in range(self.count)]
