"""The allocation-free entry point ust_tree_counts_noalloc, through the C ABI.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator that must account for every byte (a framework's caching
allocator, a fixed memory budget), or they may not allocate after start-up.
ust_tree_counts_noalloc serves them from one fixed scratch array inside the
library. Its counts must equal those of the allocating entry point
ust_tree_range_counts exactly (they are integers), and the oracle's, on
consecutive calls that reuse the same scratch array. Inputs beyond the
array's limits, and graphs that are not connected, are rejected with R_out
left as it was, and a valid call after a rejected one still gives the exact
counts.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

SENTINEL = -7


def _call(L, rp, ci, g, u, t0, t1, seed, out, stream):
    return L.ust_tree_counts_noalloc(ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()), g.n, g.nnz,
                                     u, t0, t1, seed, 0, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))


def _graph(name):
    if name == "grid48":
        return synth.grid(48, 48), 24 * 48 + 24
    g = synth.rmat(12, 16, seed=5)
    return g, synth.max_degree_vertex(g)


def _device(g):
    import torch
    return torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda()


@pytest.mark.parametrize("name", ["grid48", "rmat12"])
def test_noalloc_counts_equal_allocating_entry_point_and_oracle(name):
    import torch

    import oracle
    import paper_2006_13679_gb300 as pkg
    pkg.build()
    L = pkg.load()
    g, u = _graph(name)
    calls = [(0, 500, 0), (500, 1000, 7)]  # two calls in a row on the same scratch array
    with pkg.UST(g.row_ptr, g.col_idx, u) as h:
        refs = [h.tree_range_counts(t0, t1, seed) for t0, t1, seed in calls]
    _, _, par = oracle.bfs(g, u)
    rp, ci = _device(g)
    out = torch.full((g.n,), SENTINEL, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    for (t0, t1, seed), ref in zip(calls, refs):
        rc = _call(L, rp, ci, g, u, t0, t1, seed, out, stream)
        assert rc == 0, L.ust_strerror(rc)
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got, ref)
        R_orc, _ = oracle.sample_aggregate(g, u, par, t0, t1, seed)
        np.testing.assert_array_equal(got, R_orc)


@pytest.mark.parametrize("case", ["too_many_vertices", "too_many_path_entries", "not_connected"])
def test_noalloc_rejects_and_leaves_the_output_alone(case):
    import torch

    import oracle
    import paper_2006_13679_gb300 as pkg
    pkg.build()
    L = pkg.load()
    if case == "too_many_vertices":
        g, u, code = synth.grid(80, 80), 0, pkg.UST_EINVAL           # n = 6400 > 4096
    elif case == "too_many_path_entries":
        g, u, code = synth.path(1000), 0, pkg.UST_EINVAL             # f^c(u) = 499,500 > 262,144
    else:
        a = synth.cycle(12)                                          # two disjoint 12-cycles
        src = np.concatenate([np.repeat(np.arange(12), 2), 12 + np.repeat(np.arange(12), 2)])
        dst = np.concatenate([a.col_idx, 12 + a.col_idx])
        g = synth.from_edges(24, src, dst, lcc=False)
        u, code = 0, pkg.UST_ENOTCONNECTED
    rp, ci = _device(g)
    out = torch.full((g.n,), SENTINEL, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = _call(L, rp, ci, g, u, 0, 10, 1, out, stream)
    assert rc == code, L.ust_strerror(rc)
    assert bool((out == SENTINEL).all()), "a rejected call wrote to R_out"
    # the scratch array is still good for the next valid call
    g2, u2 = _graph("rmat12")
    rp2, ci2 = _device(g2)
    out2 = torch.full((g2.n,), SENTINEL, dtype=torch.int64, device="cuda")
    assert _call(L, rp2, ci2, g2, u2, 3, 203, 5, out2, stream) == 0
    _, _, par = oracle.bfs(g2, u2)
    np.testing.assert_array_equal(out2.cpu().numpy(), oracle.sample_aggregate(g2, u2, par, 3, 203, 5)[0])
