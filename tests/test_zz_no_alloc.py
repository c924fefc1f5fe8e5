"""The allocation-free entry point ust_tree_counts_noalloc, through the C ABI.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator that must account for every byte (a framework's caching
allocator, a fixed memory budget), or they may not allocate after start-up.
ust_tree_counts_noalloc serves them from one fixed scratch array inside the
library. Its counts must equal those of the allocating entry point
ust_tree_range_counts exactly (they are integers), on consecutive calls that
reuse the same scratch array.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _call(L, rp, ci, g, u, t0, t1, seed, out, stream):
    return L.ust_tree_counts_noalloc(ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()), g.n, g.nnz,
                                     u, t0, t1, seed, 0, ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("name", ["grid48", "rmat12"])
def test_noalloc_counts_equal_allocating_entry_point(name):
    import torch

    import paper_2006_13679_gb300 as pkg
    pkg.build()
    L = pkg.load()
    if name == "grid48":
        g, u = synth.grid(48, 48), 24 * 48 + 24
    else:
        g = synth.rmat(12, 16, seed=5)
        u = synth.max_degree_vertex(g)
    calls = [(0, 500, 0), (500, 1000, 7)]  # two calls in a row on the same scratch array
    with pkg.UST(g.row_ptr, g.col_idx, u) as h:
        refs = [h.tree_range_counts(t0, t1, seed) for t0, t1, seed in calls]
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    out = torch.full((g.n,), -7, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    for (t0, t1, seed), ref in zip(calls, refs):
        rc = _call(L, rp, ci, g, u, t0, t1, seed, out, stream)
        assert rc == 0, L.ust_strerror(rc)
        np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    import paper_2006_13679_gb300 as pkg
    L = pkg.load()
    g = synth.grid(80, 80)  # n = 6400 > 4096
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    out = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    rc = _call(L, rp, ci, g, 0, 0, 10, 1, out, torch.cuda.current_stream())
    assert rc == pkg.UST_EINVAL
    assert not out.any()
