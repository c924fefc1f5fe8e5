"""The multi-GPU path's host logic on CPU: two gloo ranks take disjoint
tree-id ranges, sum their integer counts and install them; the result must
equal one process sampling all the trees (oracle counts stand in for each
rank's GPU counts)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth

TREES_PER_RANK = 24
SEED = 77


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _OracleCtx:
    """A context whose tree counts come from the oracle (CPU)."""

    def __init__(self, g, u):
        import oracle
        self.g, self.u = g, u
        self.par = oracle.bfs(g, u)[2]
        self.installed = None
        self.solves = 0
        self.x = None

    def tree_range_counts(self, t0, t1, seed, out=None):
        import oracle
        return oracle.sample_aggregate(self.g, self.u, self.par, t0, t1, seed)[0]

    def set_counts(self, R, trees):
        self.installed = (np.array(R, dtype=np.int64), int(trees))

    def column(self, out=None):
        import oracle
        self.solves += 1
        self.x = oracle.cg(self.g, self.u, tol=1e-12)[0]
        return self.x

    def diag(self, eps=0.0, out=None):
        import oracle
        R, trees = self.installed
        return oracle.combine(R, trees, self.x, self.u)


def _rank_main(rank, world, port, results):
    import torch.distributed as dist

    from paper_2006_13679_gb300 import parallel
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = synth.grid(7, 6)
        ctx = _OracleCtx(g, 17)
        parallel.sample_sharded(ctx, TREES_PER_RANK, SEED)
        R, trees = ctx.installed
        results.put((rank, R.tolist(), trees, parallel.tree_range(rank, world, TREES_PER_RANK)))
    finally:
        dist.destroy_process_group()


def test_tree_ranges_partition_the_ids():
    from paper_2006_13679_gb300 import parallel
    ranges = [parallel.tree_range(r, 4, 10) for r in range(4)]
    assert ranges == [(0, 10), (10, 20), (20, 30), (30, 40)]
    with pytest.raises(ValueError):
        parallel.tree_range(4, 4, 10)


def test_two_gloo_ranks_equal_one_process():
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, results)) for r in range(world)]
    for p in procs:
        p.start()
    got = [results.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = synth.grid(7, 6)
    par = oracle.bfs(g, 17)[2]
    R_all, _ = oracle.sample_aggregate(g, 17, par, 0, world * TREES_PER_RANK, SEED)
    for rank, R, trees, rng in sorted(got):
        assert rng == (rank * TREES_PER_RANK, (rank + 1) * TREES_PER_RANK)
        assert trees == world * TREES_PER_RANK
        assert np.array_equal(np.array(R, dtype=np.int64), R_all)


def _diag_rank_main(rank, world, port, results):
    import torch.distributed as dist

    from paper_2006_13679_gb300 import parallel
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = synth.grid(7, 6)
        ctx = _OracleCtx(g, 17)
        d = parallel.diag_sharded(ctx, TREES_PER_RANK, SEED)
        results.put((rank, None if d is None else list(d), ctx.solves))
    finally:
        dist.destroy_process_group()


def test_only_the_solver_rank_solves_and_combines():
    """The column is solved once, by rank 0, and the diagonal formed there
    from the summed counts equals one process's diagonal over all trees."""
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_diag_rank_main, args=(r, world, port, results)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(results.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = synth.grid(7, 6)
    par = oracle.bfs(g, 17)[2]
    R_all, _ = oracle.sample_aggregate(g, 17, par, 0, world * TREES_PER_RANK, SEED)
    x = oracle.cg(g, 17, tol=1e-12)[0]
    (r0, d0, s0), (r1, d1, s1) = got
    assert (r0, s0, r1, s1) == (0, 1, 1, 0) and d1 is None
    np.testing.assert_allclose(np.array(d0), oracle.combine(R_all, world * TREES_PER_RANK, x, 17), rtol=1e-12,
                               atol=0)
