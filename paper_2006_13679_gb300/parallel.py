"""Sampling on several GPUs, one process per GPU.

Trees are independent units: a tree is fixed by (graph, pivot, seed, tree id)
through the Philox counter. So N processes take disjoint tree-id ranges under
one seed, each computes the exact Algorithm-2 counts of its range, and the
integer rows are summed. The sum equals the counts of one GPU sampling all the
trees, bit for bit. This is the paper's distributed scheme (Appendix D: trees
spread over processes, R reduced at the end), with the graph replicated on
every GPU. The sum is the only exchange of the path.

The column L^+[:, u] depends on the graph and pivot only, so one rank (the
solver rank) solves it, before the exchange, while the other ranks are still
sampling; no other rank solves. The solver rank then combines the summed
counts with its column into the diagonal.
"""
from __future__ import annotations


def tree_range(rank: int, world: int, trees_per_rank: int) -> tuple[int, int]:
    """Tree ids [t0, t1) of `rank`: rank r takes [r T, (r + 1) T)."""
    if not (0 <= rank < world) or trees_per_rank < 0:
        raise ValueError("need 0 <= rank < world and trees_per_rank >= 0")
    return rank * trees_per_rank, (rank + 1) * trees_per_rank


def sample_sharded(ctx, trees_per_rank: int, seed: int, group=None, out=None):
    """Counts of this rank's tree range, summed over the process group and
    installed in `ctx` (``set_counts``) as world * trees_per_rank trees.

    ctx: a ``UST`` context (or anything with ``tree_range_counts`` and
    ``set_counts``); out: optional int64 buffer for the counts (a CUDA tensor
    for NCCL). Returns the summed counts as a torch tensor.
    """
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    t0, t1 = tree_range(rank, world, trees_per_rank)
    R = ctx.tree_range_counts(t0, t1, seed, out=out)
    t = R if isinstance(R, torch.Tensor) else torch.from_numpy(R)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    ctx.set_counts(t if t.is_cuda else t.numpy(), world * trees_per_rank)
    return t


def diag_sharded(ctx, trees_per_rank: int, seed: int, out=None, solver_rank: int = 0, group=None,
                 counts_out=None):
    """diag(L^+) from world * trees_per_rank trees spread over the ranks.

    The solver rank solves the column first (``column()``: L^+[:, u] does not
    depend on the trees), then every rank samples its tree range and the
    counts are summed and installed (``sample_sharded``); the solver rank
    alone forms the diagonal (``diag``) into `out` and returns it, the other
    ranks return None. counts_out: optional int64 buffer for the counts.
    """
    import torch.distributed as dist

    rank = dist.get_rank(group)
    if rank == solver_rank:
        ctx.column()
    sample_sharded(ctx, trees_per_rank, seed, group=group, out=counts_out)
    if rank != solver_rank:
        return None
    return ctx.diag(0.0, out)
