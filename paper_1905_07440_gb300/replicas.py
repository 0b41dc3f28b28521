"""Replica sharding of independent chains over ranks (one process per GPU).

Chains never interact, so N GPUs run N engines on disjoint chain ranges with no collective
on the data path; the only cross-rank operations are host-side: the max of the timed
region over ranks and an optional gather of per-chain results for reporting.  Philox chain
ids stay global (first_chain = rank's offset), so a chain's trajectory does not depend on
how the chains are split.
"""


def shard(total_chains, world, rank):
    """(first_chain, n_chains) of `rank` when total_chains are split as evenly as possible."""
    if world < 1 or not (0 <= rank < world) or total_chains < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total_chains, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def max_over_ranks(value, device=None):
    """Max of a float over all ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_per_chain(rows, first_chain):
    """Gather (first_chain, rows) from every rank; returns the rows ordered by chain id."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(rows)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, (int(first_chain), list(rows)))
    out = []
    for _, r in sorted(parts, key=lambda x: x[0]):
        out.extend(r)
    return out
