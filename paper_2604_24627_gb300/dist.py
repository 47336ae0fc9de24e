"""Host-side sharding of cells across ranks (one process per GPU).

Every operator is cell-local and random numbers are keyed by the global cell
index, so a shard is a contiguous cell range with its cell_index_base and the
result does not depend on how cells are split. The only collective is the sum
of diagnostics (spectrum tally and counters).
"""
import numpy as np


def shard_range(ncells, world, rank):
    """Contiguous block partition: (first global cell, count) of `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(ncells, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def allreduce_tally(H, totals, dist_module, group=None):
    """Sum a tally (H [3, nbins], totals dict) over ranks with
    torch.distributed (any backend); returns the summed copies."""
    import torch
    keys = sorted(totals)
    flat = np.concatenate([np.asarray(H, dtype=np.float64).reshape(-1),
                           np.array([totals[k] for k in keys], dtype=np.float64)])
    t = torch.from_numpy(flat.copy())
    dist_module.all_reduce(t, group=group)
    out = t.numpy()
    n = np.asarray(H).size
    return out[:n].reshape(np.asarray(H).shape), dict(zip(keys, out[n:]))
