"""Multi-GPU partition of a pair list (host logic).

Shell pairs are independent, so a pair list splits across ranks with no
exchange of integrals: each rank evaluates a contiguous, cost-balanced slice
(estimated FP64 flops of the count model) and writes its own blocks.  Only a
reduction of per-rank timings or of forces needs a collective.
"""
import numpy as np

from . import counts


def pair_costs(l, nprim, pair_a, pair_b, op=counts.OP_COULOMB):
    l = np.asarray(l)
    k = np.asarray(nprim)
    return counts.pair_flops(l[pair_a], l[pair_b], k[pair_a], k[pair_b], op)


def shard_bounds(costs, world):
    """Contiguous slices [b[r], b[r+1]) whose cost sums are as equal as a
    prefix split allows."""
    c = np.cumsum(np.asarray(costs, dtype=np.float64))
    total = c[-1] if len(c) else 0.0
    targets = total * np.arange(1, world) / world
    inner = np.searchsorted(c, targets, side="left") + 1 if len(c) else np.zeros(world - 1, dtype=np.int64)
    return np.concatenate([[0], np.minimum(inner, len(c)), [len(c)]]).astype(np.int64)


def shard_pairs(l, nprim, pair_a, pair_b, rank, world, op=counts.OP_COULOMB):
    """(pair_a, pair_b, first index) of this rank's slice."""
    b = shard_bounds(pair_costs(l, nprim, pair_a, pair_b, op), world)
    lo, hi = int(b[rank]), int(b[rank + 1])
    return np.asarray(pair_a)[lo:hi], np.asarray(pair_b)[lo:hi], lo
