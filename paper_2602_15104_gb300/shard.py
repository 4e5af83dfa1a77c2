"""k-range sharding of the C_l quadrature across ranks.

The C_l of one cosmology is a trapezoid sum over the ln k nodes (paper App.
B.4, eq. c_ell_def).  Split the nodes into contiguous shards that share their
boundary node: the trapezoid over each shard then carries exactly the weights
the full grid gives its nodes (the shared node gets half an interval from
each side), so the per-shard C_l -- from abcmb_cl (or abcmb_cl_mixed) called
on the shard's k nodes and transfer functions -- add up to the single-pass
C_l, up to the order of summation.  The exchange step is one sum-reduction
of 3 (l_max - 1) doubles per cosmology.

Each k mode's ODE and projection are independent, so the only cross-rank
communication is that reduction; sharding by cosmology instead needs none.
"""
from __future__ import annotations


def k_shard(n_k: int, rank: int, world: int) -> tuple[int, int]:
    """Half-open node range [lo, hi) of rank's shard of n_k ascending k
    nodes; consecutive shards overlap in one node.  Every shard has at least
    two nodes, so world may not exceed n_k - 1."""
    if n_k < 2 or world < 1 or not (0 <= rank < world) or world > n_k - 1:
        raise ValueError("need 1 <= world <= n_k - 1 and 0 <= rank < world")
    intervals = n_k - 1
    lo = rank * intervals // world
    hi = (rank + 1) * intervals // world + 1
    return lo, hi


def reduce_partial_cl(cl_partial, dist, group=None):
    """Sum the ranks' partial C_l tensors in place (torch.distributed
    all_reduce; gloo for CPU tensors, NCCL for device tensors) and return
    them."""
    dist.all_reduce(cl_partial, op=dist.ReduceOp.SUM, group=group)
    return cl_partial
