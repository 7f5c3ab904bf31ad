"""The block filter shared out among several GPUs (Eq. 4step step 1).

The blocks of a decomposition decouple in the filter step: the active links
of different blocks share no plaquette and a block's Dirichlet operator holds
only the links inside it (Sec. 3), so every block's log-ratio can be computed
on any GPU that holds the gauge field.  Each rank takes one contiguous range
of block positions (block order: black blocks first, then white) of the
selected colours, computes the log-ratios of its blocks
(dd_block_ratios_range), the ranks exchange them with one sum-all-reduce of
the nblocks-long vector (the ranges are disjoint and every other entry is an
exact zero, so the sum reproduces each value bit for bit), and every rank
takes the same decisions and restores the same links (dd_block_accept) on its
copy of the field.  The communication is one all-reduce of nblocks doubles
per filter step; the gauge field itself is replicated.

`filter_partition_step` holds the host logic with the compute and
communication steps passed in, so that it runs unchanged with the CUDA
library and NCCL or gloo process groups (`partitioned_block_filter`).
"""


def block_ranges(nblocks, colour_mask, world):
    """Contiguous block-order ranges (pos0, npos), one per rank, that cover the
    blocks of the selected colours as evenly as possible."""
    if world < 1 or colour_mask not in (1, 2, 3) or nblocks % 2:
        raise ValueError("bad partition request")
    half = nblocks // 2
    first = half if colour_mask == 2 else 0
    count = nblocks if colour_mask == 3 else half
    q, r = divmod(count, world)
    out, pos = [], first
    for k in range(world):
        n = q + (1 if k < r else 0)
        out.append((pos, n))
        pos += n
    return out


def filter_partition_step(rank, world, nblocks, colour_mask, compute_range, reduce_sum, decide):
    """One partitioned filter step.
      compute_range(pos0, npos) -> ln_b of this rank's blocks (0 elsewhere)
      reduce_sum(ln_b)          -> the element-wise sum over all ranks
      decide(ln_b)              -> decisions (and the restore of rejected blocks)
    Returns (ln_b, decisions), the same on every rank."""
    pos0, npos = block_ranges(nblocks, colour_mask, world)[rank]
    ln_b = compute_range(pos0, npos)
    ln_b = reduce_sum(ln_b)
    return ln_b, decide(ln_b)


def partitioned_block_filter(h, U_old, U_new, colour_mask, n, seed, ctr, group=None):
    """dd_block_filter's stochastic filter (persistent per-block form) with
    the blocks shared out over the ranks of `group` (torch.distributed; one
    GPU per rank, every rank holding the same U_old and U_new).  U_new gets
    the rejected blocks restored on every rank.  Returns (ln_b, accept)."""
    import torch.distributed as dist

    from . import api

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0

    def compute_range(pos0, npos):
        return api.dd_block_ratios_range(h, U_old, U_new, pos0, npos, n, seed, ctr)

    def reduce_sum(ln_b):
        if world > 1:
            dist.all_reduce(ln_b, op=dist.ReduceOp.SUM, group=group)
        return ln_b

    def decide(ln_b):
        return api.dd_block_accept(h, U_old, U_new, colour_mask, ln_b, seed, ctr)

    return filter_partition_step(rank, world, h.nfine, colour_mask, compute_range, reduce_sum, decide)
