"""RowSel sharded across GPUs by NTT point (one process per GPU).

The paper spreads its database over several GPUs (Sec. 6, "DB sharding") so
that each GPU holds and scans only part of it. RowSel is one independent GEMM
per NTT point p = (limb, slot) (Sec. 2.3), so the cheapest split is by point:
rank r of W keeps slots [t0, t1) of every limb of every database polynomial,
receives the same slots of every selection ciphertext, and computes the same
slots of every output. Each rank's work is a complete RowSel on a ring of
T = t1 - t0 points; no data moves between ranks while RowSel runs. Assembling
a full output polynomial (needed by a following ColTor, whose NTTs mix all
points) is one gather of the ranks' slices along the slot axis.

Constraints: W divides N and T = N / W is a power of two, so each shard is a
valid parameter set for the library (q = 1 mod 2N implies q = 1 mod 2T), and
T is a multiple of 8 whenever N / W >= 8 (the tensor-core path's 8-slot
groups stay whole).

This module only plans the split and moves slices (numpy or torch arrays, on
any device); every RowSel step still runs in libgpir.so.
"""


class SlotShard:
    """Rank `rank` of `world`: slots [t0, t1) of a ring of N points."""

    def __init__(self, N, world, rank):
        N, world, rank = int(N), int(world), int(rank)
        if world < 1 or not 0 <= rank < world:
            raise ValueError("rank %d of world %d" % (rank, world))
        if N % world:
            raise ValueError("world %d does not divide N = %d" % (world, N))
        T = N // world
        if T & (T - 1):
            raise ValueError("N / world = %d is not a power of two" % T)
        self.N, self.world, self.rank = N, world, rank
        self.T = T
        self.t0 = rank * T
        self.t1 = self.t0 + T

    def take(self, x):
        """This rank's slots of an array whose last axis is the N slots
        ([..., L, N] layouts: db, ct, out), as a new contiguous array."""
        if x.shape[-1] != self.N:
            raise ValueError("last axis %d is not N = %d" % (x.shape[-1], self.N))
        s = x[..., self.t0:self.t1]
        return s.contiguous() if hasattr(s, "contiguous") else s.copy()

    def __repr__(self):
        return "SlotShard(N=%d, world=%d, rank=%d, slots=[%d, %d))" % (self.N, self.world, self.rank, self.t0,
                                                                         self.t1)


def assemble(parts):
    """Full array from the W ranks' slices (rank order) along the slot axis."""
    if hasattr(parts[0], "contiguous"):
        import torch
        return torch.cat(list(parts), dim=-1)
    import numpy as np
    return np.concatenate(list(parts), axis=-1)


def gather(part, group=None):
    """All-gather of every rank's slice (a torch tensor; any process-group
    backend) and reassembly of the full array on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(parts, part.contiguous(), group=group)
    return assemble(parts)
