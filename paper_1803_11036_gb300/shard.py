"""Routers spread over several GPUs, one process per GPU: the merge of Algorithm 5 across ranks.

The paper deploys one monitor server per edge router and ships every server's RSEA to one server,
which merges them with UnionSE (Sec. 4); it leaves the transport open. Here each rank (one GPU)
holds the RSEAs of some routers, and the end of a slot runs in four steps:

1. local merge: the rank's routers are merged on its GPU (ssd_merge, the minimum of the union
   reading) into one RSEA, read out as distance recorders (ssd_sketch_export to device memory);
2. reduce-scatter by recorder range: that RSEA is cut into `world` ranges of whole estimators;
   range j goes to rank j (one all_to_all of bytes), which folds the `world` slices it then holds
   with the elementwise minimum (ssd_min_merge) into its range of the global RSEA;
3. gather: the root rank receives every range into one distance array, loads it into its global
   sketch (ssd_sketch_import from device memory) and regains the sliding super points
   (ssd_regain); the other ranks send theirs;
4. every rank advances its routers (ssd_advance).

The exchange carries distances, not the library's stored stamps, so it does not depend on the
ranks' sketch clocks.

Per slot every rank sends and receives (world-1)/world of one RSEA in step 2, and the root
receives (world-1)/world of one more in step 3, however many routers a rank holds. Collective
libraries offer no 16-bit minimum, so they move bytes and the library's kernel reduces them.
The minimum commutes with the saturating advance and is associative, so the global RSEA, and the
list, are those of one process merging every router (checked by the tests on gloo ranks).
"""
from __future__ import annotations

from typing import Callable, Sequence


def estimator_ranges(n_estimators: int, eta: int, world: int) -> list[tuple[int, int]]:
    """(first recorder, recorder count) of each rank's range of an RSEA of n_estimators
    estimators of eta recorders: whole estimators, contiguous, in rank order, sizes differing by
    at most one estimator. A rank may get an empty range when there are more ranks than
    estimators."""
    if world < 1 or n_estimators < 0 or eta < 1:
        raise ValueError("estimator_ranges needs world >= 1, n_estimators >= 0, eta >= 1")
    base, extra = divmod(n_estimators, world)
    out, first = [], 0
    for j in range(world):
        n = base + (1 if j < extra else 0)
        out.append((first * eta, n * eta))
        first += n
    return out


def reduce_scatter_min(full, ranges: Sequence[tuple[int, int]], rank: int,
                       fold: Callable, group=None):
    """Step 2: this rank's range of the global RSEA. `full` is this rank's merged RSEA (a 1-D
    tensor of 16-bit recorders); every rank sends range j of it to rank j and receives its own
    range from every rank (one all_to_all of bytes), then `fold(out, slices)` writes the
    elementwise minimum of the `world` slices into `out`."""
    import torch
    import torch.distributed as dist
    world = len(ranges)
    first, count = ranges[rank]
    recv = torch.empty(world * count * 2, dtype=torch.uint8, device=full.device)
    dist.all_to_all_single(recv, full.view(torch.uint8),
                           output_split_sizes=[count * 2] * world,
                           input_split_sizes=[c * 2 for _, c in ranges], group=group)
    slices = list(recv.view(full.dtype).split(count)) if count else []
    out = torch.empty(count, dtype=full.dtype, device=full.device)
    if count:
        fold(out, slices)
    return out


def gather_ranges(shard, ranges: Sequence[tuple[int, int]], rank: int, root: int, dest=None, group=None):
    """Step 3: the root receives every rank's range into `dest` (its global RSEA's recorders, a
    1-D 16-bit tensor); the other ranks send theirs. Ranges are moved as bytes."""
    import torch
    import torch.distributed as dist
    if rank == root:
        if dest is None:
            raise ValueError("the root needs a destination for the global RSEA")
        first, count = ranges[root]
        dest[first:first + count].copy_(shard)
        reqs = []
        for j, (f, c) in enumerate(ranges):
            if j != root and c:
                peer = j if group is None else dist.get_global_rank(group, j)
                reqs.append(dist.irecv(dest[f:f + c].view(torch.uint8), src=peer, group=group))
        for q in reqs:
            q.wait()
    elif shard.numel():
        peer = root if group is None else dist.get_global_rank(group, root)
        dist.send(shard.view(torch.uint8), dst=peer, group=group)


class ShardedDetector:
    """One rank's share of a detector whose routers are spread over the ranks of a process group,
    one GPU per rank (torch.distributed initialised by the caller; NCCL for CUDA tensors).

    Per slot, every rank scans its own routers' pairs (Context.scan / scan_batch), then calls
    close_slot(), which runs steps 1-4 above on torch's current stream and returns the sliding
    super point list (ips, rk) on the root and None elsewhere. Every rank's routers share one
    parameter set, hash tables and view, and stay at one slot."""

    def __init__(self, ctx, routers, root: int = 0, group=None):
        import torch.distributed as dist
        if not routers:
            raise ValueError("a rank holds at least one router")
        self.ctx, self.routers, self.root, self.group = ctx, list(routers), root, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        view = self.routers[0].view
        self.local = ctx.sketch().set_view(*view)
        self.glob = ctx.sketch().set_view(*view) if self.rank == root else None
        p = ctx.params
        self.ranges = estimator_ranges(p.r << p.q, 1 << p.log2_eta, self.world)
        self._local_dist = None      # the local merge as distances (step 1)
        self._global_dist = None     # the gathered global RSEA as distances (root, step 3)

    def _fold(self, out, slices):
        self.ctx.min_merge(out, slices)

    def close_slot(self, cap: int = 1 << 16):
        import torch
        ctx = self.ctx
        ctx.merge(self.routers, self.local)                               # step 1
        self._local_dist = self.local.export_device(self._local_dist)
        shard = reduce_scatter_min(self._local_dist, self.ranges, self.rank, self._fold,
                                   self.group)                            # step 2
        dest = None
        if self.glob is not None:
            if self._global_dist is None:
                self._global_dist = torch.empty_like(self._local_dist)
            dest = self._global_dist
        gather_ranges(shard, self.ranges, self.rank, self.root, dest, self.group)   # step 3
        result = None
        if self.glob is not None:
            self.glob.load_device(self._global_dist, self.routers[0].slot)
            result = ctx.regain(self.glob, cap=cap)
        ctx.advance(self.routers)                                         # step 4
        return result

    def close(self) -> None:
        self.local.close()
        if self.glob is not None:
            self.glob.close()
