"""Sharded single-linkage tree over several processes (one GPU each).

FAMSA Methods, "Pairwise similarities calculation": the pairs are
independent; "Determination of the guide tree": single linkage depends only
on a minimum spanning tree of the distance graph.  Each rank takes a range
of rows of the pair set, reduces it on its own device to a minimum spanning
tree of fewer than k edges (famsa_msf_rows), one all-gather exchanges the
trees, and every rank builds the tree of the whole family from their union
(famsa_tree_from_edges) -- the same tree one device would build.

The exchange is the only collective: a torch.distributed all-gather of
fixed-size edge tensors (NCCL between GPUs; gloo on the CPU in the tests).
Every step's arithmetic runs in the library's kernels; this module only
splits rows and moves buffers.
"""
from __future__ import annotations

import math

import numpy as np

FIELDS = (("edge_a", np.int32), ("edge_b", np.int32), ("h_num", np.uint64), ("h_den", np.uint32))


def shard_rows(k: int, world: int):
    """Row ranges [b_r, b_{r+1}) covering rows 1..k-1, with about equal pair counts
    (row i holds i pairs, so the cut points grow like sqrt(r / world))."""
    if k < 2:
        return [(1, 1)] * world
    cuts = [1]
    total = k * (k - 1) / 2
    for r in range(1, world):
        # rows 1..b-1 hold b(b-1)/2 pairs
        b = int(round(0.5 + math.sqrt(0.25 + 2 * total * r / world)))
        cuts.append(min(max(b, cuts[-1] + 1 if cuts[-1] < k else k), k))
    cuts.append(k)
    return [(cuts[r], max(cuts[r], cuts[r + 1])) for r in range(world)]


def _exchange(edges: dict, k: int, ranges, rank: int, world: int, dist, device):
    """All-gather every rank's edges (rank r holds ranges[r][1] - 1 of them)."""
    import torch
    n_max = max(k - 1, 1)
    counts = [max(e - 1, 0) if e > b else 0 for b, e in ranges]
    out = {}
    for name, dt in FIELDS:
        tdt = {np.int32: torch.int32, np.uint64: torch.int64, np.uint32: torch.int32}[dt]
        mine = torch.zeros(n_max, dtype=tdt, device=device)
        src = edges[name]
        if not isinstance(src, torch.Tensor):
            src = torch.from_numpy(np.ascontiguousarray(src).view(
                {np.int32: np.int32, np.uint64: np.int64, np.uint32: np.int32}[dt]))
        else:
            src = src.view(tdt)
        mine[:counts[rank]] = src[:counts[rank]].to(device)
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine)
        cat = torch.cat([parts[r][:counts[r]] for r in range(world)])
        out[name] = cat.cpu().numpy().view(dt) if device == "cpu" else cat.view(
            {np.int32: torch.int32, np.uint64: torch.uint64, np.uint32: torch.uint32}[dt])
    return out


def sharded_tree(residues, offsets, local_msf=None, merge=None, device=None):
    """The family's single-linkage tree, each rank of the default process group
    computing one shard of the pairs.

    local_msf(row_begin, row_end) -> edge dict of the rank's shard, and
    merge(k, edges) -> tree dict; by default the library's famsa_msf_rows on a
    family packed on this rank's GPU and famsa_tree_from_edges.  Returns the
    tree on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_initialized() else 1
    rank = dist.get_rank() if dist.is_initialized() else 0
    k = len(offsets) - 1
    ranges = shard_rows(k, world)
    fam = None
    if local_msf is None or merge is None:
        import paper_1603_06958_gb300 as fg
        if device is None:
            device = "cuda"
        if local_msf is None:
            fam = fg.pack_peq(residues, offsets)

            def local_msf(b, e):
                return fg.msf_rows(fam, b, e, device=True)
        if merge is None:
            def merge(kk, edges):
                return fg.tree_from_edges(kk, edges, device=(device != "cpu"))
    if device is None:
        device = "cpu"
    try:
        b, e = ranges[rank]
        if e > b:
            edges = local_msf(b, e)
        else:
            edges = {name: np.zeros(0, dt) for name, dt in FIELDS}
        if world > 1:
            edges = _exchange(edges, k, ranges, rank, world, dist, device)
        if k < 2:
            edges = {name: np.zeros(0, dt) for name, dt in FIELDS}
        return merge(k, edges)
    finally:
        if fam is not None:
            fam.free()
