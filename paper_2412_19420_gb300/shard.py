"""One mine split over the ranks of a torch.distributed group.

Every rank holds the whole database, builds its bit matrix and mines its own
share of the prefix classes (``fim_mine_shard``: the paper's decomposition
into parts mined separately, Section II); the only exchange is the gather of
the parts on one rank, which merges them into the canonical answer
(``fim_merge_results``).  Nothing is exchanged while the GPUs mine.

The collective is plain ``torch.distributed`` point-to-point traffic: the
part sizes by ``all_gather``, then each rank's three arrays to the
destination with ``isend``/``irecv``.  It runs on NCCL between GPUs and on
gloo between CPU processes.
"""
from __future__ import annotations


def gather_parts(part, group=None, dst: int = 0):
    """Collect every rank's part -- (offsets, items, supports) tensors, all on
    the process group's device -- on rank ``dst``, in rank order.  Returns
    the list there and None on the other ranks."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    off, it, sup = part
    sizes = torch.tensor([off.shape[0], it.shape[0], sup.shape[0]], dtype=torch.int64, device=off.device)
    all_sizes = [torch.empty_like(sizes) for _ in range(world)]
    dist.all_gather(all_sizes, sizes, group=group)
    if rank != dst:
        reqs = [dist.isend(t.contiguous(), dst, group=group) for t in (off, it, sup) if t.numel()]
        for q in reqs:
            q.wait()
        return None
    parts, reqs = [], []
    for r in range(world):
        if r == rank:
            parts.append((off, it, sup))
            continue
        no, ni, ns = (int(v) for v in all_sizes[r].tolist())
        bufs = (torch.empty(no, dtype=off.dtype, device=off.device),
                torch.empty(ni, dtype=it.dtype, device=it.device),
                torch.empty(ns, dtype=sup.dtype, device=sup.device))
        reqs += [dist.irecv(b, r, group=group) for b in bufs if b.numel()]
        parts.append(bufs)
    for q in reqs:
        q.wait()
    return parts


def mine_sharded(ctx, indptr, indices, n_items: int, minsup: int, flags: int = 0, group=None, dst: int = 0,
                 api=None):
    """Mine one database split over the group's ranks; rank ``dst`` ends with
    the merged canonical itemsets held by its ctx (fetch them with
    ``fim_fetch_results``, derive rules with ``fim_rules``).  Returns the
    number of sets on ``dst`` and None elsewhere.  ``indptr``/``indices`` are
    the whole CSR on every rank (numpy or CUDA tensors); ``api`` replaces the
    library binding (tests)."""
    import torch
    import torch.distributed as dist

    if api is None:
        from . import fim as api
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n_trans = int(indptr.shape[0]) - 1
    api.fim_build_bitmaps(ctx, indptr, indices, n_items)
    api.fim_mine_shard(ctx, minsup, flags, rank, world)
    R, T = api.fim_result_sizes(ctx)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    out = (torch.empty(R + 1, dtype=torch.int64, device=dev), torch.empty(max(T, 1), dtype=torch.int32, device=dev),
           torch.empty(max(R, 1), dtype=torch.int32, device=dev))
    api.fim_fetch_results(ctx, out if dev != "cpu" else tuple(x.numpy() for x in out))
    parts = gather_parts((out[0], out[1][:T], out[2][:R]), group, dst)
    if rank != dst:
        return None
    if dev == "cpu":
        parts = [tuple(x.numpy() for x in p) for p in parts]
    api.fim_merge_results(ctx, n_trans, n_items, parts)
    return api.fim_result_sizes(ctx)[0]
