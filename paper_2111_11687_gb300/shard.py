"""Sharding one Monte Carlo run over ranks (one process per GPU).

Histories are independent and a history's random numbers depend only on the
seed and its id (Philox4x32-10 keyed by both, §2.1's histories), so a run of
n histories splits into contiguous id ranges, one per rank, that run with no
exchange at all.  The run's one exchange step is the merge of the ranks'
statistics at the end: the integer tallies add exactly, so the merged tally is
bit-identical to one device running every range in turn.
"""
from __future__ import annotations


def history_range(n_total: int, world_size: int, rank: int) -> tuple[int, int]:
    """(first id, count) of ``rank``'s contiguous share of ids [0, n_total).

    The first ``n_total % world_size`` ranks take one history more; the
    ranges are disjoint and cover every id once.
    """
    if world_size < 1 or not 0 <= rank < world_size or n_total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(int(n_total), int(world_size))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def gather_images(image, dst: int = 0, group=None):
    """Gathers every rank's checkpoint image (a flat uint8 tensor, equal sizes
    on all ranks: same grid and options) onto rank ``dst``.

    Returns the list of images, indexed by rank, on ``dst`` and None
    elsewhere.  CPU tensors with gloo, device tensors with NCCL.
    """
    import torch
    import torch.distributed as dist

    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    size = torch.tensor([image.numel()], dtype=torch.int64, device=image.device)
    sizes = [torch.zeros_like(size) for _ in range(ws)]
    dist.all_gather(sizes, size, group=group)
    if any(int(s.item()) != image.numel() for s in sizes):
        raise ValueError("checkpoint images differ in size between ranks")
    if rank == dst:
        out = [torch.empty_like(image) for _ in range(ws)]
        dist.gather(image, out, dst=dst, group=group)
        return out
    dist.gather(image, None, dst=dst, group=group)
    return None


def sharded_run(dose, n_total: int, seed: int, dst: int = 0, group=None) -> bool:
    """Runs this rank's share of ``n_total`` histories on ``dose`` (an
    ``nmdose.Dose`` on this rank's GPU), then merges every other rank's
    statistics into rank ``dst``'s handle.  Returns True on ``dst``, whose
    handle then holds the statistics of the whole run.
    """
    import torch
    import torch.distributed as dist

    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    first, n = history_range(n_total, ws, rank)
    dose.seek(first)
    dose.run(n, seed)
    size = dose.checkpoint_size()
    device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    image = dose.checkpoint(torch.empty(size, dtype=torch.uint8, device=device))
    images = gather_images(image, dst, group)
    if rank != dst:
        return False
    for r, im in enumerate(images):
        if r != dst:
            dose.merge(im)
    return True
