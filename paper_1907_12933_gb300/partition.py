"""One query split across ranks: contiguous slices of the index space and the
exchange step that merges the ranks' partial results.

The points of a box are independent (Eq. 10 holds or fails at each point by
itself; a sign change or an SS-Cover pair of Sec. III-B is set by some point or
not), so [0, R^s) splits into contiguous slices, one per rank, and the whole
query's result is a merge of the slices' results:

    adversarial count, tie count, points checked    sum
    first witness (smallest adversarial index)      min
    sign-change, SS-Cover masks and their ties      bitwise or
    verdict bitmap                                  bitwise or (slices are
                                                    32-aligned, so the words
                                                    of different ranks are
                                                    disjoint)
    tie indices                                     concatenation, sorted

Class D and the base margin come from the unperturbed image, the same on every
rank. The exchange uses torch.distributed collectives only (all_reduce SUM and
MIN, all_gather), so it runs on NCCL between GPUs and on gloo between CPU
processes alike.
"""
from __future__ import annotations

NO_WITNESS = 2**64 - 1
_NONE64 = 2**63 - 1  # "no witness" inside an int64 collective


def rank_range(n: int, rank: int, world: int, align: int = 32) -> tuple[int, int]:
    """Contiguous slice [lo, hi) of [0, n) for `rank` of `world`; every boundary
    but the last is a multiple of `align` (verdict-bitmap words stay whole)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the world")
    units = -(-n // align)
    lo = min(n, align * ((units * rank) // world))
    hi = n if rank == world - 1 else min(n, align * ((units * (rank + 1)) // world))
    return lo, hi


def merge_partials(part: dict, group=None, device=None) -> dict:
    """Merge one rank's partial result of a split query with the others'.

    part: n_points, n_adv, n_ties (ints), first_witness (int or None), D,
    base_margin, and optionally the coverage masks flip, flip_tie, ss, ss_tie
    and the verdict bitmap (numpy uint32 words, the same length on every rank)
    and ties (numpy int64 indices). Returns the merged dict in the same form
    (ties sorted, first_witness None when no rank found one). Every rank
    receives the merged result."""
    import numpy as np
    import torch
    import torch.distributed as dist

    dev = torch.device("cpu") if device is None else torch.device(device)
    out = dict(part)
    cnt = torch.tensor([int(part["n_points"]), int(part["n_adv"]), int(part["n_ties"])],
                       dtype=torch.int64, device=dev)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM, group=group)
    fw = part.get("first_witness")
    first = torch.tensor([_NONE64 if fw is None else int(fw)], dtype=torch.int64, device=dev)
    dist.all_reduce(first, op=dist.ReduceOp.MIN, group=group)
    out["n_points"], out["n_adv"], out["n_ties"] = (int(x) for x in cnt.tolist())
    f = int(first.item())
    out["first_witness"] = None if f == _NONE64 else f
    world = dist.get_world_size(group)

    def gather_or(words):
        t = torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint32).view(np.int32)).to(dev)
        bufs = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(bufs, t, group=group)
        acc = bufs[0].clone()
        for b in bufs[1:]:
            acc = torch.bitwise_or(acc, b)
        return acc.cpu().numpy().view(np.uint32)

    for key in ("flip", "flip_tie", "ss", "ss_tie", "bitmap"):
        if part.get(key) is not None:
            out[key] = gather_or(part[key])
    if part.get("ties") is not None:
        mine = np.ascontiguousarray(part["ties"], dtype=np.int64)
        n = torch.tensor([mine.size], dtype=torch.int64, device=dev)
        ns = [torch.empty_like(n) for _ in range(world)]
        dist.all_gather(ns, n, group=group)
        cap = max(1, max(int(x.item()) for x in ns))
        pad = torch.full((cap,), -1, dtype=torch.int64, device=dev)
        pad[:mine.size] = torch.from_numpy(mine).to(dev)
        bufs = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(bufs, pad, group=group)
        allt = np.concatenate([b.cpu().numpy()[:int(c.item())] for b, c in zip(bufs, ns)])
        out["ties"] = np.sort(allt)
    return out


def merged_verdict(m: dict, whole: bool = True) -> str:
    """Verdict of a merged result (the whole box checked unless whole is False)."""
    if not whole:
        return "PARTIAL"
    if m["n_adv"]:
        return "UNSAFE"
    return "TIES_ONLY" if m["n_ties"] else "SAFE"
