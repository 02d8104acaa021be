"""Packet-id sharding across processes.

Packets are independent (the paper's Sect. 3.4), and each packet's random
stream is keyed by its id, so an emission of N packets split into disjoint
id ranges over R ranks gives, after one sum over ranks of the accumulated
outputs, the same result as one process running all N (up to the order of
FP64 additions).  This is exact for the iterative (frozen-temperature)
scheme; Bjorkman & Wood couples packets through the temperatures, so ranks
run replicas instead and their outputs are averaged.
"""
from __future__ import annotations

from typing import Iterable, Tuple


def packet_range(n_packets: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [begin, end) share of packet ids for `rank` of `world`."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    b = n_packets * rank // world
    e = n_packets * (rank + 1) // world
    return b, e


def allreduce_sum(tensors: Iterable, group=None) -> None:
    """Sum accumulated outputs (E_abs, counts, SEDs, ...) over all ranks in place."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


def allreduce_mean(tensors: Iterable, group=None) -> None:
    """Average replica outputs over all ranks in place (Bjorkman & Wood)."""
    import torch.distributed as dist
    w = dist.get_world_size(group)
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        t.div_(w)
