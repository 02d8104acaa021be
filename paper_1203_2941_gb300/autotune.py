"""Schedule autotuner for the transport: picks the warp-scheduling parameters
of ``rt_transport`` / ``rt_batch`` (lanes still marching below which a warp
serves its pending interactions, threads per block, blocks per SM) by timing
candidates on a bounded packet sample of the caller's own workload.

The tuned parameters change only how packets are scheduled on the GPU, not
what is computed: every candidate runs the same packets with the same
Philox streams (results differ only through the order of the B&W
temperature updates, as between any two parallel runs).

    best = tune_transport(ctx, grid, opac, srcs, n_packets=10**7)
    out = transport(ctx, grid, opac, srcs, 10**7, **best.params)

    best = tune_batch(ctx, opac, models, [10**7] * len(models))
    b = Batch(ctx, opac, models, [10**7] * len(models), **best.params)
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

DEFAULT_GRID = {
    "march_min_active": (2, 4, 6, 8, 12, 16, 20, 24),
    "threads_per_block": (256, 128),
    "blocks_per_sm": (0,),
}


@dataclass
class TuneResult:
    params: Dict[str, int]
    seconds: float
    table: List[Tuple[Dict[str, int], float]] = field(default_factory=list)


def candidates(grid: Optional[Dict[str, Iterable[int]]] = None) -> List[Dict[str, int]]:
    """All combinations of the grid's values, in a fixed order."""
    g = dict(DEFAULT_GRID)
    if grid:
        g.update({k: tuple(v) for k, v in grid.items()})
    keys = sorted(g)
    return [dict(zip(keys, vals)) for vals in itertools.product(*(g[k] for k in keys))]


def select(cands: Sequence[Dict[str, int]], timer: Callable[[Dict[str, int]], float],
           repeats: int = 3) -> TuneResult:
    """Time each candidate ``repeats`` times (the timer returns seconds for
    one run) and keep the one with the smallest median; ties go to the
    earlier candidate."""
    if not cands:
        raise ValueError("no candidates")
    table = []
    best_i, best_t = 0, math.inf
    for i, c in enumerate(cands):
        ts = sorted(timer(c) for _ in range(max(1, repeats)))
        t = ts[len(ts) // 2]
        table.append((dict(c), t))
        if t < best_t:
            best_i, best_t = i, t
    return TuneResult(dict(cands[best_i]), best_t, table)


def _cuda_timer(run):
    import torch

    def timer(c):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run(c)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3
    return timer


def tune_transport(ctx, grid, opac, sources, n_packets: int, sample: int = 2_000_000,
                   grid_values: Optional[Dict[str, Iterable[int]]] = None, repeats: int = 3,
                   event_cap: int = 0, **kw) -> TuneResult:
    """Tune ``transport`` for one model on min(n_packets, sample) packets of
    the same emission (same xi = L / n_packets, same packet ids); with
    record_events in ``kw``, ``event_cap`` sizes the sample's event buffer
    (events beyond it are counted as dropped, as in any call)."""
    import torch

    from . import sim
    n = int(min(n_packets, sample))
    out = sim.TransportOut(grid.ncell, grid.ns, opac.nf, event_cap=int(event_cap))

    def run(c):
        out.zero_()
        out.stats.zero_()
        sim.transport(ctx, grid, opac, sources, int(n_packets), out=out, pid_end=n, **kw, **c)

    cands = candidates(grid_values)
    run(cands[0])                                     # warm-up (tables, packing)
    torch.cuda.synchronize()
    return select(cands, _cuda_timer(run), repeats)


def tune_batch(ctx, opac, models, n_packets: Sequence[int], sample: int = 200_000,
               grid_values: Optional[Dict[str, Iterable[int]]] = None, repeats: int = 2,
               **kw) -> TuneResult:
    """Tune a ``Batch`` of models on min(n_packets[m], sample) packets each."""
    import torch

    from . import sim
    n = [int(min(p, sample)) for p in n_packets]
    held = {}                      # one Batch (with its outputs) alive at a time

    def run(c):
        key = tuple(sorted(c.items()))
        if held.get("key") != key:
            held.clear()
            torch.cuda.synchronize()
            held["key"], held["b"] = key, sim.Batch(ctx, opac, models, n, **kw, **c)
        for o in held["b"].outs:
            o.zero_()
        held["b"].run()

    cands = candidates(grid_values)
    run(cands[0])
    torch.cuda.synchronize()
    return select(cands, _cuda_timer(run), repeats)
