"""Multi-GPU form of the hot path: the iterative scheme sharded by packet id,
the ray tracer and its adjoint sharded by camera.  One process per GPU.

Packets are independent (Sect. 3.4) and each packet's random stream is keyed
by its id, so an emission of N packets split into disjoint id ranges over R
ranks gives, after one sum over ranks of the accumulated outputs, the result
of one process running all N (up to the order of FP64 additions).  This holds
for the iterative scheme (Eq. 5 re-emission at the previous iteration's
temperatures, Eq. 4 between iterations): each iteration is one transport of
the rank's packet range, one sum all-reduce of the accumulators (E_abs,
absorption counts, sum of squared deposits, escaped SED, counters), then the
temperatures, identical on every rank.  Bjorkman & Wood couples packets
through the temperatures as they change, so it does not shard exactly.

The ray tracer (Sect. 4) needs every stored scattering event for every
camera: the ranks gather the events (in rank order, i.e. packet-id order),
then each traces its share of the cameras (round robin) and the images and
SEDs are assembled on every rank by a sum all-reduce of zero-padded arrays.
Its adjoint sums the per-camera density gradients over the ranks.

The drivers take a backend with the operations of one rank (``transport``,
``temperatures``, ``events``, ``raytrace``, ``raytrace_backward``):
``DeviceBackend`` runs them in the CUDA library; tests may pass any object
with the same methods.  Collectives go through torch.distributed (NCCL on
GPUs, gloo on CPU); with world = 1 no collective is issued.
"""
from __future__ import annotations

from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import torch

ACC_KEYS = ("E_abs", "count", "esq", "sed_esc", "sed_cnt", "stats")
EVENT_BYTES = 20


def packet_range(n_packets: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [begin, end) share of packet ids for `rank` of `world`."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    b = n_packets * rank // world
    e = n_packets * (rank + 1) // world
    return b, e


def cameras_of(n_cams: int, rank: int, world: int) -> List[int]:
    """Camera indices traced by `rank` (round robin)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    return list(range(rank, n_cams, world))


def _dist(world):
    if world == 1:
        return None
    import torch.distributed as dist
    return dist


def allreduce_sum(tensors: Iterable, group=None) -> None:
    """Sum accumulated outputs (E_abs, counts, SEDs, ...) over all ranks in place."""
    import torch.distributed as dist
    for t in tensors:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


def gather_events(events: Optional[torch.Tensor], world: int, group=None) -> Optional[torch.Tensor]:
    """Every rank's stored event records (uint8, EVENT_BYTES each),
    concatenated in rank order on every rank."""
    dist = _dist(world)
    if dist is None:
        return events
    dev = events.device if events is not None else torch.device("cpu")
    mine = events if events is not None else torch.zeros(0, dtype=torch.uint8, device=dev)
    n = torch.tensor([mine.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    mx = max(sizes)
    if mx == 0:
        return None
    pad = torch.zeros(mx, dtype=torch.uint8, device=dev)
    pad[:mine.numel()] = mine
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)])


def frozen_t_iterations(backend, T0: torch.Tensor, n_iter: int, n_packets: int, seed: int,
                        rank: int = 0, world: int = 1, group=None):
    """The iterative scheme sharded by packet id: n_iter iterations, each the
    transport of this rank's share of an n_packets emission at the previous
    temperatures (T0 first), the sum of the accumulators over the ranks and
    the Eq. 4 temperatures.  Returns (T, summed outputs of the last
    iteration, this rank's events of the last iteration)."""
    dist = _dist(world)
    T = T0
    out = None
    b, e = packet_range(n_packets, rank, world)
    for it in range(n_iter):
        out = backend.transport(T, b, e, n_packets, seed + it)
        if dist is not None:
            allreduce_sum([out[k] for k in ACC_KEYS if out.get(k) is not None], group)
        T = backend.temperatures(out["E_abs"])
    return T, out, backend.events()


def raytrace_views(backend, T, events, cams: Sequence, rank: int = 0, world: int = 1, group=None):
    """Images and SEDs of every camera, each rank tracing its share; the
    arrays are assembled on every rank."""
    dist = _dist(world)
    mine = cameras_of(len(cams), rank, world)
    if dist is None:
        return backend.raytrace(T, events, list(cams))
    img_m, sed_m = backend.raytrace(T, events, [cams[i] for i in mine]) if mine else (None, None)
    shape_img, shape_sed = backend.image_shape(len(cams)), backend.sed_shape(len(cams))
    img = torch.zeros(shape_img, dtype=torch.float32, device=backend.device)
    sed = torch.zeros(shape_sed, dtype=torch.float64, device=backend.device)
    if mine:
        img[mine] = img_m
        sed[mine] = sed_m
    allreduce_sum([img, sed], group)
    return img, sed


def raytrace_views_backward(backend, T, events, cams: Sequence, dL_dimg, dL_dsed, rank: int = 0,
                            world: int = 1, group=None):
    """d(loss)/d(rho) and d(loss)/d(scale) of a loss over every camera's
    images and SEDs (upstream gradients for all cameras on every rank): each
    rank takes its cameras' share and the gradients are summed."""
    dist = _dist(world)
    mine = cameras_of(len(cams), rank, world)
    if dist is None:
        return backend.raytrace_backward(T, events, list(cams), dL_dimg, dL_dsed)
    if mine:
        gi = None if dL_dimg is None else dL_dimg[mine]
        gs = None if dL_dsed is None else dL_dsed[mine]
        drho, dscale = backend.raytrace_backward(T, events, [cams[i] for i in mine], gi, gs)
    else:
        drho, dscale = backend.zero_gradient()
    allreduce_sum([drho, dscale], group)
    return drho, dscale


class DeviceBackend:
    """One rank's operations in the CUDA library: transport of a packet-id
    range in the frozen-T mode into reused device buffers, temperatures, the
    stored events, ray tracing of a camera subset and its adjoint."""

    def __init__(self, ctx, grid, opac, sources, freq_idx: Sequence[int], npix: int,
                 event_cap: int = 0, stream=None, **transport_kw):
        from . import rtgb as R
        from .sim import TransportOut
        self.ctx, self.grid, self.opac, self.sources = ctx, grid, opac, sources
        self.freq_idx = list(freq_idx)
        self.npix = npix
        self.stream = stream
        self.kw = dict(transport_kw)
        self.out = TransportOut(grid.ncell, grid.ns, opac.nf, event_cap=event_cap)
        self.device = self.out.E_abs.device
        self.xi = None
        self._R = R

    def transport(self, T_prev, pid_begin, pid_end, n_packets, seed) -> Dict[str, torch.Tensor]:
        from .sim import transport
        o = self.out.zero_()
        transport(self.ctx, self.grid, self.opac, self.sources, n_packets, out=o, T_prev=T_prev,
                  mode=self._R.RT_MODE_FROZEN_T, pid_begin=pid_begin, pid_end=pid_end, seed=seed,
                  stream=self.stream, **self.kw)
        self.xi = o.xi
        return {"E_abs": o.E_abs, "count": o.count, "esq": o.esq, "sed_esc": o.sed_esc,
                "sed_cnt": o.sed_cnt, "stats": o.stats}

    def temperatures(self, E_abs):
        from .sim import temperatures
        return temperatures(self.ctx, self.grid, self.opac, E_abs, stream=self.stream)

    def events(self) -> Optional[torch.Tensor]:
        n = min(int(self.out.stats[13].item()), self.out.event_cap)
        return self.out.events[:n * EVENT_BYTES] if n else None

    def image_shape(self, n_cams):
        return (n_cams, len(self.freq_idx), self.npix, self.npix)

    def sed_shape(self, n_cams):
        return (n_cams, len(self.freq_idx))

    def raytrace(self, T, events, cams):
        from .sim import raytrace
        return raytrace(self.ctx, self.grid, self.opac, T, events, self.xi or 0.0, self.sources, cams,
                        self.freq_idx, stream=self.stream)

    def raytrace_backward(self, T, events, cams, dL_dimg, dL_dsed):
        from .sim import raytrace_backward
        return raytrace_backward(self.ctx, self.grid, self.opac, T, events, self.xi or 0.0,
                                 self.sources, cams, self.freq_idx, dL_dimg=dL_dimg, dL_dsed=dL_dsed,
                                 stream=self.stream)

    def zero_gradient(self):
        return (torch.zeros((self.grid.ns, self.grid.ncell), dtype=torch.float32, device=self.device),
                torch.zeros(1, dtype=torch.float64, device=self.device))
