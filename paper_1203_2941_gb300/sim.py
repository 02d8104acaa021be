"""Convenience layer over the C ABI: torch tensors own the device buffers,
torch streams carry the work, and every step runs in librtgb's kernels.

    ctx = Context()
    grid, opac, srcs = ctx.grid(model), ctx.opacity(model), Sources(model.sources)
    out = transport(ctx, grid, opac, srcs, n_packets=10**7)
    T = temperatures(ctx, grid, opac, out.E_abs)
    img, sed = raytrace(ctx, grid, opac, T, out, srcs, cams, freq_idx)
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import rtgb as R


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


class Context:
    """A library context on one CUDA device."""

    def __init__(self, device: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("rtgb needs a CUDA GPU; none is visible")
        R.load()
        torch.cuda.set_device(device)
        self.device = device
        self.h = R.rt_ctx_create(device)

    def close(self):
        if getattr(self, "h", None):
            R.rt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def grid(self, model, stream=None) -> "Grid":
        return Grid(self, model.rho, model.box_min, model.cell, stream,
                    refine=getattr(model, "refine", 0), refined=getattr(model, "refined", None))

    def opacity(self, model) -> "Opacity":
        return Opacity(self, model.nu, model.dnu, model.kabs, model.ksca, model.g, model.is_pah)


class Grid:
    """Density grid on the device.  Uniform: rho [ns, nz, ny, nx].  One level
    of refinement: ``refine`` = r and ``refined`` [nz, ny, nx] (nonzero =
    divided cube) with rho [ns, ncell] in the library's cell numbering."""

    def __init__(self, ctx: Context, rho, box_min, cell, stream=None, refine: int = 0,
                 refined=None):
        self.ctx = ctx
        if isinstance(rho, torch.Tensor):
            t = rho.detach().to(dtype=torch.float32).contiguous()
        else:
            t = torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32))
        self.box_min = [float(v) for v in box_min]
        self.cell = float(cell)
        self.refine = int(refine or 0)
        self._src = t           # keep alive until the copy finished (upload syncs)
        if self.refine:
            mask = np.ascontiguousarray(refined, dtype=np.uint8)
            nz, ny, nx = mask.shape
            ns = t.shape[0]
            self.h = R.rt_grid_upload_refined(ctx.h, nx, ny, nz, ns, self.box_min, self.cell,
                                              self.refine, mask.ctypes.data_as(C.c_void_p),
                                              t.data_ptr(), _stream(stream))
            self.ncell = R.rt_grid_ncell(self.h)
            if t.shape != (ns, self.ncell):
                R.rt_grid_free(self.h)
                self.h = None
                raise ValueError(f"refined grid needs rho of shape ({ns}, {self.ncell})")
        else:
            ns, nz, ny, nx = t.shape
            self.h = R.rt_grid_upload(ctx.h, nx, ny, nz, ns, self.box_min, self.cell, t.data_ptr(),
                                      _stream(stream))
            self.ncell = nx * ny * nz
        self.shape = (nx, ny, nz)
        self.ns = ns
        self._src = None

    def update(self, rho, stream=None) -> "Grid":
        """New densities of the same shape (host or device), copied into the
        grid's own buffer (no allocation); checked synchronously."""
        if isinstance(rho, torch.Tensor):
            t = rho.detach().to(dtype=torch.float32).contiguous()
        else:
            t = torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32))
        if t.numel() != self.ns * self.ncell:
            raise ValueError(f"density needs {self.ns * self.ncell} values, got {t.numel()}")
        R.rt_grid_update(self.h, t.data_ptr(), _stream(stream))
        return self

    def __del__(self):
        try:
            if self.h:
                R.rt_grid_free(self.h)
                self.h = None
        except Exception:
            pass


class Opacity:
    def __init__(self, ctx: Context, nu, dnu, kabs, ksca, g, is_pah=None):
        self.ctx = ctx
        self.nu = np.asarray(nu, dtype=np.float64)
        self.nf = self.nu.size
        self.ns = np.atleast_2d(kabs).shape[0]
        self.h = R.rt_opacity_upload(ctx.h, nu, dnu, np.atleast_2d(kabs), np.atleast_2d(ksca),
                                     np.atleast_2d(g), is_pah)

    def __del__(self):
        try:
            if self.h:
                R.rt_opacity_free(self.h)
                self.h = None
        except Exception:
            pass


class Sources:
    """rt_source array built from workloads.Source objects (keeps L_nu alive)."""

    def __init__(self, sources):
        self._lnu = []
        arr = (R.rt_source * len(sources))()
        for i, s in enumerate(sources):
            lnu = None if s.L_nu is None else np.ascontiguousarray(s.L_nu, dtype=np.float64)
            self._lnu.append(lnu)
            arr[i].pos = (C.c_double * 3)(*[float(v) for v in s.pos])
            arr[i].L = float(s.L)
            arr[i].T_eff = float(s.T_eff)
            arr[i].L_nu = None if lnu is None else lnu.ctypes.data
        self.arr = arr
        self.n = len(sources)
        self.L = float(sum(s.L for s in sources))


class TransportOut:
    """Device outputs of rt_transport (accumulated across calls)."""

    def __init__(self, ncell: int, ns: int, nf: int, event_cap: int = 0, pah_cap: int = 0,
                 traj_cap: int = 0, esq: bool = True, device=None):
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.E_abs = torch.zeros((ns, ncell), dtype=torch.float64, device=dev)
        self.count = torch.zeros((ns, ncell), dtype=torch.int32, device=dev)
        self.esq = torch.zeros((ns, ncell), dtype=torch.float64, device=dev) if esq else None
        self.sed_esc = torch.zeros((10, nf), dtype=torch.float64, device=dev)
        self.sed_cnt = torch.zeros((10, nf), dtype=torch.int64, device=dev)
        self.events = torch.zeros(max(event_cap, 1) * 20, dtype=torch.uint8, device=dev)
        self.event_cap = event_cap
        self.pah = torch.zeros(max(pah_cap, 1) * 8, dtype=torch.uint8, device=dev)
        self.pah_cap = pah_cap
        self.traj = torch.zeros(max(traj_cap, 1) * 72, dtype=torch.uint8, device=dev)
        self.traj_cap = traj_cap
        self.stats = torch.zeros(R.RT_STAT_COUNT, dtype=torch.int64, device=dev)
        self.xi = None
        self.nf = nf
        self.pc_npix: List[int] = []
        self.pc_img = None           # flat: one [nf, npix, npix] block per camera

    def zero_(self):
        for t in (self.E_abs, self.count, self.esq, self.sed_esc, self.sed_cnt, self.stats,
                  self.pc_img):
            if t is not None:
                t.zero_()
        return self

    def ensure_pc(self, cams) -> None:
        """Allocate (once) the photon-counting images of ``cams``."""
        npix = [int(c.npix) for c in cams]
        if self.pc_img is not None and npix == self.pc_npix:
            return
        if self.pc_img is not None:
            raise ValueError("TransportOut already holds images of other photon-counting cameras")
        self.pc_npix = npix
        self.pc_img = torch.zeros(sum(self.nf * n * n for n in npix), dtype=torch.float64,
                                  device=self.E_abs.device)

    def pc_images(self) -> List[torch.Tensor]:
        """Photon-counting images, one [nf, npix, npix] view per camera."""
        out, o = [], 0
        for n in self.pc_npix:
            out.append(self.pc_img[o:o + self.nf * n * n].view(self.nf, n, n))
            o += self.nf * n * n
        return out

    def c_struct(self) -> R.rt_transport_out:
        return R.rt_transport_out(
            _ptr(self.E_abs), _ptr(self.count), _ptr(self.esq), _ptr(self.sed_esc),
            _ptr(self.sed_cnt),
            _ptr(self.events) if self.event_cap else None, self.event_cap,
            _ptr(self.pah) if self.pah_cap else None, self.pah_cap,
            _ptr(self.traj) if self.traj_cap else None, self.traj_cap,
            _ptr(self.stats), _ptr(self.pc_img))

    def stats_dict(self):
        v = self.stats.cpu().numpy()
        return {k: int(v[i]) for i, k in enumerate(R.STAT_NAMES)}

    @property
    def n_events(self):
        return int(min(self.stats[13].item(), self.event_cap))

    def events_numpy(self):
        n = self.n_events
        return self.events[:n * 20].cpu().numpy().view(R.EVENT_DTYPE)

    def pah_numpy(self):
        n = int(min(self.stats[14].item(), self.pah_cap))
        return self.pah[:n * 8].cpu().numpy().view(R.PAH_DTYPE)

    def traj_numpy(self):
        n = int(min(self.stats[15].item(), self.traj_cap))
        return self.traj[:n * 72].cpu().numpy().view(R.TRAJ_DTYPE)

    def numpy(self):
        return dict(E_abs=self.E_abs.cpu().numpy(),
                    count=self.count.cpu().numpy().view(np.uint32),
                    esq=None if self.esq is None else self.esq.cpu().numpy(),
                    sed_esc=self.sed_esc.cpu().numpy(),
                    sed_cnt=self.sed_cnt.cpu().numpy().view(np.uint64),
                    stats=self.stats_dict(), xi=self.xi)


def make_params(n_packets: int, mode=R.RT_MODE_BW, lucy_mode=R.RT_LUCY_THIN,
                lucy_form=R.RT_LUCY_LINEAR, lucy_tau=1e-2, mrw=False, mrw_tau_cell=10.0,
                mrw_gamma=2.0, seed=1, model_id=0, pid_begin=0, pid_end=None,
                max_events=10_000_000, record_events=False, precision=R.RT_PREC_FP32,
                schedule=R.RT_SCHED_PERSISTENT, threads_per_block=0, blocks_per_sm=0,
                march_min_active=-1, defer_events=0, source_bins=0,
                record_nu=None, compact_swap=-1, source_grid=None) -> R.rt_transport_params:
    """Transport parameters; ``record_nu`` lists the frequency bins whose
    scattering events are stored (None: every bin); ``source_grid`` is the
    (model bin, source) table pair of ``source_grid()`` for source_bins."""
    p = R.rt_transport_params_default()
    p.mode, p.lucy_mode, p.lucy_form, p.lucy_tau = mode, lucy_mode, lucy_form, lucy_tau
    p.mrw, p.mrw_tau_cell, p.mrw_gamma = int(bool(mrw)), mrw_tau_cell, mrw_gamma
    p.seed, p.model_id = int(seed), int(model_id)
    p.n_packets = int(n_packets)
    p.pid_begin = int(pid_begin)
    p.pid_end = int(n_packets if pid_end is None else pid_end)
    p.max_events = int(max_events)
    p.record_events = int(bool(record_events))
    p.precision, p.schedule = precision, schedule
    p.threads_per_block, p.blocks_per_sm = threads_per_block, blocks_per_sm
    p.march_min_active = march_min_active
    p.defer_events = int(defer_events)
    p.source_bins = int(source_bins)
    p.compact_swap = int(compact_swap)
    if source_grid is not None:
        nu_t = np.ascontiguousarray(source_grid[0], dtype=np.int32)
        src_t = np.ascontiguousarray(source_grid[1], dtype=np.int32)
        if len(nu_t) != int(source_bins) or len(src_t) != int(source_bins):
            raise ValueError("source_grid tables need source_bins entries each")
        p._source_grid = (nu_t, src_t)              # kept alive with the struct
        p.source_grid_nu = nu_t.ctypes.data_as(C.c_void_p)
        p.source_grid_src = src_t.ctypes.data_as(C.c_void_p)
    if record_nu is not None:
        idx = [int(j) for j in record_nu]
        words = (C.c_uint32 * max(1, (max(idx, default=0) // 32) + 1))()
        for j in idx:
            words[j // 32] |= 1 << (j % 32)
        p._record_nu_words = words            # kept alive with the struct
        p.record_nu_mask = C.cast(words, C.c_void_p)
    return p


@dataclass
class PcCamera:
    """Photon-counting camera (Sect. 4): packets leaving the grid with
    k . k_obs >= cos_accept are counted in the pixel of their projected exit
    point; pixel 0 means box diagonal / npix."""
    theta: float
    phi: float
    npix: int
    cos_accept: float
    pixel: float = 0.0


def pc_cameras(cams) -> "C.Array":
    arr = (R.rt_pc_camera * max(1, len(cams)))()
    for i, c in enumerate(cams):
        arr[i].theta, arr[i].phi, arr[i].npix = float(c.theta), float(c.phi), int(c.npix)
        arr[i].pixel, arr[i].cos_accept = float(c.pixel), float(c.cos_accept)
    return arr


def transport(ctx: Context, grid: Grid, opac: Opacity, sources: Sources, n_packets: int,
              out: Optional[TransportOut] = None, T_prev: Optional[torch.Tensor] = None,
              event_cap: int = 0, pah_cap: int = 0, traj_cap: int = 0, stream=None,
              pc_cams: Sequence[PcCamera] = (), **kw) -> TransportOut:
    """One rt_transport call; ``pc_cams`` adds photon-counting images
    (``out.pc_images()``)."""
    if out is None:
        out = TransportOut(grid.ncell, grid.ns, opac.nf, event_cap, pah_cap, traj_cap)
    if kw.get("record_events") is None and out.event_cap:
        kw["record_events"] = True
    p = make_params(n_packets, **kw)
    pca = None
    if pc_cams:
        out.ensure_pc(pc_cams)
        pca = pc_cameras(pc_cams)
        p.pc_cams, p.n_pc_cams = C.cast(pca, C.c_void_p), len(pc_cams)
    if T_prev is not None:
        T_prev = T_prev.to(dtype=torch.float64).contiguous()
    R.rt_transport(ctx.h, grid.h, opac.h, sources.arr, sources.n, p, _ptr(T_prev),
                   out.c_struct(), _stream(stream))
    out.xi = sources.L / n_packets
    return out


def _pah_records(records):
    """Stored PAH absorptions as a device uint8 tensor (8 bytes each) and
    their count."""
    if isinstance(records, TransportOut):
        n = int(min(records.stats[14].item(), records.pah_cap))
        return records.pah, n
    if isinstance(records, np.ndarray):
        rec = np.zeros(len(records), R.PAH_DTYPE)
        rec["cell"] = records["cell"]
        if len(rec) == 0:
            return None, 0
        return torch.from_numpy(rec.view(np.uint8).copy()).cuda(), len(rec)
    raise TypeError("records must be a TransportOut or a numpy PAH record array")


def pah_reemit(ctx: Context, grid: Grid, opac: Opacity, records, xi: float, eps,
               eps_class: Optional[torch.Tensor] = None, out: Optional[TransportOut] = None,
               T_prev: Optional[torch.Tensor] = None, event_cap: int = 0, pah_cap: int = 0,
               traj_cap: int = 0, stream=None, pc_cams: Sequence[PcCamera] = (),
               **kw) -> TransportOut:
    """PAH re-emission pass (rt_pah_reemit): one packet of energy ``xi`` per
    stored PAH absorption of ``records`` (a TransportOut of an earlier pass
    or a numpy record array), bins drawn from ``eps`` [n_eps][nf] by the
    cells' ``eps_class`` (device int32 [ncell] or None).  Results accumulate
    into ``out`` (a new TransportOut by default; its PAH buffer receives this
    pass's PAH absorptions and must not be the records' buffer)."""
    rec, n = _pah_records(records)
    if out is None:
        out = TransportOut(grid.ncell, grid.ns, opac.nf, event_cap, pah_cap, traj_cap)
    if isinstance(records, TransportOut) and records is out:
        raise ValueError("the pass's output must not hold its own input records")
    out.xi = float(xi)
    if n == 0:
        return out
    if kw.get("record_events") is None and out.event_cap:
        kw["record_events"] = True
    p = make_params(n, **kw)
    pca = None
    if pc_cams:
        out.ensure_pc(pc_cams)
        pca = pc_cameras(pc_cams)
        p.pc_cams, p.n_pc_cams = C.cast(pca, C.c_void_p), len(pc_cams)
    e = np.ascontiguousarray(eps, dtype=np.float64).reshape(-1, opac.nf)
    cls = None
    if eps_class is not None:
        cls = torch.as_tensor(eps_class, dtype=torch.int32, device="cuda").contiguous()
    if T_prev is not None:
        T_prev = T_prev.to(dtype=torch.float64).contiguous()
    R.rt_pah_reemit(ctx.h, grid.h, opac.h, _ptr(rec), n, float(xi),
                    e.ctypes.data_as(C.c_void_p), e.shape[0], _ptr(cls), p, _ptr(T_prev),
                    out.c_struct(), _stream(stream))
    return out


def temperatures(ctx: Context, grid: Grid, opac: Opacity, E_abs: torch.Tensor,
                 T: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    E_abs = E_abs.contiguous()
    if T is None:
        T = torch.empty_like(E_abs, dtype=torch.float64)
    R.rt_temperatures(ctx.h, grid.h, opac.h, _ptr(E_abs), _ptr(T), _stream(stream))
    return T


def temperature_guess(ctx: Context, grid: Grid, sources: Sources, stream=None) -> torch.Tensor:
    T = torch.empty((grid.ns, grid.ncell), dtype=torch.float64, device="cuda")
    R.rt_temperature_guess(ctx.h, grid.h, sources.arr, sources.n, _ptr(T), _stream(stream))
    return T


def cameras(cams) -> "C.Array":
    arr = (R.rt_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].theta, arr[i].phi, arr[i].npix = float(c.theta), float(c.phi), int(c.npix)
        arr[i].D, arr[i].pixel = float(c.D), float(c.pixel)
    return arr


def _events_tensor(events):
    """Events as a device uint8 tensor (20 bytes each), their count (or the
    buffer capacity) and the address of a device-side count (or None).  A
    TransportOut passes its event cursor in device memory, so no host copy of
    the count (and no stream synchronisation) is needed."""
    if events is None:
        return None, 0, None
    if isinstance(events, TransportOut):
        return events.events, events.event_cap, events.stats.data_ptr() + 8 * 13
    if isinstance(events, torch.Tensor):
        # device event records (uint8, 20 bytes each), e.g. gathered from several ranks
        if events.dtype != torch.uint8 or events.numel() % 20 or not events.is_cuda:
            raise TypeError("device events must be a CUDA uint8 tensor of 20-byte records")
        n = events.numel() // 20
        return (events.contiguous(), n, None) if n else (None, 0, None)
    if isinstance(events, np.ndarray):
        if events.dtype != R.EVENT_DTYPE:
            ev = np.zeros(len(events), R.EVENT_DTYPE)
            ev["cell"] = events["cell"]; ev["nu"] = events["nu"]; ev["species"] = events["species"]
            ev["k"] = events["k"]
            events = ev
        if len(events) == 0:
            return None, 0, None
        t = torch.from_numpy(np.ascontiguousarray(events).view(np.uint8).copy()).cuda()
        return t, len(events), None
    raise TypeError("events must be a TransportOut, a numpy event array or a device record tensor")


def raytrace(ctx: Context, grid: Grid, opac: Opacity, T: torch.Tensor, events, xi_ev: float,
             sources: Optional[Sources], cams, freq_idx: Sequence[int], stream=None,
             steps: Optional[torch.Tensor] = None):
    """Images [n_cams, n_f, npix, npix] (float32) and SED [n_cams, n_f] (float64);
    ``steps`` (int64 device tensor of one element) accumulates ray-cell steps."""
    ev, nev, nev_dev = _events_tensor(events)
    ca = cameras(cams)
    fi = (C.c_int * len(freq_idx))(*[int(f) for f in freq_idx])
    npix = cams[0].npix
    img = torch.empty((len(cams), len(freq_idx), npix, npix), dtype=torch.float32, device="cuda")
    sed = torch.empty((len(cams), len(freq_idx)), dtype=torch.float64, device="cuda")
    T = T.to(dtype=torch.float64).contiguous()
    R.rt_raytrace(ctx.h, grid.h, opac.h, _ptr(T), _ptr(ev), nev, nev_dev, float(xi_ev),
                  None if sources is None else sources.arr, 0 if sources is None else sources.n,
                  ca, len(cams), fi, len(freq_idx), _ptr(img), _ptr(sed), _ptr(steps),
                  _stream(stream))
    return img, sed


def visibilities(ctx: Context, grid: Grid, cams, images: torch.Tensor, uv, stream=None) -> torch.Tensor:
    """Complex visibilities [n_cams, n_f, n_uv] (complex128) of images from
    ``raytrace`` at ``uv`` ([n_uv, 2], cycles per radian along the image axes)."""
    ca = cameras(cams)
    uv = np.ascontiguousarray(np.asarray(uv, dtype=np.float64).reshape(-1, 2))
    images = images.to(dtype=torch.float32).contiguous()
    ncam, nf = images.shape[0], images.shape[1]
    vis = torch.empty((ncam, nf, len(uv), 2), dtype=torch.float64, device="cuda")
    R.rt_visibilities(ctx.h, grid.h, ca, len(cams), _ptr(images), nf,
                      uv.ctypes.data_as(C.c_void_p), len(uv), _ptr(vis), _stream(stream))
    return torch.view_as_complex(vis)


def raytrace_backward(ctx: Context, grid: Grid, opac: Opacity, T: torch.Tensor, events, xi_ev,
                      sources: Optional[Sources], cams, freq_idx, dL_dimg=None, dL_dsed=None,
                      stream=None, steps: Optional[torch.Tensor] = None):
    """dL/drho [ns, ncell] (float32) and dL/dscale (float64 scalar tensor)."""
    ev, nev, nev_dev = _events_tensor(events)
    ca = cameras(cams)
    fi = (C.c_int * len(freq_idx))(*[int(f) for f in freq_idx])
    drho = torch.zeros((grid.ns, grid.ncell), dtype=torch.float32, device="cuda")
    dscale = torch.zeros(1, dtype=torch.float64, device="cuda")
    T = T.to(dtype=torch.float64).contiguous()
    gi = None if dL_dimg is None else dL_dimg.to(dtype=torch.float32).contiguous()
    gs = None if dL_dsed is None else dL_dsed.to(dtype=torch.float64).contiguous()
    R.rt_raytrace_backward(ctx.h, grid.h, opac.h, _ptr(T), _ptr(ev), nev, nev_dev, float(xi_ev),
                           None if sources is None else sources.arr,
                           0 if sources is None else sources.n, ca, len(cams), fi, len(freq_idx),
                           _ptr(gi), _ptr(gs), _ptr(drho), _ptr(dscale), _ptr(steps),
                           _stream(stream))
    return drho, dscale


class RayTrace(torch.autograd.Function):
    """Differentiable ray tracer: (rho, scale) -> (images, sed) with the
    density scale * rho; temperatures and scattering events held fixed.
    Refined grids: pass ``refine`` and ``refined`` after ``freq_idx``."""

    @staticmethod
    def forward(fctx, rho, scale, ctx, box_min, cell, opac, T, events, xi_ev, sources, cams, freq_idx,
                refine=0, refined=None):
        dens = (rho * scale).detach().contiguous()
        grid = Grid(ctx, dens, box_min, cell, refine=refine, refined=refined)
        img, sed = raytrace(ctx, grid, opac, T, events, xi_ev, sources, cams, freq_idx)
        fctx.save_for_backward(rho, scale)
        fctx.stuff = (ctx, grid, opac, T, events, xi_ev, sources, cams, freq_idx)
        return img, sed

    @staticmethod
    def backward(fctx, g_img, g_sed):
        rho, scale = fctx.saved_tensors
        ctx, grid, opac, T, events, xi_ev, sources, cams, freq_idx = fctx.stuff
        drho_eff, dscale_eff = raytrace_backward(ctx, grid, opac, T, events, xi_ev, sources, cams,
                                                 freq_idx, g_img, g_sed)
        drho = (drho_eff.view_as(rho) * scale).to(rho.dtype)
        dscale = (dscale_eff / scale.to(torch.float64)).to(scale.dtype).reshape(scale.shape)
        return drho, dscale, None, None, None, None, None, None, None, None, None, None, None, None


def philox(ctx: Context, ctr0, key, n: int, stream=None) -> np.ndarray:
    out = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    R.rt_philox(ctx.h, ctr0, key, n, _ptr(out), _stream(stream))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def source_grid(opac: Opacity, sources: Sources, m: int):
    """The separate source frequency grid of Eq. 1 (rt_source_grid): model
    bin index, source index and frequency (Hz) of each of m equal-energy bins."""
    nu = np.zeros(m, np.int32)
    src = np.zeros(m, np.int32)
    fr = np.zeros(m)
    R.rt_source_grid(opac.h, sources.arr, sources.n, int(m), nu.ctypes.data_as(C.c_void_p),
                     src.ctypes.data_as(C.c_void_p), fr.ctypes.data_as(C.c_void_p))
    return nu, src, fr


def mrw_sample(ctx: Context, opac, u, stream=None) -> np.ndarray:
    """The FP32 transport's MRW first-passage times y for uniforms u in (0, 1]."""
    ut = torch.as_tensor(np.ascontiguousarray(u, dtype=np.float32)).to("cuda")
    y = torch.empty_like(ut)
    R.rt_mrw_sample(ctx.h, opac.h, _ptr(ut), ut.numel(), _ptr(y), _stream(stream))
    torch.cuda.synchronize()
    return y.cpu().numpy()


class Batch:
    """Many models in one persistent launch (rt_batch_*); run() is graph-capturable."""

    def __init__(self, ctx: Context, opac: Opacity, models, n_packets: Sequence[int], event_cap=0,
                 pah_cap=0, T_prev=None, **kw):
        self.ctx, self.opac = ctx, opac
        self.grids = [ctx.grid(m) for m in models]
        self.sources = [Sources(m.sources) for m in models]
        self.outs = [TransportOut(g.ncell, g.ns, opac.nf, event_cap, pah_cap) for g in self.grids]
        self.T_prev = T_prev
        arr = (R.rt_model * len(models))()
        for i, (g, s, o) in enumerate(zip(self.grids, self.sources, self.outs)):
            arr[i].grid = g.h
            arr[i].sources = C.cast(s.arr, C.c_void_p)
            arr[i].n_sources = s.n
            arr[i].n_packets = int(n_packets[i])
            arr[i].T_prev = None if T_prev is None else _ptr(T_prev[i])
            arr[i].out = o.c_struct()
        self.models = arr
        self.params = make_params(1, **kw)
        self.h = R.rt_batch_create(ctx.h, opac.h, len(models), arr, self.params)

    def run(self, stream=None):
        R.rt_batch_run(self.h, _stream(stream))

    def __del__(self):
        try:
            if self.h:
                R.rt_batch_free(self.h)
                self.h = None
        except Exception:
            pass
