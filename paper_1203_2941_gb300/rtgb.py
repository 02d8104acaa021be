"""Python binding of librtgb (argument marshalling only).

The ``rt_*`` functions mirror the C ABI in ``include/rtgb.h`` one to one and
take plain integers (device pointers, stream handles) or numpy arrays (host
data).  Every computation runs in the library's CUDA kernels; PyTorch is used
only by the convenience layer below to own device memory and streams.  If the
library is missing or no GPU is present, the calls raise instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(os.environ.get("RTGB_BUILD_DIR") or os.path.join(HERE, "_build"), "librtgb.so")

RT_OK, RT_ERR_INVALID_ARG, RT_ERR_CUDA, RT_ERR_OOM, RT_ERR_CAPACITY, RT_ERR_STUCK, RT_ERR_STATE = range(7)
RT_MODE_BW, RT_MODE_FROZEN_T, RT_MODE_NOREEMIT = 0, 1, 2
RT_LUCY_OFF, RT_LUCY_THIN, RT_LUCY_ALL = 0, 1, 2
RT_LUCY_LINEAR, RT_LUCY_EXPM1 = 0, 1
RT_PREC_FP32, RT_PREC_FP64, RT_PREC_FP32_ACC32 = 0, 1, 2
RT_SCHED_PERSISTENT, RT_SCHED_SERIAL, RT_SCHED_COMPACT = 0, 1, 2
STAT_NAMES = ["crossings", "interactions", "scatters", "absorptions", "mrw_steps", "escaped",
              "stuck", "pah", "events_dropped", "lucy_deposits", "emitted", "pah_dropped",
              "traj_dropped", "n_events", "n_pah", "n_traj", "deferred"]
RT_STAT_COUNT = 17
EXPORTS = ["rt_last_error", "rt_version", "rt_ctx_create", "rt_ctx_destroy", "rt_grid_upload",
           "rt_grid_free", "rt_opacity_upload", "rt_opacity_free", "rt_transport_params_default",
           "rt_transport", "rt_temperatures", "rt_temperature_guess", "rt_raytrace",
           "rt_raytrace_backward", "rt_batch_create", "rt_batch_run", "rt_batch_free",
           "rt_transport_batched", "rt_philox", "rt_mrw_sample", "rt_probe_gather", "rt_source_grid", "rt_kernel_launches", "rt_transport_noalloc", "rt_visibilities",
           "rt_pah_reemit", "rt_grid_upload_refined", "rt_grid_ncell", "rt_grid_update"]


class RtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rtgb error {code}: {msg}")
        self.code = code


class rt_source(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("L", C.c_double), ("T_eff", C.c_double),
                ("L_nu", C.c_void_p)]


class rt_transport_params(C.Structure):
    _fields_ = [("mode", C.c_int), ("lucy_mode", C.c_int), ("lucy_form", C.c_int),
                ("lucy_tau", C.c_double), ("mrw", C.c_int), ("mrw_tau_cell", C.c_double),
                ("mrw_gamma", C.c_double), ("seed", C.c_uint64), ("model_id", C.c_uint32),
                ("n_packets", C.c_uint64), ("pid_begin", C.c_uint64), ("pid_end", C.c_uint64),
                ("max_events", C.c_uint64), ("record_events", C.c_int), ("precision", C.c_int),
                ("schedule", C.c_int), ("threads_per_block", C.c_int), ("blocks_per_sm", C.c_int),
                ("march_min_active", C.c_int), ("defer_events", C.c_uint64),
                ("source_bins", C.c_uint32), ("pc_cams", C.c_void_p), ("n_pc_cams", C.c_int),
                ("record_nu_mask", C.c_void_p), ("source_grid_nu", C.c_void_p),
                ("source_grid_src", C.c_void_p), ("compact_swap", C.c_int)]


class rt_transport_out(C.Structure):
    _fields_ = [("E_abs", C.c_void_p), ("count", C.c_void_p), ("esq", C.c_void_p),
                ("sed_esc", C.c_void_p), ("sed_cnt", C.c_void_p),
                ("events", C.c_void_p), ("event_cap", C.c_uint64),
                ("pah", C.c_void_p), ("pah_cap", C.c_uint64),
                ("traj", C.c_void_p), ("traj_cap", C.c_uint64),
                ("stats", C.c_void_p), ("pc_img", C.c_void_p)]


class rt_camera(C.Structure):
    _fields_ = [("theta", C.c_double), ("phi", C.c_double), ("npix", C.c_int),
                ("D", C.c_double), ("pixel", C.c_double)]


class rt_pc_camera(C.Structure):
    _fields_ = [("theta", C.c_double), ("phi", C.c_double), ("npix", C.c_int),
                ("pixel", C.c_double), ("cos_accept", C.c_double)]


class rt_model(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("sources", C.c_void_p), ("n_sources", C.c_int),
                ("n_packets", C.c_uint64), ("T_prev", C.c_void_p), ("out", rt_transport_out)]


EVENT_DTYPE = np.dtype([("cell", "<u4"), ("nu", "<u2"), ("species", "u1"), ("model", "u1"),
                        ("k", "<f4", (3,))])
PAH_DTYPE = np.dtype([("cell", "<u4"), ("nu", "<u2"), ("model", "<u2")])
TRAJ_DTYPE = np.dtype([("pid", "<u8"), ("seq", "<u4"), ("type", "<u4"), ("cell", "<u4"),
                       ("nu", "<u4"), ("x", "<f8", (3,)), ("k", "<f8", (3,))])
assert EVENT_DTYPE.itemsize == 20 and TRAJ_DTYPE.itemsize == 72

_lib = None


def load(path: str = LIB_PATH):
    """Load librtgb.so (built by ``paper_1203_2941_gb300.build``).  Raises if
    it is missing: there is no other implementation to fall back to."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librtgb.so not found at {path}; run paper_1203_2941_gb300.build.build()")
    L = C.CDLL(path)
    vp, u64, i32, dbl = C.c_void_p, C.c_uint64, C.c_int, C.c_double
    sig = {
        "rt_last_error": (C.c_char_p, []),
        "rt_version": (C.c_char_p, []),
        "rt_ctx_create": (i32, [i32, C.POINTER(vp)]),
        "rt_ctx_destroy": (None, [vp]),
        "rt_grid_upload": (i32, [vp, i32, i32, i32, i32, C.POINTER(dbl), dbl, vp, vp, C.POINTER(vp)]),
        "rt_grid_upload_refined": (i32, [vp, i32, i32, i32, i32, C.POINTER(dbl), dbl, i32, vp, vp, vp,
                                         C.POINTER(vp)]),
        "rt_grid_ncell": (u64, [vp]),
        "rt_grid_update": (i32, [vp, vp, vp]),
        "rt_grid_free": (None, [vp]),
        "rt_opacity_upload": (i32, [vp, i32, vp, vp, i32, vp, vp, vp, vp, C.POINTER(vp)]),
        "rt_opacity_free": (None, [vp]),
        "rt_transport_params_default": (None, [C.POINTER(rt_transport_params)]),
        "rt_transport": (i32, [vp, vp, vp, vp, i32, C.POINTER(rt_transport_params), vp,
                               C.POINTER(rt_transport_out), vp]),
        "rt_transport_noalloc": (i32, [vp, vp, vp, vp, i32, C.POINTER(rt_transport_params), vp,
                                       C.POINTER(rt_transport_out), vp]),
        "rt_pah_reemit": (i32, [vp, vp, vp, vp, u64, dbl, vp, i32, vp,
                                C.POINTER(rt_transport_params), vp, C.POINTER(rt_transport_out), vp]),
        "rt_temperatures": (i32, [vp, vp, vp, vp, vp, vp]),
        "rt_temperature_guess": (i32, [vp, vp, vp, i32, vp, vp]),
        "rt_raytrace": (i32, [vp, vp, vp, vp, vp, u64, vp, dbl, vp, i32, vp, i32, vp, i32, vp, vp,
                              vp, vp]),
        "rt_raytrace_backward": (i32, [vp, vp, vp, vp, vp, u64, vp, dbl, vp, i32, vp, i32, vp, i32,
                                       vp, vp, vp, vp, vp, vp]),
        "rt_visibilities": (i32, [vp, vp, vp, i32, vp, i32, vp, i32, vp, vp]),
        "rt_kernel_launches": (u64, []),
        "rt_batch_create": (i32, [vp, vp, i32, vp, C.POINTER(rt_transport_params), C.POINTER(vp)]),
        "rt_batch_run": (i32, [vp, vp]),
        "rt_batch_free": (None, [vp]),
        "rt_transport_batched": (i32, [vp, vp, i32, vp, C.POINTER(rt_transport_params), vp]),
        "rt_philox": (i32, [vp, vp, vp, u64, vp, vp]),
        "rt_mrw_sample": (i32, [vp, vp, vp, u64, vp, vp]),
        "rt_probe_gather": (i32, [vp, vp, C.c_size_t, u64, C.c_uint32, vp, vp]),
        "rt_source_grid": (i32, [vp, vp, C.c_int, C.c_uint32, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(code, what=""):
    if code != RT_OK:
        msg = load().rt_last_error().decode()
        raise RtError(code, f"{what}: {msg}" if what else msg)


# ----------------------------------------------------------------- raw ABI (same names)
def rt_version() -> str:
    return load().rt_version().decode()


def rt_ctx_create(device: int = 0) -> int:
    h = C.c_void_p()
    _check(load().rt_ctx_create(device, C.byref(h)), "rt_ctx_create")
    return h.value


def rt_ctx_destroy(ctx: int) -> None:
    load().rt_ctx_destroy(ctx)


def rt_grid_upload_refined(ctx, nx, ny, nz, n_species, box_min, cell, refine, refined_ptr, rho_ptr,
                           stream=0) -> int:
    h = C.c_void_p()
    bm = (C.c_double * 3)(*[float(v) for v in box_min])
    _check(load().rt_grid_upload_refined(ctx, nx, ny, nz, n_species, bm, float(cell), int(refine),
                                         refined_ptr, rho_ptr, stream, C.byref(h)),
           "rt_grid_upload_refined")
    return h.value


def rt_grid_update(grid, rho_ptr, stream=0):
    _check(load().rt_grid_update(grid, rho_ptr, stream), "rt_grid_update")


def rt_grid_ncell(grid) -> int:
    return int(load().rt_grid_ncell(grid))


def rt_grid_upload(ctx, nx, ny, nz, n_species, box_min, cell, rho_ptr, stream=0) -> int:
    h = C.c_void_p()
    bm = (C.c_double * 3)(*[float(v) for v in box_min])
    _check(load().rt_grid_upload(ctx, nx, ny, nz, n_species, bm, float(cell), rho_ptr, stream,
                                 C.byref(h)), "rt_grid_upload")
    return h.value


def rt_grid_free(grid) -> None:
    load().rt_grid_free(grid)


def rt_opacity_upload(ctx, nu, dnu, kabs, ksca, g, is_pah=None) -> int:
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    dnu = np.ascontiguousarray(dnu, dtype=np.float64)
    kabs = np.ascontiguousarray(kabs, dtype=np.float64)
    ksca = np.ascontiguousarray(ksca, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    ns = kabs.shape[0] if kabs.ndim == 2 else 1
    ip = None if is_pah is None else np.ascontiguousarray(is_pah, dtype=np.int32)
    h = C.c_void_p()
    _check(load().rt_opacity_upload(ctx, nu.size, nu.ctypes.data, dnu.ctypes.data, ns,
                                    kabs.ctypes.data, ksca.ctypes.data, g.ctypes.data,
                                    None if ip is None else ip.ctypes.data, C.byref(h)),
           "rt_opacity_upload")
    return h.value


def rt_opacity_free(op) -> None:
    load().rt_opacity_free(op)


def rt_transport_params_default() -> rt_transport_params:
    p = rt_transport_params()
    load().rt_transport_params_default(C.byref(p))
    return p


def rt_transport(ctx, grid, opac, sources, n_sources, params, T_prev_ptr, out, stream=0):
    _check(load().rt_transport(ctx, grid, opac, sources, n_sources, C.byref(params), T_prev_ptr,
                               C.byref(out), stream), "rt_transport")


def rt_transport_noalloc(ctx, grid, opac, sources, n_sources, params, T_prev_ptr, out, stream=0):
    _check(load().rt_transport_noalloc(ctx, grid, opac, sources, n_sources, C.byref(params),
                                       T_prev_ptr, C.byref(out), stream), "rt_transport_noalloc")


def rt_pah_reemit(ctx, grid, opac, rec_ptr, n_rec, xi, eps, n_eps, cls_ptr, params, T_prev_ptr,
                  out, stream=0):
    _check(load().rt_pah_reemit(ctx, grid, opac, rec_ptr, n_rec, xi, eps, n_eps, cls_ptr,
                                C.byref(params), T_prev_ptr, C.byref(out), stream), "rt_pah_reemit")


def rt_temperatures(ctx, grid, opac, E_ptr, T_ptr, stream=0):
    _check(load().rt_temperatures(ctx, grid, opac, E_ptr, T_ptr, stream), "rt_temperatures")


def rt_temperature_guess(ctx, grid, sources, n_sources, T_ptr, stream=0):
    _check(load().rt_temperature_guess(ctx, grid, sources, n_sources, T_ptr, stream),
           "rt_temperature_guess")


def rt_raytrace(ctx, grid, opac, T_ptr, ev_ptr, n_ev, n_ev_dev, xi_ev, sources, n_sources, cams,
                n_cams, fidx, n_f, img_ptr, sed_ptr, steps_ptr=None, stream=0):
    _check(load().rt_raytrace(ctx, grid, opac, T_ptr, ev_ptr, n_ev, n_ev_dev, xi_ev, sources,
                              n_sources, cams, n_cams, fidx, n_f, img_ptr, sed_ptr, steps_ptr,
                              stream),
           "rt_raytrace")


def rt_visibilities(ctx, grid, cams, n_cams, img_ptr, n_f, uv, n_uv, vis_ptr, stream=0):
    _check(load().rt_visibilities(ctx, grid, cams, n_cams, img_ptr, n_f, uv, n_uv, vis_ptr, stream),
           "rt_visibilities")


def rt_raytrace_backward(ctx, grid, opac, T_ptr, ev_ptr, n_ev, n_ev_dev, xi_ev, sources,
                         n_sources, cams, n_cams, fidx, n_f, dimg_ptr, dsed_ptr, drho_ptr,
                         dscale_ptr, steps_ptr=None, stream=0):
    _check(load().rt_raytrace_backward(ctx, grid, opac, T_ptr, ev_ptr, n_ev, n_ev_dev, xi_ev,
                                       sources, n_sources, cams, n_cams, fidx, n_f, dimg_ptr,
                                       dsed_ptr, drho_ptr, dscale_ptr, steps_ptr, stream),
           "rt_raytrace_backward")


def rt_kernel_launches() -> int:
    return int(load().rt_kernel_launches())


def rt_batch_create(ctx, opac, n_models, models, params) -> int:
    h = C.c_void_p()
    _check(load().rt_batch_create(ctx, opac, n_models, models, C.byref(params), C.byref(h)),
           "rt_batch_create")
    return h.value


def rt_batch_run(batch, stream=0):
    _check(load().rt_batch_run(batch, stream), "rt_batch_run")


def rt_batch_free(batch):
    load().rt_batch_free(batch)


def rt_transport_batched(ctx, opac, n_models, models, params, stream=0):
    _check(load().rt_transport_batched(ctx, opac, n_models, models, C.byref(params), stream),
           "rt_transport_batched")


def rt_source_grid(opac, sources, n_sources, m, nu_ptr, src_ptr, star_ptr):
    _check(load().rt_source_grid(opac, sources, n_sources, m, nu_ptr, src_ptr, star_ptr), "rt_source_grid")


def rt_probe_gather(ctx, buf_ptr, nbytes, n_reads, seed, sink_ptr, stream=0):
    _check(load().rt_probe_gather(ctx, buf_ptr, nbytes, n_reads, seed, sink_ptr, stream), "rt_probe_gather")


def rt_mrw_sample(ctx, opac, u_ptr, n, y_ptr, stream=0):
    _check(load().rt_mrw_sample(ctx, opac, u_ptr, n, y_ptr, stream), "rt_mrw_sample")


def rt_philox(ctx, ctr0, key, n, out_ptr, stream=0):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr0])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    _check(load().rt_philox(ctx, c, k, n, out_ptr, stream), "rt_philox")
