"""GB300-native Monte Carlo dust radiative transfer (the method of Heymann &
Siebenmorgen 2012, arXiv:1203.2941): photon-packet transport, dust
temperatures, ray-traced images/SEDs and their density adjoint, as
hand-written sm_103a CUDA kernels behind the C ABI in include/rtgb.h.

``rtgb`` is the one-to-one ctypes binding of that ABI; ``sim`` is a thin
convenience layer that lets torch tensors own the device buffers.
"""
from . import autotune, rtgb
from .builder import build
from .rtgb import RtError, load, rt_version
from .sim import (Batch, Context, Grid, Opacity, PcCamera, RayTrace, Sources, TransportOut,
                  cameras, make_params, mrw_sample, pah_reemit, philox, raytrace, raytrace_backward,
                  source_grid, temperature_guess, temperatures, transport, visibilities)

__all__ = ["rtgb", "autotune", "build", "load", "rt_version", "RtError", "Context", "Grid", "Opacity",
           "Sources", "TransportOut", "transport", "temperatures", "temperature_guess",
           "raytrace", "raytrace_backward", "RayTrace", "philox", "mrw_sample", "Batch", "cameras",
           "make_params", "visibilities", "PcCamera", "pah_reemit", "source_grid"]
