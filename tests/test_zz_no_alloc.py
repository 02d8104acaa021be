"""The allocation-free transport entry point gives the same results as
rt_transport.

rt_transport_noalloc serves callers that cannot allocate device memory (a
host whose GPU memory belongs to another allocator with a fixed budget, or
code that must not trigger the synchronisation cudaMalloc/cudaFree can imply):
its scratch is one static device array.  Called twice in a row through the C
ABI, each call must reproduce rt_transport on the same inputs -- the second
call starts from the first call's leftover scratch, which it must clear.
Frozen-temperature transport is used so both entry points follow identical
packet histories (no dependence on the order of atomic updates): counts and
crossings agree exactly, energies and escaped SEDs to 1e-9.  This file is
collected last so that a stop at the first failure has already run every
other test.  Around a warm call, the device's free memory and the default
memory pool's usage high-water mark (the pool cudaMallocAsync draws on) must
not move: the call allocates nothing, not even memory it frees again.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _cudart():
    """The CUDA runtime already loaded into this process (by the library or torch)."""
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            return C.CDLL(name)
        except OSError:
            pass
    with open("/proc/self/maps") as f:
        for line in f:
            if "libcudart.so" in line:
                return C.CDLL(line.split()[-1])
    pytest.fail("no CUDA runtime library loaded")


class _AllocProbe:
    """Device free memory and the default pool's used-memory high-water mark."""
    RESERVED_HIGH, USED_CURRENT, USED_HIGH = 6, 7, 8      # cudaMemPoolAttr values

    def __init__(self, device=0):
        self.rt = _cudart()
        self.pool = C.c_void_p()
        assert self.rt.cudaDeviceGetDefaultMemPool(C.byref(self.pool), device) == 0

    def _attr(self, a):
        v = C.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, a, C.byref(v)) == 0
        return v.value

    def _free(self):
        free, total = C.c_size_t(), C.c_size_t()
        assert self.rt.cudaMemGetInfo(C.byref(free), C.byref(total)) == 0
        return free.value

    def start(self):
        torch.cuda.synchronize()
        zero = C.c_uint64(0)
        for a in (self.RESERVED_HIGH, self.USED_HIGH):      # reset the marks to the current use
            assert self.rt.cudaMemPoolSetAttribute(self.pool, a, C.byref(zero)) == 0
        self.used0 = self._attr(self.USED_CURRENT)
        self.free0 = self._free()

    def check(self):
        torch.cuda.synchronize()
        assert self._attr(self.USED_HIGH) == self.used0, "the pool served an allocation during the call"
        assert self._free() == self.free0, "device free memory changed during the call"


def _run(rt, fn, ctx, grid, opac, srcs, N, T_prev, seed, probe=None):
    from paper_1203_2941_gb300 import rtgb as R
    out = rt.TransportOut(grid.ncell, grid.ns, opac.nf, event_cap=8 * N)
    p = rt.make_params(N, mode=R.RT_MODE_FROZEN_T, seed=seed, record_events=True)
    stream = int(torch.cuda.current_stream().cuda_stream)
    cs = out.c_struct()
    if probe:
        probe.start()
    code = fn(ctx.h, grid.h, opac.h, srcs.arr, srcs.n, C.byref(p), int(T_prev.data_ptr()),
              C.byref(cs), stream)
    assert code == R.RT_OK, R.load().rt_last_error().decode()
    torch.cuda.synchronize()
    if probe:
        probe.check()
    return out.numpy()


def test_noalloc_matches_rt_transport_twice():
    import __graft_entry__ as g
    g.build()
    import paper_1203_2941_gb300 as rt
    from paper_1203_2941_gb300 import rtgb as R
    lib = R.load()
    ctx = rt.Context(0)
    m = W.r2_shell(n=24, tau_1um=10.0, nf=32)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    T0 = torch.tensor(W_guess(m), device="cuda")
    N = 40000
    ref = _run(rt, lib.rt_transport, ctx, grid, opac, srcs, N, T0, seed=5)
    probe = _AllocProbe(0)
    for call in range(2):
        # the first call on the device looks up the scratch array's address;
        # the second, warm call is watched for allocations
        got = _run(rt, lib.rt_transport_noalloc, ctx, grid, opac, srcs, N, T0, seed=5,
                   probe=probe if call == 1 else None)
        for k in ("crossings", "interactions", "absorptions", "scatters", "escaped", "lucy_deposits"):
            assert got["stats"][k] == ref["stats"][k], k
        np.testing.assert_array_equal(got["count"], ref["count"])
        np.testing.assert_allclose(got["E_abs"], ref["E_abs"], rtol=1e-9, atol=1e-12 * ref["E_abs"].max())
        np.testing.assert_allclose(got["esq"], ref["esq"], rtol=1e-9, atol=1e-12 * ref["esq"].max())
        np.testing.assert_allclose(got["sed_esc"], ref["sed_esc"], rtol=1e-9, atol=0)
    # a grid beyond the static scratch is refused before anything runs
    big = W.uniform_cube(n=256, tau_cell=0.1)
    gbig, opbig, sbig = ctx.grid(big), ctx.opacity(big), rt.Sources(big.sources)
    obig = rt.TransportOut(gbig.ncell, 1, opbig.nf)
    p = rt.make_params(10)
    code = lib.rt_transport_noalloc(ctx.h, gbig.h, opbig.h, sbig.arr, 1, C.byref(p), None,
                                    C.byref(obig.c_struct()),
                                    int(torch.cuda.current_stream().cuda_stream))
    assert code == R.RT_ERR_CAPACITY
    # the deferred-packet queue needs an allocation: refused, not ignored
    p = rt.make_params(N, mode=R.RT_MODE_FROZEN_T, seed=5)
    p.defer_events = 4
    out = rt.TransportOut(grid.ncell, grid.ns, opac.nf)
    code = lib.rt_transport_noalloc(ctx.h, grid.h, opac.h, srcs.arr, srcs.n, C.byref(p),
                                    int(T0.data_ptr()), C.byref(out.c_struct()),
                                    int(torch.cuda.current_stream().cuda_stream))
    assert code == R.RT_ERR_INVALID_ARG


def W_guess(m):
    # constant temperatures are enough for frozen-T transport
    return np.full((m.ns, m.ncell), 120.0)


def test_noalloc_on_refined_grid():
    """The allocation-free entry serves refined grids too (the cube tables
    belong to the grid)."""
    import __graft_entry__ as g
    g.build()
    import paper_1203_2941_gb300 as rt
    from paper_1203_2941_gb300 import rtgb as R
    lib = R.load()
    ctx = rt.Context(0)
    m = W.r2_shell_refined(n=16, tau_1um=10.0, nf=16, r=2, refine_radius=3.0)
    grid, opac, srcs = ctx.grid(m), ctx.opacity(m), rt.Sources(m.sources)
    T0 = torch.tensor(W_guess(m), device="cuda")
    N = 20000
    ref = _run(rt, lib.rt_transport, ctx, grid, opac, srcs, N, T0, seed=6)
    got = _run(rt, lib.rt_transport_noalloc, ctx, grid, opac, srcs, N, T0, seed=6)
    for k in ("crossings", "interactions", "absorptions", "escaped", "lucy_deposits"):
        assert got["stats"][k] == ref["stats"][k], k
    np.testing.assert_array_equal(got["count"], ref["count"])
    np.testing.assert_allclose(got["E_abs"], ref["E_abs"], rtol=1e-9, atol=1e-12 * ref["E_abs"].max())
