"""ctypes wrapper of the FP64 CPU oracle (rt_oracle.c).

TEST INFRASTRUCTURE ONLY: the slow, plain restatement of the paper's method
(Heymann & Siebenmorgen 2012, Sects. 2-4) that the CUDA library is checked
against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
import it.  It shares no code with the CUDA library; the inputs both consume
come from the separate ``workloads`` module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = os.path.join(HERE, "rt_oracle.c")

MODE_BW, MODE_FROZEN_T, MODE_NOREEMIT = 0, 1, 2
LUCY_OFF, LUCY_THIN, LUCY_ALL = 0, 1, 2
LUCY_LINEAR, LUCY_EXPM1 = 0, 1
T_EMIT, T_SCATTER, T_ABSORB, T_MRW, T_ESCAPE, T_PAH, T_STUCK, T_ABSORB_END = range(8)
STAT_NAMES = ["crossings", "interactions", "scatters", "absorptions", "mrw_steps", "escaped",
              "stuck", "pah", "events_dropped", "lucy_deposits", "emitted", "pah_dropped",
              "traj_dropped"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, IEEE semantics, OpenMP).

    With ``RT_ORACLE_LIB`` set in the environment, that prebuilt library is
    used instead: the mutation tests load builds of ``rt_oracle.c`` with one
    planted mistake each and check that the pins catch it."""
    alt = os.environ.get("RT_ORACLE_LIB")
    if alt:
        return alt
    os.makedirs(BUILD, exist_ok=True)
    hdr = os.path.join(HERE, "rt_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _Model(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("ns", C.c_int), ("nf", C.c_int),
                ("box_min", C.c_double * 3), ("cell", C.c_double),
                ("rho", C.c_void_p), ("nu", C.c_void_p), ("dnu", C.c_void_p),
                ("kabs", C.c_void_p), ("ksca", C.c_void_p), ("g", C.c_void_p),
                ("is_pah", C.c_void_p), ("refine", C.c_int), ("refined", C.c_void_p),
                ("leaf_base", C.c_void_p), ("nleaf", C.c_int64)]


class _Source(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("L", C.c_double), ("T_eff", C.c_double),
                ("L_nu", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("mode", C.c_int), ("lucy_mode", C.c_int), ("lucy_form", C.c_int),
                ("lucy_tau", C.c_double), ("mrw", C.c_int), ("mrw_tau_cell", C.c_double),
                ("mrw_gamma", C.c_double), ("seed", C.c_uint64), ("model_id", C.c_uint32),
                ("n_packets", C.c_uint64), ("pid_begin", C.c_uint64), ("pid_end", C.c_uint64),
                ("max_events", C.c_uint64), ("record_events", C.c_int),
                ("source_bins", C.c_uint32), ("pc", C.c_void_p), ("n_pc", C.c_int),
                ("sg_nu", C.c_void_p), ("sg_src", C.c_void_p)]


class _PcCamera(C.Structure):
    _fields_ = [("theta", C.c_double), ("phi", C.c_double), ("npix", C.c_int),
                ("pixel", C.c_double), ("cos_accept", C.c_double)]


EVENT_DTYPE = np.dtype([("cell", "<u4"), ("nu", "<u4"), ("species", "<u4"), ("pad", "<u4"),
                        ("k", "<f8", (3,))])
PAH_DTYPE = np.dtype([("cell", "<u4"), ("nu", "<u4")])
TRAJ_DTYPE = np.dtype([("pid", "<u8"), ("seq", "<u4"), ("type", "<u4"), ("cell", "<u4"),
                       ("nu", "<u4"), ("x", "<f8", (3,)), ("k", "<f8", (3,))])


class _Out(C.Structure):
    _fields_ = [("E_abs", C.c_void_p), ("count", C.c_void_p), ("esq", C.c_void_p),
                ("sed_esc", C.c_void_p), ("sed_cnt", C.c_void_p),
                ("events", C.c_void_p), ("event_cap", C.c_uint64), ("n_events", C.c_uint64),
                ("pah", C.c_void_p), ("pah_cap", C.c_uint64), ("n_pah", C.c_uint64),
                ("traj", C.c_void_p), ("traj_cap", C.c_uint64), ("n_traj", C.c_uint64),
                ("stats", C.c_uint64 * 16), ("pc_img", C.c_void_p), ("loop_seconds", C.c_double)]


class _PahSrc(C.Structure):
    _fields_ = [("rec", C.c_void_p), ("n_rec", C.c_uint64), ("xi", C.c_double),
                ("eps", C.c_void_p), ("n_eps", C.c_int), ("eps_class", C.c_void_p)]


class _Camera(C.Structure):
    _fields_ = [("theta", C.c_double), ("phi", C.c_double), ("npix", C.c_int),
                ("D", C.c_double), ("pixel", C.c_double)]


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.or_planck_B.restype = C.c_double
            L.or_planck_B.argtypes = [C.c_double, C.c_double]
            L.or_planck_dBdT.restype = C.c_double
            L.or_planck_dBdT.argtypes = [C.c_double, C.c_double]
            L.or_planck_mean.restype = C.c_double
            L.or_planck_mean.argtypes = [C.POINTER(_Model), C.c_int, C.c_double]
            L.or_solve_temperature.restype = C.c_double
            L.or_solve_temperature.argtypes = [C.POINTER(_Model), C.c_int, C.c_double]
            L.or_hg_mu.restype = C.c_double
            L.or_hg_mu.argtypes = [C.c_double, C.c_double]
            L.or_rotate.restype = None
            L.or_rotate.argtypes = [dp, C.c_double, C.c_double]
            L.or_mrw_survival.restype = C.c_double
            L.or_mrw_survival.argtypes = [C.c_double]
            L.or_mrw_sample_y.restype = C.c_double
            L.or_mrw_sample_y.argtypes = [C.c_double]
            L.or_philox4x32_10.restype = None
            L.or_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_uniforms.restype = None
            L.or_uniforms.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32, C.c_void_p]
            L.or_source_lnu.restype = None
            L.or_source_lnu.argtypes = [C.POINTER(_Model), C.POINTER(_Source), C.c_void_p]
            L.or_dda_segments.restype = C.c_int
            L.or_dda_segments.argtypes = [C.POINTER(_Model), C.c_void_p, C.c_void_p, C.c_int,
                                          C.c_void_p, C.c_void_p]
            L.or_transport.restype = C.c_int
            L.or_transport.argtypes = [C.POINTER(_Model), C.POINTER(_Source), C.c_int,
                                       C.POINTER(_Params), C.c_void_p, C.POINTER(_Out), C.c_int]
            L.or_source_grid.restype = C.c_int
            L.or_source_grid.argtypes = [C.POINTER(_Model), C.POINTER(_Source), C.c_int, C.c_uint32,
                                         C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_pah_reemit.restype = C.c_int
            L.or_pah_reemit.argtypes = [C.POINTER(_Model), C.POINTER(_PahSrc), C.POINTER(_Params),
                                        C.c_void_p, C.POINTER(_Out), C.c_int]
            L.or_temperatures.restype = None
            L.or_temperatures.argtypes = [C.POINTER(_Model), C.c_void_p, C.c_void_p]
            L.or_temperature_guess.restype = None
            L.or_temperature_guess.argtypes = [C.POINTER(_Model), C.POINTER(_Source), C.c_int,
                                               C.c_void_p]
            L.or_raytrace.restype = None
            L.or_raytrace.argtypes = [C.POINTER(_Model), C.c_void_p, C.c_void_p, C.c_uint64,
                                      C.c_double, C.POINTER(_Source), C.c_int,
                                      C.POINTER(_Camera), C.c_int, C.c_void_p, C.c_int,
                                      C.c_void_p, C.c_void_p]
            L.or_raytrace_backward.restype = None
            L.or_raytrace_backward.argtypes = [C.POINTER(_Model), C.c_void_p, C.c_void_p,
                                               C.c_uint64, C.c_double, C.POINTER(_Source), C.c_int,
                                               C.POINTER(_Camera), C.c_int, C.c_void_p, C.c_int,
                                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleModel:
    """Holds contiguous copies of a workloads.Model for the C oracle."""

    def __init__(self, model):
        self.src_model = model
        self.rho = np.ascontiguousarray(model.rho, dtype=np.float32)
        self.nu = np.ascontiguousarray(model.nu, dtype=np.float64)
        self.dnu = np.ascontiguousarray(model.dnu, dtype=np.float64)
        self.kabs = np.ascontiguousarray(model.kabs, dtype=np.float64)
        self.ksca = np.ascontiguousarray(model.ksca, dtype=np.float64)
        self.g = np.ascontiguousarray(model.g, dtype=np.float64)
        self.is_pah = np.ascontiguousarray(model.is_pah, dtype=np.int32)
        ns = self.rho.shape[0]
        nz, ny, nx = model.shape
        r = int(getattr(model, "refine", 0) or 0)
        self.refined = self.leaf_base = None
        nleaf = 0
        if r:
            self.refined = np.ascontiguousarray(model.refined, dtype=np.uint8).reshape(-1)
            per = np.where(self.refined > 0, r ** 3, 1).astype(np.int64)
            self.leaf_base = np.ascontiguousarray(np.concatenate([[0], np.cumsum(per)[:-1]]),
                                                  dtype=np.int64)
            nleaf = int(per.sum())
            assert self.rho.shape == (ns, nleaf)
        self.c = _Model(nx, ny, nz, ns, self.nu.shape[0], (C.c_double * 3)(*model.box_min),
                        float(model.cell), _ptr(self.rho), _ptr(self.nu), _ptr(self.dnu),
                        _ptr(self.kabs), _ptr(self.ksca), _ptr(self.g), _ptr(self.is_pah),
                        r, _ptr(self.refined), _ptr(self.leaf_base), nleaf)
        self._lnu = []
        srcs = []
        for s in model.sources:
            lnu = None if s.L_nu is None else np.ascontiguousarray(s.L_nu, dtype=np.float64)
            self._lnu.append(lnu)
            srcs.append(_Source((C.c_double * 3)(*s.pos), float(s.L), float(s.T_eff), _ptr(lnu)))
        self.srcs = (_Source * len(srcs))(*srcs)
        self.nsrc = len(srcs)
        self.ncell = nleaf if r else nx * ny * nz
        self.ns = ns
        self.nf = self.nu.shape[0]


def _om(model):
    return model if isinstance(model, OracleModel) else OracleModel(model)


def transport(model, n_packets, seed=1, model_id=0, mode=MODE_BW, lucy_mode=LUCY_THIN,
              lucy_form=LUCY_LINEAR, lucy_tau=1e-2, mrw=False, mrw_tau_cell=10.0, mrw_gamma=2.0,
              pid_begin=0, pid_end=None, max_events=10_000_000, record_events=False,
              event_cap=0, pah_cap=0, traj_cap=0, T_prev=None, n_threads=1, esq=True,
              accumulate=None, source_bins=0, pc_cameras=(), source_grid=None, _pah=None):
    """Run packets [pid_begin, pid_end) of an N = n_packets emission and return
    a dict of numpy arrays (E_abs, count, esq, sed_esc, sed_cnt, events, pah,
    traj, stats, pc_img).  ``accumulate`` may hold a previous result dict whose
    accumulators are continued (the B&W temperatures then see them).
    ``pc_cameras``: (theta, phi, npix, pixel, cos_accept) tuples of
    photon-counting cameras; pc_img is a list of [nf, npix, npix] images."""
    om = _om(model)
    L = lib()
    pid_end = n_packets if pid_end is None else pid_end
    p = _Params(mode, lucy_mode, lucy_form, lucy_tau, int(bool(mrw)), mrw_tau_cell, mrw_gamma,
                seed, model_id, n_packets, pid_begin, pid_end, max_events, int(bool(record_events)),
                int(source_bins))
    nc, ns, nf = om.ncell, om.ns, om.nf
    pcs = [tuple(c) for c in pc_cameras]
    pc_arr = (_PcCamera * max(1, len(pcs)))(*[_PcCamera(float(c[0]), float(c[1]), int(c[2]),
                                                         float(c[3]), float(c[4])) for c in pcs])
    if pcs:
        p.pc, p.n_pc = C.cast(pc_arr, C.c_void_p), len(pcs)
    if source_grid is not None:
        sg_nu = np.ascontiguousarray(source_grid[0], dtype=np.int32)
        sg_src = np.ascontiguousarray(source_grid[1], dtype=np.int32)
        assert len(sg_nu) == len(sg_src) == int(source_bins)
        p.sg_nu, p.sg_src = _ptr(sg_nu), _ptr(sg_src)
    pc_img = np.zeros(sum(nf * int(c[2]) ** 2 for c in pcs))
    if accumulate is not None and pcs:
        pc_img = np.concatenate([a.reshape(-1) for a in accumulate["pc_img"]]).copy()
    if accumulate is not None:
        E = accumulate["E_abs"].copy(); cnt = accumulate["count"].copy()
        q = accumulate["esq"].copy() if esq else None
        sed = accumulate["sed_esc"].copy(); sc = accumulate["sed_cnt"].copy()
    else:
        E = np.zeros((ns, nc)); cnt = np.zeros((ns, nc), np.uint32)
        q = np.zeros((ns, nc)) if esq else None
        sed = np.zeros((10, nf)); sc = np.zeros((10, nf), np.uint64)
    ev = np.zeros(event_cap, EVENT_DTYPE)
    pah = np.zeros(pah_cap, PAH_DTYPE)
    tr = np.zeros(traj_cap, TRAJ_DTYPE)
    out = _Out(_ptr(E), _ptr(cnt), _ptr(q), _ptr(sed), _ptr(sc),
               _ptr(ev) if event_cap else None, event_cap, 0,
               _ptr(pah) if pah_cap else None, pah_cap, 0,
               _ptr(tr) if traj_cap else None, traj_cap, 0)
    out.pc_img = _ptr(pc_img) if pcs else None
    Tp = None if T_prev is None else np.ascontiguousarray(T_prev, dtype=np.float64).reshape(ns, nc)
    if _pah is None:
        rc = L.or_transport(C.byref(om.c), om.srcs, om.nsrc, C.byref(p), _ptr(Tp), C.byref(out),
                            int(n_threads))
    else:
        rc = L.or_pah_reemit(C.byref(om.c), C.byref(_pah), C.byref(p), _ptr(Tp), C.byref(out),
                             int(n_threads))
    if rc != 0:
        raise ValueError("oracle transport rejected its arguments")
    stats = {k: int(out.stats[i]) for i, k in enumerate(STAT_NAMES)}
    imgs, o = [], 0
    for c in pcs:
        n = int(c[2])
        imgs.append(pc_img[o:o + nf * n * n].reshape(nf, n, n))
        o += nf * n * n
    return dict(E_abs=E, count=cnt, esq=q, sed_esc=sed, sed_cnt=sc,
                events=ev[:out.n_events], pah=pah[:out.n_pah], traj=tr[:out.n_traj],
                stats=stats, xi=model_luminosity(om) / n_packets if _pah is None else _pah.xi,
                pc_img=imgs, loop_seconds=float(out.loop_seconds))


def source_grid(model, m_bins):
    """The Eq. 1 source frequency grid: (model bin index, source index,
    frequency in Hz) of each of the m_bins equal-energy source bins."""
    om = _om(model)
    nu = np.zeros(m_bins, np.int32)
    src = np.zeros(m_bins, np.int32)
    fr = np.zeros(m_bins)
    rc = lib().or_source_grid(C.byref(om.c), om.srcs, om.nsrc, int(m_bins), _ptr(nu), _ptr(src), _ptr(fr))
    if rc != 0:
        raise ValueError("oracle source grid rejected its arguments")
    return nu, src, fr


def pah_reemit(model, records, xi, eps, eps_class=None, **kw):
    """PAH re-emission pass (Sect. 2.1, Eqs. 6-7): one packet of energy xi per
    stored PAH absorption (``records``, PAH_DTYPE or any array with a 'cell'
    field), emitted uniformly in the record's cell with its bin drawn from
    eps[n] (eps [n_eps][nf], n = eps_class[cell] or 0).  Other keywords as for
    ``transport`` (n_packets is len(records); source_bins must stay 0)."""
    om = _om(model)
    rec = np.zeros(len(records), PAH_DTYPE)
    rec["cell"] = np.asarray(records["cell"])
    eps = np.ascontiguousarray(eps, dtype=np.float64).reshape(-1, om.nf)
    cls = None if eps_class is None else np.ascontiguousarray(eps_class, dtype=np.int32).reshape(om.ncell)
    ps = _PahSrc(_ptr(rec), len(rec), float(xi), _ptr(eps), eps.shape[0], _ptr(cls))
    keep = (rec, eps, cls)
    r = transport(model, len(rec), _pah=ps, **kw)
    del keep
    return r


def model_luminosity(om):
    return float(sum(s.L for s in om.src_model.sources))


def temperatures(model, E_abs):
    om = _om(model)
    E = np.ascontiguousarray(E_abs, dtype=np.float64).reshape(om.ns, om.ncell)
    T = np.zeros_like(E)
    lib().or_temperatures(C.byref(om.c), _ptr(E), _ptr(T))
    return T


def temperature_guess(model):
    om = _om(model)
    T = np.zeros((om.ns, om.ncell))
    lib().or_temperature_guess(C.byref(om.c), om.srcs, om.nsrc, _ptr(T))
    return T


def solve_temperature(model, s, target):
    om = _om(model)
    return lib().or_solve_temperature(C.byref(om.c), int(s), float(target))


def planck_mean(model, s, T):
    om = _om(model)
    return lib().or_planck_mean(C.byref(om.c), int(s), float(T))


def planck_B(nu, T):
    return lib().or_planck_B(float(nu), float(T))


def planck_dBdT(nu, T):
    return lib().or_planck_dBdT(float(nu), float(T))


def source_lnu(model, i=0):
    om = _om(model)
    out = np.zeros(om.nf)
    lib().or_source_lnu(C.byref(om.c), C.byref(om.srcs[i]), _ptr(out))
    return out


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def uniforms(seed, model_id, pid, n):
    o = np.zeros(n)
    lib().or_uniforms(seed, model_id, pid, n, _ptr(o))
    return o


def hg_mu(g, u):
    return lib().or_hg_mu(float(g), float(u))


def rotate(k, mu, phi):
    a = (C.c_double * 3)(*k)
    lib().or_rotate(a, float(mu), float(phi))
    return np.array(a[:])


def mrw_survival(y):
    return lib().or_mrw_survival(float(y))


def mrw_sample_y(u):
    return lib().or_mrw_sample_y(float(u))


def dda_segments(model, x, k, max_seg=100000):
    om = _om(model)
    cells = np.zeros(max_seg, np.int64)
    lens = np.zeros(max_seg)
    xa = np.ascontiguousarray(x, dtype=np.float64)
    ka = np.ascontiguousarray(k, dtype=np.float64)
    n = lib().or_dda_segments(C.byref(om.c), _ptr(xa), _ptr(ka), max_seg, _ptr(cells), _ptr(lens))
    return cells[:n], lens[:n]


def _cams(cams):
    arr = (_Camera * len(cams))(*[_Camera(c.theta, c.phi, c.npix, c.D, c.pixel) for c in cams])
    return arr


def events_f64(events):
    """Accept oracle-format or CUDA-format (float32 direction) event arrays."""
    if events is None or len(events) == 0:
        return np.zeros(0, EVENT_DTYPE)
    if events.dtype == EVENT_DTYPE:
        return np.ascontiguousarray(events)
    out = np.zeros(len(events), EVENT_DTYPE)
    out["cell"] = events["cell"]
    out["nu"] = events["nu"]
    out["species"] = events["species"]
    out["k"] = np.asarray(events["k"], dtype=np.float64)
    return out


def raytrace(model, T, events, xi_ev, cams, fidx):
    om = _om(model)
    Tt = np.ascontiguousarray(T, dtype=np.float64).reshape(om.ns, om.ncell)
    ev = events_f64(events)
    fi = np.ascontiguousarray(fidx, dtype=np.int32)
    npix = cams[0].npix
    assert all(c.npix == npix for c in cams)
    img = np.zeros((len(cams), len(fi), npix, npix))
    sed = np.zeros((len(cams), len(fi)))
    lib().or_raytrace(C.byref(om.c), _ptr(Tt), _ptr(ev), len(ev), float(xi_ev), om.srcs, om.nsrc,
                      _cams(cams), len(cams), _ptr(fi), len(fi), _ptr(img), _ptr(sed))
    return img, sed


def raytrace_backward(model, T, events, xi_ev, cams, fidx, dL_dimg, dL_dsed):
    om = _om(model)
    Tt = np.ascontiguousarray(T, dtype=np.float64).reshape(om.ns, om.ncell)
    ev = events_f64(events)
    fi = np.ascontiguousarray(fidx, dtype=np.int32)
    gi = np.ascontiguousarray(dL_dimg, dtype=np.float64)
    gs = np.ascontiguousarray(dL_dsed, dtype=np.float64)
    drho = np.zeros((om.ns, om.ncell))
    dscale = np.zeros(1)
    lib().or_raytrace_backward(C.byref(om.c), _ptr(Tt), _ptr(ev), len(ev), float(xi_ev),
                               om.srcs, om.nsrc, _cams(cams), len(cams), _ptr(fi), len(fi),
                               _ptr(gi), _ptr(gs), _ptr(drho), _ptr(dscale))
    return drho, float(dscale[0])


def visibilities(model, images, cams, uv):
    """Complex visibilities of ray-traced images by their plain definition
    (FP64): V(u, v) = sum over pixels of I A_pix / D^2 exp(-2 pi i (u alpha +
    v beta)), alpha and beta the pixel centre's offsets along the image axes
    divided by D; images [n_cams][n_f][npix][npix] as or_raytrace returns
    them, uv [n_uv][2] in cycles per radian."""
    images = np.asarray(images, dtype=np.float64)
    uv = np.asarray(uv, dtype=np.float64).reshape(-1, 2)
    nz, ny, nx = model.shape
    diag = model.cell * np.sqrt(float(nx * nx + ny * ny + nz * nz))
    out = np.zeros(images.shape[:2] + (len(uv),), dtype=np.complex128)
    for c, cam in enumerate(cams):
        npix = images.shape[-1]
        pix = cam.pixel if cam.pixel > 0 else diag / cam.npix
        a = (np.arange(npix) + 0.5 - 0.5 * npix) * pix / cam.D
        for k, (u, v) in enumerate(uv):
            ph = np.exp(-2j * np.pi * (u * a[None, :] + v * a[:, None]))   # [y][x]
            out[c, :, k] = (images[c] * ph[None]).sum(axis=(1, 2)) * pix * pix / (cam.D * cam.D)
    return out
