"""FP64 CPU oracle for the per-pixel Bragg-spot sum (Sec. III-B).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.
It shares no code with the CUDA library: the C source ``nb_oracle.c`` is
compiled here with gcc (FP64, no FMA contraction, OpenMP over pixels) and
called through ctypes.  Its inputs are the ``Shot`` objects of the seeded
generators, read by attribute only.

Pins (tests/test_oracle_pins.py) tie it to closed forms, invariances,
special cases and brute force; every function here has one.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIB = None

R_E = 2.8179403262e-15  # classical electron radius, m (CODATA 2018)


def _lib_path() -> str:
    return os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile nb_oracle.c (gcc, -O2, FP64 without FMA contraction)."""
    out = _lib_path()
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _Params(ctypes.Structure):
    _fields_ = [
        ("axes", ctypes.c_double * 9),
        ("umats", ctypes.POINTER(ctypes.c_double)),
        ("n_mosaic", ctypes.c_int),
        ("n_phi", ctypes.c_int),
        ("phi0_deg", ctypes.c_double),
        ("phistep_deg", ctypes.c_double),
        ("spindle", ctypes.c_double * 3),
        ("ncells", ctypes.c_double * 3),
        ("shape", ctypes.c_int),
        ("scale", ctypes.c_double),
        ("F", ctypes.POINTER(ctypes.c_double)),
        ("hkl_min", ctypes.c_int * 3),
        ("hkl_n", ctypes.c_int * 3),
        ("interp", ctypes.c_int),
        ("default_F", ctypes.c_double),
        ("dirs", ctypes.POINTER(ctypes.c_double)),
        ("lambdas", ctypes.POINTER(ctypes.c_double)),
        ("weights", ctypes.POINTER(ctypes.c_double)),
        ("n_src", ctypes.c_int),
        ("fluence", ctypes.c_double),
        ("kahn", ctypes.c_double),
        ("evec", ctypes.c_double * 3),
        ("n_panels", ctypes.c_int),
        ("panel_geom", ctypes.POINTER(ctypes.c_double)),
        ("panel_dims", ctypes.POINTER(ctypes.c_int)),
        ("oversample", ctypes.c_int),
        ("n_layers", ctypes.c_int),
        ("thickness", ctypes.c_double),
        ("atten", ctypes.c_double),
        ("sinc_mode", ctypes.c_int),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_llp = ctypes.POINTER(ctypes.c_longlong)


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            L.orc_image.argtypes = [ctypes.POINTER(_Params), _llp,
                                    ctypes.c_longlong, _dp, ctypes.c_int]
            L.orc_image.restype = ctypes.c_int
            L.orc_sincg.argtypes = [ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int]
            L.orc_sincg.restype = ctypes.c_double
            L.orc_flatt.argtypes = [ctypes.POINTER(_Params), _dp]
            L.orc_flatt.restype = ctypes.c_double
            L.orc_fcell.argtypes = [ctypes.POINTER(_Params), _dp]
            L.orc_fcell.restype = ctypes.c_double
            L.orc_polar.argtypes = [_dp, _dp, ctypes.c_double, _dp]
            L.orc_polar.restype = ctypes.c_double
            L.orc_omega.argtypes = [ctypes.c_double, _dp, _dp]
            L.orc_omega.restype = ctypes.c_double
            L.orc_capture.argtypes = [ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double]
            L.orc_capture.restype = ctypes.c_double
            L.orc_background.argtypes = [ctypes.POINTER(_Params), _dp, _dp,
                                         ctypes.c_int, ctypes.c_double,
                                         _llp, ctypes.c_longlong, _dp,
                                         ctypes.c_int]
            L.orc_background.restype = ctypes.c_int
            L.orc_bg_factor.argtypes = [_dp, _dp, ctypes.c_int,
                                        ctypes.c_double]
            L.orc_bg_factor.restype = ctypes.c_double
            L.orc_max_threads.argtypes = []
            L.orc_max_threads.restype = ctypes.c_int
            L.orc_param_axes.argtypes = [_dp, _dp, _dp, _dp, _dp]
            L.orc_param_axes.restype = None
            L.orc_loss_grad.argtypes = [ctypes.POINTER(_Params), _dp, _dp,
                                        _dp, _llp, ctypes.c_longlong, _dp,
                                        ctypes.c_double, _dp, _dp, _dp, _dp,
                                        ctypes.c_int]
            L.orc_loss_grad.restype = ctypes.c_int
            _LIB = L
    return _LIB


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


class _Bound:
    """A ctypes parameter block plus the arrays it points into."""

    def __init__(self, shot, sinc_mode: str = "reduced"):
        keep = []

        def arr(a, dt=np.float64):
            x = np.ascontiguousarray(np.asarray(a, dtype=dt))
            keep.append(x)
            return x

        p = _Params()
        p.axes[:] = list(np.asarray(shot.axes, dtype=np.float64).ravel())
        umats = arr(shot.umats)
        p.umats = _ptr(umats)
        p.n_mosaic = int(umats.shape[0])
        p.n_phi = int(shot.n_phi)
        p.phi0_deg = float(shot.phi0_deg)
        p.phistep_deg = float(shot.phistep_deg)
        p.spindle[:] = [float(v) for v in shot.spindle]
        p.ncells[:] = [float(v) for v in shot.ncells]
        p.shape = int(shot.shape)
        p.scale = float(shot.scale)
        F = arr(shot.F)  # float32 table -> exact float64 copy
        p.F = _ptr(F)
        p.hkl_min[:] = [int(v) for v in shot.hkl_min]
        p.hkl_n[:] = [int(v) for v in F.shape]
        p.interp = int(shot.interp)
        p.default_F = float(shot.default_F)
        dirs, lam, w = arr(shot.dirs), arr(shot.lambdas), arr(shot.weights)
        p.dirs, p.lambdas, p.weights = _ptr(dirs), _ptr(lam), _ptr(w)
        p.n_src = int(lam.shape[0])
        p.fluence = float(shot.fluence)
        p.kahn = float(shot.kahn)
        p.evec[:] = [float(v) for v in shot.evec]
        geom = arr(np.concatenate([
            np.concatenate([q.origin, q.fdir, q.sdir, q.ndir, [q.pixel_m]])
            for q in shot.panels]))
        dims = arr(np.array([[q.nfast, q.nslow] for q in shot.panels]),
                   np.int32)
        p.n_panels = len(shot.panels)
        p.panel_geom = _ptr(geom)
        p.panel_dims = _ptr(dims, _ip)
        p.oversample = int(shot.oversample)
        p.n_layers = int(shot.n_layers)
        p.thickness = float(shot.thickness_m)
        p.atten = float(shot.atten_m)
        p.sinc_mode = {"literal": 0, "reduced": 1}[sinc_mode]
        self.p = p
        self.keep = keep


def max_threads() -> int:
    return int(lib().orc_max_threads())


def image(shot, pixels=None, nthreads: int = 0,
          sinc_mode: str = "reduced") -> np.ndarray:
    """FP64 image values (photons) of the given global pixel indices
    (panel-major, then slow, then fast); all pixels if None."""
    if pixels is None:
        pixels = np.arange(shot.npix, dtype=np.int64)
    pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
    out = np.zeros(pix.shape[0], dtype=np.float64)
    b = _Bound(shot, sinc_mode)
    rc = lib().orc_image(ctypes.byref(b.p), _ptr(pix, _llp), pix.shape[0],
                         _ptr(out), int(nthreads))
    if rc != 0:
        raise ValueError(f"orc_image failed ({rc})")
    return out


def background(shot, bg, pixels=None, nthreads: int = 0) -> np.ndarray:
    """FP64 amorphous-background values (photons) of the given pixels: the
    detector and beam of ``shot`` and the table of ``bg`` (attributes
    ``stol``, ``F``, ``n_molecules``); all pixels if None."""
    if pixels is None:
        pixels = np.arange(shot.npix, dtype=np.int64)
    pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
    out = np.zeros(pix.shape[0], dtype=np.float64)
    b = _Bound(shot)
    st, F = _f64(bg.stol), _f64(bg.F)
    rc = lib().orc_background(ctypes.byref(b.p), _ptr(st), _ptr(F),
                              int(st.shape[0]), float(bg.n_molecules),
                              _ptr(pix, _llp), pix.shape[0], _ptr(out),
                              int(nthreads))
    if rc != 0:
        raise ValueError(f"orc_background failed ({rc})")
    return out


def background_factor(bg, stol: float) -> float:
    st, F = _f64(bg.stol), _f64(bg.F)
    return lib().orc_bg_factor(_ptr(st), _ptr(F), int(st.shape[0]),
                               float(stol))


def sincg(h: float, N: float, mode: str = "reduced") -> float:
    return lib().orc_sincg(float(h), float(N),
                           {"literal": 0, "reduced": 1}[mode])


def flatt(shot, hkl) -> float:
    b = _Bound(shot)
    v = _f64(hkl)
    return lib().orc_flatt(ctypes.byref(b.p), _ptr(v))


def fcell(shot, hkl) -> float:
    b = _Bound(shot)
    v = _f64(hkl)
    return lib().orc_fcell(ctypes.byref(b.p), _ptr(v))


def polarization(d, inc, K: float, e) -> float:
    d, inc, e = _f64(d), _f64(inc), _f64(e)
    return lib().orc_polar(_ptr(d), _ptr(inc), float(K), _ptr(e))


def solid_angle(px: float, n, P) -> float:
    n, P = _f64(n), _f64(P)
    return lib().orc_omega(float(px), _ptr(n), _ptr(P))


def capture(t: int, dt: float, atten: float, rho: float,
            thickness: float) -> float:
    return lib().orc_capture(int(t), float(dt), float(atten), float(rho),
                             float(thickness))


def param_axes(U, cell, rot):
    """(axes rows a, b, c; derivatives w.r.t. tx, ty, tz, a, b, c)."""
    U, cell, rot = _f64(U), _f64(cell), _f64(rot)
    axes = np.zeros(9)
    d = np.zeros(54)
    lib().orc_param_axes(_ptr(U), _ptr(cell), _ptr(rot), _ptr(axes),
                         _ptr(d))
    return axes.reshape(3, 3), d.reshape(6, 3, 3)


def loss_grad(shot, U, cell, rot, y, bkg: float, pixels=None,
              want_F: bool = True, nthreads: int = 0):
    """Poisson loss sum_p (I_p + bkg - y_p log(I_p + bkg)) over `pixels`
    with lab axes Rx Ry Rz U diag(cell); returns (loss, grad[10], gradF or
    None, model).  grad order: tx, ty, tz, a, b, c, Na, Nb, Nc, scale."""
    if pixels is None:
        pixels = np.arange(shot.npix, dtype=np.int64)
    pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
    y = _f64(y)
    assert y.shape[0] == pix.shape[0]
    b = _Bound(shot)
    U, cell, rot = _f64(U), _f64(cell), _f64(rot)
    loss = np.zeros(1)
    grad = np.zeros(10)
    gF = np.zeros(shot.F.size) if want_F else None
    model = np.zeros(pix.shape[0])
    rc = lib().orc_loss_grad(ctypes.byref(b.p), _ptr(U), _ptr(cell),
                             _ptr(rot), _ptr(pix, _llp), pix.shape[0],
                             _ptr(y), float(bkg), _ptr(loss), _ptr(grad),
                             _ptr(gF) if want_F else None, _ptr(model),
                             int(nthreads))
    if rc != 0:
        raise ValueError(f"orc_loss_grad failed ({rc})")
    return float(loss[0]), grad, (gF.reshape(shot.F.shape) if want_F
                                  else None), model
