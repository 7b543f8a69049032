"""Thin ctypes binding of libnbgb (include/nbgb.h): argument marshalling
only.  Every step of the Bragg-spot sum runs in the library's CUDA kernels;
there is no CPU fallback, and loading fails loudly when the library (or a
GPU) is missing.

The functions keep the C names (``nb_sim_create``, ``nb_set_crystal`` ...);
``Sim`` is a small convenience wrapper that feeds a ``workloads.Shot``
through them.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

NB_OK, NB_EINVAL, NB_ENOMEM, NB_ECUDA, NB_ESTATE, NB_ETIMEOUT = (
    0, -1, -2, -3, -4, -5)
NB_F64, NB_MIXED, NB_F32 = 0, 1, 2
NB_DTYPE_F32, NB_DTYPE_F64 = 0, 1
PRECISIONS = {"f64": NB_F64, "mixed": NB_MIXED, "f32": NB_F32}
NB_OPT_VARIANT = 1
NB_OPT_COUNT_WORK = 2
NB_OPT_FAIL_ALLOCS = 3
WORK_NAMES = ("pixel_steps", "units", "items", "intervals", "blocks",
              "pairs", "terms")
VARIANTS = {"auto": 0, "thread": 1, "warp": 2}

_LOCK = threading.Lock()
_LIB = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_llp = ctypes.POINTER(ctypes.c_longlong)
_vp = ctypes.c_void_p


class NbPanel(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("fdir", ctypes.c_double * 3),
                ("sdir", ctypes.c_double * 3), ("ndir", ctypes.c_double * 3),
                ("pixel_m", ctypes.c_double), ("nfast", ctypes.c_int),
                ("nslow", ctypes.c_int)]


# name -> (restype, argtypes); every symbol declared in include/nbgb.h
SIGNATURES = {
    "nb_sim_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int,
                                     ctypes.c_int, _vp]),
    "nb_set_crystal": (ctypes.c_int, [
        _vp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
        ctypes.c_double, _dp, ctypes.c_double, ctypes.c_double,
        ctypes.c_double, ctypes.c_int, _fp, _ip, _ip, ctypes.c_int,
        ctypes.c_double]),
    "nb_set_scale": (ctypes.c_int, [_vp, ctypes.c_double]),
    "nb_set_beam": (ctypes.c_int, [_vp, _dp, _dp, _dp, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, _dp]),
    "nb_set_detector": (ctypes.c_int, [_vp, ctypes.c_int,
                                       ctypes.POINTER(NbPanel), ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double]),
    "nb_num_pixels": (ctypes.c_longlong, [_vp]),
    "nb_add_spots": (ctypes.c_int, [_vp]),
    "nb_add_spots_pixels": (ctypes.c_int, [_vp, _llp, ctypes.c_longlong]),
    "nb_zero_image": (ctypes.c_int, [_vp]),
    "nb_get_image": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int,
                                    ctypes.c_int]),
    "nb_image_device_ptr": (_vp, [_vp]),
    "nb_get_stats": (ctypes.c_int, [_vp, _llp, _llp]),
    "nb_get_work": (ctypes.c_int, [_vp, _llp, ctypes.c_int]),
    "nb_set_fcell_device": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "nb_set_option": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_longlong]),
    "nb_set_crystal_params": (ctypes.c_int, [_vp, _dp, _dp, _dp, _dp,
                                             ctypes.c_double]),
    "nb_adjoint": (ctypes.c_int, [_vp, _vp, _dp, _vp]),
    "nb_poisson_loss": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp, _dp]),
    "nb_set_background": (ctypes.c_int, [_vp, _dp, _dp, ctypes.c_int,
                                         ctypes.c_double]),
    "nb_add_background": (ctypes.c_int, [_vp]),
    "nb_add_spots_noalloc": (ctypes.c_int, [
        ctypes.POINTER(NbPanel), ctypes.c_int, ctypes.c_int, ctypes.c_double,
        ctypes.c_double, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
        ctypes.c_double, ctypes.c_double, _vp, _ip, _ip, ctypes.c_int,
        ctypes.c_double, _vp, _vp, ctypes.c_int, _dp, ctypes.c_double,
        ctypes.c_double, _dp, _vp, _vp]),
    "nb_synchronize": (ctypes.c_int, [_vp]),
    "nb_fp64_peak_tflops": (ctypes.c_int, [ctypes.c_int, _dp]),
    "nb_server_create": (ctypes.c_int, [
        ctypes.POINTER(_vp), ctypes.c_int, _vp, ctypes.c_int,
        ctypes.c_longlong, ctypes.c_longlong, ctypes.POINTER(NbPanel),
        ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _fp,
        _ip, _ip, ctypes.c_int, ctypes.c_double, ctypes.c_double,
        ctypes.c_double, ctypes.c_double, _dp, ctypes.c_double,
        ctypes.c_double, _dp]),
    "nb_server_submit": (ctypes.c_int, [
        _vp, _dp, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_double,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _llp]),
    "nb_server_step": (ctypes.c_int, [_vp, ctypes.c_double, _ip]),
    "nb_server_completed": (ctypes.c_int, [_vp, _llp, ctypes.c_int, _ip]),
    "nb_server_state": (ctypes.c_int, [_vp, ctypes.c_longlong, _ip]),
    "nb_server_result": (ctypes.c_int, [_vp, ctypes.c_longlong, _vp,
                                        ctypes.c_size_t, ctypes.c_int,
                                        ctypes.c_int]),
    "nb_server_info": (ctypes.c_int, [_vp, _llp, _llp, _llp, _llp]),
    "nb_server_last_error": (ctypes.c_char_p, [_vp]),
    "nb_server_free": (ctypes.c_int, [_vp]),
    "nb_free": (ctypes.c_int, [_vp]),
    "nb_last_error": (ctypes.c_char_p, [_vp]),
    "nb_version": (ctypes.c_char_p, []),
}


def variant() -> str:
    """The library build to load: "release", or "check" (the bounds-checked
    debug build) when the environment variable NBGB_VARIANT says so."""
    return os.environ.get("NBGB_VARIANT", "release")


def library_path() -> str:
    return _build.lib_path(variant())


def load(build: bool = True):
    """Load libnbgb.so (building it first if asked); raises if missing."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = (_build.build(variant=variant()) if build
                    else _build.lib_path(variant()))
            if not os.path.exists(path):
                raise RuntimeError(f"libnbgb.so not found at {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = lib
    return _LIB


class NbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nbgb error {code}: {msg}")
        self.code = code


def _check(rc, handle=None):
    if rc != NB_OK:
        msg = load().nb_last_error(handle).decode() if handle else ""
        raise NbError(rc, msg)


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def panels_array(panels):
    arr = (NbPanel * len(panels))()
    for i, p in enumerate(panels):
        arr[i].origin[:] = [float(v) for v in p.origin]
        arr[i].fdir[:] = [float(v) for v in p.fdir]
        arr[i].sdir[:] = [float(v) for v in p.sdir]
        arr[i].ndir[:] = [float(v) for v in p.ndir]
        arr[i].pixel_m = float(p.pixel_m)
        arr[i].nfast = int(p.nfast)
        arr[i].nslow = int(p.nslow)
    return arr


class Sim:
    """One nb_sim handle.  `stream` is a torch.cuda.Stream, a raw
    cudaStream_t (int) or None (legacy default stream)."""

    def __init__(self, precision: str = "mixed", device: int = 0,
                 stream=None):
        self.lib = load()
        h = _vp()
        raw = 0
        if stream is not None:
            raw = int(getattr(stream, "cuda_stream", stream))
        self.stream = stream
        _check(self.lib.nb_sim_create(ctypes.byref(h), int(device),
                                      PRECISIONS[precision], _vp(raw)))
        self.h = h
        self.precision = precision
        self.device = int(device)
        self.npix = 0
        self.shot = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.nb_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setters ---------------------------------------------------------
    def set_crystal(self, shot, with_F: bool = True, axes=None):
        axes = _d(shot.axes if axes is None else axes).ravel()
        umats = _d(shot.umats).reshape(-1)
        if with_F:
            F = np.ascontiguousarray(shot.F, dtype=np.float32)
            fptr = F.ctypes.data_as(_fp)
        else:
            F, fptr = None, None
        hmin = (ctypes.c_int * 3)(*[int(v) for v in shot.hkl_min])
        hn = (ctypes.c_int * 3)(*[int(v) for v in shot.F.shape])
        sp = _d(shot.spindle)
        N = [float(v) for v in shot.ncells]
        _check(self.lib.nb_set_crystal(
            self.h, _ptr(axes), _ptr(umats), int(shot.umats.shape[0]),
            int(shot.n_phi), float(shot.phi0_deg), float(shot.phistep_deg),
            _ptr(sp), N[0], N[1], N[2], int(shot.shape), fptr,
            ctypes.cast(hmin, _ip), ctypes.cast(hn, _ip), int(shot.interp),
            float(shot.default_F)), self.h)
        _check(self.lib.nb_set_scale(self.h, float(shot.scale)), self.h)

    def set_beam(self, shot):
        dirs, lam, w, e = (_d(shot.dirs).ravel(), _d(shot.lambdas),
                           _d(shot.weights), _d(shot.evec))
        _check(self.lib.nb_set_beam(self.h, _ptr(dirs), _ptr(lam), _ptr(w),
                                    int(lam.shape[0]), float(shot.fluence),
                                    float(shot.kahn), _ptr(e)), self.h)

    def set_detector(self, shot):
        arr = panels_array(shot.panels)
        _check(self.lib.nb_set_detector(
            self.h, len(shot.panels), arr, int(shot.oversample),
            int(shot.n_layers), float(shot.thickness_m),
            float(shot.atten_m)), self.h)
        self.npix = int(self.lib.nb_num_pixels(self.h))

    def upload_F(self, F):
        """Replace the structure-factor table (same shape and origin)."""
        s = self.shot.copy()
        s.F = np.ascontiguousarray(F, dtype=np.float32)
        self.set_crystal(s)

    def set_fcell_device(self, ptr: int, n: int):
        """Replace the resident table's values from n float32 values at a
        device pointer (stream-ordered device-to-device copy)."""
        _check(self.lib.nb_set_fcell_device(self.h, _vp(ptr), int(n)), self.h)

    def set_shot(self, shot):
        self.shot = shot
        self.set_crystal(shot)
        self.set_beam(shot)
        self.set_detector(shot)
        return self

    # -- work --------------------------------------------------------------
    def add_spots(self, pixels=None):
        if pixels is None:
            _check(self.lib.nb_add_spots(self.h), self.h)
        else:
            pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
            _check(self.lib.nb_add_spots_pixels(self.h, _ptr(pix, _llp),
                                                pix.shape[0]), self.h)

    def zero(self):
        _check(self.lib.nb_zero_image(self.h), self.h)

    def set_params(self, U, cell, rot, ncells, scale):
        """Lab axes = rows of Rx Ry Rz U diag(cell); sets N and scale."""
        U, cell, rot, N = _d(U).ravel(), _d(cell), _d(rot), _d(ncells)
        _check(self.lib.nb_set_crystal_params(self.h, _ptr(U), _ptr(cell),
                                              _ptr(rot), _ptr(N),
                                              float(scale)), self.h)
        return self

    def adjoint(self, dLdI_ptr: int, gradF_ptr: int = 0) -> np.ndarray:
        """dL/d(tx, ty, tz, a, b, c, Na, Nb, Nc, scale) given a device
        array of dL/dI; adds dL/dF into the device array at gradF_ptr."""
        g = np.zeros(10)
        _check(self.lib.nb_adjoint(self.h, _vp(dLdI_ptr), _ptr(g),
                                   _vp(gradF_ptr) if gradF_ptr else None),
               self.h)
        return g

    def poisson_loss(self, y_ptr: int, bkg: float, dLdI_ptr: int) -> float:
        out = ctypes.c_double()
        _check(self.lib.nb_poisson_loss(self.h, _vp(y_ptr), float(bkg),
                                        _vp(dLdI_ptr), ctypes.byref(out)),
               self.h)
        return float(out.value)

    def set_background(self, bg):
        """Copies an amorphous-background table (attributes stol, F,
        n_molecules) into the handle."""
        st = np.ascontiguousarray(bg.stol, dtype=np.float64)
        F = np.ascontiguousarray(bg.F, dtype=np.float64)
        _check(self.lib.nb_set_background(self.h, _ptr(st), _ptr(F),
                                          int(st.shape[0]),
                                          float(bg.n_molecules)), self.h)
        return self

    def add_background(self):
        """Queues the background of every pixel into the image."""
        _check(self.lib.nb_add_background(self.h), self.h)
        return self

    def set_variant(self, name: str):
        _check(self.lib.nb_set_option(self.h, NB_OPT_VARIANT,
                                      VARIANTS[name]), self.h)
        return self

    def stats(self):
        """(evaluated_terms, pixel_steps) of the last add_spots call."""
        ev, ps = ctypes.c_longlong(), ctypes.c_longlong()
        _check(self.lib.nb_get_stats(self.h, ctypes.byref(ev),
                                     ctypes.byref(ps)), self.h)
        return int(ev.value), int(ps.value)

    def fail_allocations(self, n: int):
        """Test hook: the library's next n device allocations (any handle)
        fail as if the device were out of memory; 0 turns it off."""
        _check(self.lib.nb_set_option(self.h, NB_OPT_FAIL_ALLOCS, int(n)),
               self.h)
        return self

    def count_work(self, on: bool = True):
        """Make the following launches count the work work() reports."""
        _check(self.lib.nb_set_option(self.h, NB_OPT_COUNT_WORK, int(on)),
               self.h)
        return self

    def work(self):
        """Work counts of the last add_spots call (nb_get_work), by name."""
        v = (ctypes.c_longlong * len(WORK_NAMES))()
        _check(self.lib.nb_get_work(self.h, ctypes.cast(v, _llp),
                                    len(WORK_NAMES)), self.h)
        return dict(zip(WORK_NAMES, [int(x) for x in v]))

    def synchronize(self):
        _check(self.lib.nb_synchronize(self.h), self.h)

    def image(self, dtype=np.float64) -> np.ndarray:
        out = np.empty(self.npix, dtype=dtype)
        code = NB_DTYPE_F64 if out.dtype == np.float64 else NB_DTYPE_F32
        _check(self.lib.nb_get_image(self.h, out.ctypes.data_as(_vp),
                                     out.shape[0], code, 0), self.h)
        return out

    def image_to_device(self, dst_ptr: int, n: int, dtype_code: int):
        _check(self.lib.nb_get_image(self.h, _vp(dst_ptr), n, dtype_code, 1),
               self.h)

    def image_device_ptr(self) -> int:
        return int(self.lib.nb_image_device_ptr(self.h) or 0)


def simulate(shot, precision: str = "mixed", pixels=None,
             device: int = 0, variant: str = "auto") -> np.ndarray:
    """Image of `shot` (all pixels, or the listed ones in list order)."""
    sim = Sim(precision, device).set_shot(shot).set_variant(variant)
    try:
        sim.add_spots(pixels)
        img = sim.image()
        if pixels is not None:
            return img[np.asarray(pixels, dtype=np.int64)]
        return img
    finally:
        sim.close()


def fp64_peak_tflops(device: int = 0) -> float:
    """Measured FP64 FMA throughput of `device` in TFLOP/s."""
    out = ctypes.c_double(0.0)
    _check(load().nb_fp64_peak_tflops(int(device), ctypes.byref(out)))
    return out.value


NB_REQ_UNKNOWN, NB_REQ_QUEUED, NB_REQ_RUNNING, NB_REQ_DONE = -1, 0, 1, 2


def _check_srv(rc, lib, h):
    if rc != NB_OK:
        raise NbError(rc, lib.nb_server_last_error(h).decode() if h else "")


class Server:
    """Continuous-batching shot server (nb_server_*).  `shot` supplies the
    resident state: its first panel, oversample, layers, F table, N,
    beam direction, fluence and polarization."""

    def __init__(self, shot, max_slots=64, pool_bytes=1 << 30,
                 step_budget=0, device=0, stream=None):
        self.lib = load()
        h = _vp()
        raw = 0 if stream is None else int(getattr(stream, "cuda_stream",
                                                   stream))
        p = panels_array(shot.panels[:1])
        F = np.ascontiguousarray(shot.F, dtype=np.float32)
        hmin = (ctypes.c_int * 3)(*[int(v) for v in shot.hkl_min])
        hn = (ctypes.c_int * 3)(*[int(v) for v in F.shape])
        d = _d(shot.dirs[0])
        e = _d(shot.evec)
        N = [float(v) for v in shot.ncells]
        rc = self.lib.nb_server_create(
            ctypes.byref(h), int(device), _vp(raw), int(max_slots),
            int(pool_bytes), int(step_budget), p, int(shot.oversample),
            int(shot.n_layers), float(shot.thickness_m), float(shot.atten_m),
            F.ctypes.data_as(_fp), ctypes.cast(hmin, _ip),
            ctypes.cast(hn, _ip), int(shot.interp), float(shot.default_F),
            N[0], N[1], N[2], _ptr(d), float(shot.fluence), float(shot.kahn),
            _ptr(e))
        if rc != NB_OK:
            raise NbError(rc, "nb_server_create")
        self.h = h
        self.npix_of = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.nb_server_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, axes, umats, lambdas, weights, scale, roi):
        f0, s0, nf, ns = [int(v) for v in roi]
        axes, umats = _d(axes).ravel(), _d(umats).ravel()
        lam, w = _d(lambdas), _d(weights)
        rid = ctypes.c_longlong()
        _check_srv(self.lib.nb_server_submit(
            self.h, _ptr(axes), _ptr(umats), int(umats.size // 9),
            _ptr(lam), _ptr(w), int(lam.size), float(scale), f0, s0, nf, ns,
            ctypes.byref(rid)), self.lib, self.h)
        self.npix_of[rid.value] = nf * ns
        return rid.value

    def step(self, timeout_s=60.0):
        n = ctypes.c_int()
        _check_srv(self.lib.nb_server_step(self.h, float(timeout_s),
                                           ctypes.byref(n)), self.lib, self.h)
        return n.value

    def completed(self, max_ids=4096):
        ids = (ctypes.c_longlong * max_ids)()
        n = ctypes.c_int()
        _check_srv(self.lib.nb_server_completed(
            self.h, ctypes.cast(ids, _llp), max_ids, ctypes.byref(n)),
            self.lib, self.h)
        return [ids[i] for i in range(n.value)]

    def state(self, rid):
        st = ctypes.c_int()
        _check_srv(self.lib.nb_server_state(self.h, int(rid),
                                            ctypes.byref(st)),
                   self.lib, self.h)
        return st.value

    def result(self, rid, out=None):
        n = self.npix_of[rid]
        if out is None:
            out = np.empty(n, dtype=np.float64)
        _check_srv(self.lib.nb_server_result(
            self.h, int(rid), out.ctypes.data_as(_vp), n, NB_DTYPE_F64, 0),
            self.lib, self.h)
        del self.npix_of[rid]
        return out

    def info(self):
        v = [ctypes.c_longlong() for _ in range(4)]
        _check_srv(self.lib.nb_server_info(self.h, *[ctypes.byref(x)
                                                     for x in v]),
                   self.lib, self.h)
        return dict(zip(("queued", "running", "done", "pool_free_bytes"),
                        [x.value for x in v]))

    def run_all(self, timeout_s=60.0, fetch=False):
        """Step until nothing is queued or running.  Returns the completed
        ids in completion order, or with fetch=True a dict id -> image
        (fetching as they complete, which frees their pool memory)."""
        done, images = [], {}
        while True:
            active = self.step(timeout_s)
            new = self.completed()
            done += new
            if fetch:
                for rid in new:
                    images[rid] = self.result(rid)
            if active == 0:
                break
        return images if fetch else done
