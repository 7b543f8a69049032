"""nb_add_spots_noalloc, the entry point that allocates nothing.

It serves callers that cannot call cudaMalloc (all their device memory
comes from their own pool, or their host forbids device allocations): they
pass every input and the output as device memory they own, and the
library's scratch lives in a fixed device array.  Here the inputs are
allocated by the test (torch), and two calls in a row must each reproduce
the image of the regular entry point within the FP32-mixed tolerance.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2205_07976_gb300 import nbgb
from paper_2205_07976_gb300 import workloads as W
from tests.helpers import abs_err_frac, masked_rel_err

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5


def _call(lib, shot, axes_pm, F, lam, w, image, stream):
    p = nbgb.panels_array(shot.panels)
    hmin = (ctypes.c_int * 3)(*[int(v) for v in shot.hkl_min])
    hn = (ctypes.c_int * 3)(*[int(v) for v in shot.F.shape])
    d = np.ascontiguousarray(shot.dirs[0], dtype=np.float64)
    e = np.ascontiguousarray(shot.evec, dtype=np.float64)
    N = [float(v) for v in shot.ncells]
    return lib.nb_add_spots_noalloc(
        p, int(shot.oversample), int(shot.n_layers), float(shot.thickness_m),
        float(shot.atten_m), nbgb._vp(axes_pm.data_ptr()),
        int(axes_pm.shape[0]), N[0], N[1], N[2], float(shot.scale),
        nbgb._vp(F.data_ptr()), ctypes.cast(hmin, nbgb._ip),
        ctypes.cast(hn, nbgb._ip), int(shot.interp), float(shot.default_F),
        nbgb._vp(lam.data_ptr()), nbgb._vp(w.data_ptr()), int(lam.shape[0]),
        d.ctypes.data_as(nbgb._dp), float(shot.fluence), float(shot.kahn),
        e.ctypes.data_as(nbgb._dp), nbgb._vp(image.data_ptr()),
        nbgb._vp(stream.cuda_stream))


def test_noalloc_matches_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    shot = W.shrink(W.large_shot(), 37, 29, 2500, 700)
    ref = nbgb.simulate(shot, "mixed", variant="warp")

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    # one crystal orientation per mosaic domain (one phi step at 0 deg)
    axes_pm = np.stack([(U @ shot.axes.T).T for U in shot.umats])
    axes_t = torch.from_numpy(np.ascontiguousarray(axes_pm)).to(dev)
    F = torch.from_numpy(np.ascontiguousarray(shot.F)).to(dev)
    lam = torch.from_numpy(np.ascontiguousarray(shot.lambdas)).to(dev)
    w = torch.from_numpy(np.ascontiguousarray(shot.weights)).to(dev)
    lib = nbgb.load()
    outs = []
    for _ in range(2):
        image = torch.zeros(shot.npix, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        rc = _call(lib, shot, axes_t, F, lam, w, image, stream)
        assert rc == nbgb.NB_OK
        stream.synchronize()
        got = image.cpu().numpy()
        rel, n = masked_rel_err(got, ref, 1e-3)
        assert rel <= MIXED_TOL, (rel, n)
        assert abs_err_frac(got, ref) <= MIXED_TOL
        outs.append(got)
    # the scratch is rewritten per call: the two calls agree exactly
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    shot = W.shrink(W.large_shot(), 8, 8, 2500, 700)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    big = torch.zeros((2049, 9), dtype=torch.float64, device=dev)
    F = torch.from_numpy(np.ascontiguousarray(shot.F)).to(dev)
    lam = torch.from_numpy(np.ascontiguousarray(shot.lambdas)).to(dev)
    w = torch.from_numpy(np.ascontiguousarray(shot.weights)).to(dev)
    image = torch.zeros(shot.npix, dtype=torch.float64, device=dev)
    rc = _call(nbgb.load(), shot, big, F, lam, w, image, stream)
    assert rc == nbgb.NB_EINVAL
    assert not image.any().item()
