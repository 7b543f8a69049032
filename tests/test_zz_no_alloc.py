"""nb_add_spots_noalloc, the entry point that allocates nothing.

It serves callers that cannot call cudaMalloc (all their device memory
comes from their own pool, or their host forbids device allocations): they
pass every input and the output as device memory they own, and the
library's scratch lives in a fixed device array.  Here the inputs are
allocated by the test (torch).  Two calls in a row must each reproduce the
FP64 oracle's image and the regular entry point's image within the
FP32-mixed tolerance, for nearest and tricubic lookup and for sources in
any order, without changing the device's free memory.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2205_07976_gb300 import nbgb
from paper_2205_07976_gb300 import workloads as W
from tests.helpers import abs_err_frac, masked_rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

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


def _device_inputs(shot, dev):
    # one crystal orientation per mosaic domain (one phi step at 0 deg)
    axes_pm = np.stack([(U @ shot.axes.T).T for U in shot.umats])
    return (torch.from_numpy(np.ascontiguousarray(axes_pm)).to(dev),
            torch.from_numpy(np.ascontiguousarray(shot.F)).to(dev),
            torch.from_numpy(np.ascontiguousarray(shot.lambdas)).to(dev),
            torch.from_numpy(np.ascontiguousarray(shot.weights)).to(dev))


def _check(got, ref):
    rel, n = masked_rel_err(got, ref, 1e-3)
    assert rel <= MIXED_TOL, (rel, n)
    assert abs_err_frac(got, ref) <= MIXED_TOL


CASES = [("tricubic", W.INTERP_TRICUBIC, False),
         ("nearest", W.INTERP_NEAREST, False),
         ("tricubic-unsorted-sources", W.INTERP_TRICUBIC, True)]


@pytest.mark.parametrize("name,interp,shuffle", CASES,
                         ids=[c[0] for c in CASES])
def test_noalloc_matches_oracle_twice(name, interp, shuffle):
    shot = W.shrink(W.large_shot(), 37, 29, 2500, 700)
    shot.interp = interp
    if shuffle:
        # sources in no order of wavelength: the kernel cannot use its
        # sorted-interval bounds and prunes by source blocks instead
        perm = np.random.default_rng(11).permutation(shot.n_src)
        shot.lambdas = shot.lambdas[perm].copy()
        shot.weights = shot.weights[perm].copy()
        shot.dirs = shot.dirs[perm].copy()
        assert np.any(np.diff(1.0 / shot.lambdas) < 0)
    ref = oracle.image(shot)
    lib_img = nbgb.simulate(shot, "mixed", variant="warp")

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    axes_t, F, lam, w = _device_inputs(shot, dev)
    lib = nbgb.load()
    images = [torch.zeros(shot.npix, dtype=torch.float64, device=dev)
              for _ in range(2)]
    torch.cuda.synchronize()
    outs = []
    for i in range(2):
        free0 = torch.cuda.mem_get_info(dev)[0]
        alloc0 = torch.cuda.memory_allocated(dev)
        rc = _call(lib, shot, axes_t, F, lam, w, images[i], stream)
        assert rc == nbgb.NB_OK
        stream.synchronize()
        if i == 1:
            # the warm call takes no device memory, from torch or CUDA
            assert torch.cuda.mem_get_info(dev)[0] == free0
            assert torch.cuda.memory_allocated(dev) == alloc0
        got = images[i].cpu().numpy()
        _check(got, ref)
        _check(got, lib_img)
        outs.append(got)
    # the scratch is rewritten per call: the two calls agree exactly
    assert np.array_equal(outs[0], outs[1])


def _try(lib, shot, n_pm, n_src, dev, stream):
    axes = torch.zeros((n_pm, 9), dtype=torch.float64, device=dev)
    axes[:, 0] = shot.axes[0, 0]  # never launched when rejected
    F = torch.from_numpy(np.ascontiguousarray(shot.F)).to(dev)
    lam = torch.ones(n_src, dtype=torch.float64, device=dev)
    w = torch.ones(n_src, dtype=torch.float64, device=dev)
    image = torch.zeros(shot.npix, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    return _call(lib, shot, axes, F, lam, w, image, stream), image


def test_noalloc_rejects_sizes_beyond_its_scratch():
    shot = W.shrink(W.large_shot(), 8, 8, 2500, 700)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    lib = nbgb.load()
    # beyond the scratch array's tables
    rc, image = _try(lib, shot, 2049, 100, dev, stream)
    assert rc == nbgb.NB_EINVAL
    assert not image.any().item()
    rc, _ = _try(lib, shot, 50, 1025, dev, stream)
    assert rc == nbgb.NB_EINVAL
    # each limit alone fits the scratch, but not both together: the staged
    # tables must also fit the kernel's shared memory
    rc, image = _try(lib, shot, 2048, 1024, dev, stream)
    assert rc == nbgb.NB_EINVAL
    assert not image.any().item()


def test_noalloc_largest_accepted_tables_match_regular_entry():
    """The most sources accepted with 2048 orientations (found by
    bisection on the entry point's own answer, which is decided on the
    host before any launch) give the regular entry point's image."""
    base = W.shrink(W.large_shot(), 37, 29, 2500, 700)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    lib = nbgb.load()

    umats = W.mosaic_umats(np.random.default_rng(12), 2048, 0.05)

    def accepted(S):
        s = base.copy()
        s.umats = umats
        s.dirs, s.lambdas, s.weights = W.gaussian_spectrum(S, 9.5, 0.005)
        axes_t, F, lam, w = _device_inputs(s, dev)
        image = torch.zeros(s.npix, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        rc = _call(lib, s, axes_t, F, lam, w, image, stream)
        stream.synchronize()
        return rc, s, image

    lo, hi = 1, 1024  # accepted(lo), not accepted(hi + 1) by the limit
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if accepted(mid)[0] == nbgb.NB_OK:
            lo = mid
        else:
            hi = mid - 1
    rc, s, image = accepted(lo)
    assert rc == nbgb.NB_OK and 100 <= lo < 1024
    assert accepted(lo + 1)[0] == nbgb.NB_EINVAL
    ref = nbgb.simulate(s, "mixed", variant="warp")
    assert ref.max() > 0
    _check(image.cpu().numpy(), ref)
