"""The C ABI library builds for sm_103a, loads, and exports every symbol
that include/nbgb.h declares.  No compute call is made here (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2205_07976_gb300 import _build, nbgb
from tests.helpers import gpu_available

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(nb_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert {"nb_sim_create", "nb_set_crystal", "nb_set_beam",
            "nb_set_detector", "nb_add_spots", "nb_get_image",
            "nb_free"} <= syms
    for name in sorted(syms):
        assert hasattr(lib, name), name
    # the Python binding covers exactly the declared functions
    assert syms == set(nbgb.SIGNATURES)


def test_host_only_entry_points():
    lib = nbgb.load()
    assert lib.nb_version().decode().startswith("nbgb")
    assert lib.nb_free(None) == nbgb.NB_OK
    assert lib.nb_last_error(None) == b"null handle"
    assert lib.nb_num_pixels(None) == 0
    assert lib.nb_add_spots(None) == nbgb.NB_EINVAL
    assert lib.nb_set_scale(None, 1.0) == nbgb.NB_EINVAL
    assert lib.nb_sim_create(None, 0, 1, None) == nbgb.NB_EINVAL
    assert lib.nb_add_background(None) == nbgb.NB_EINVAL
    assert lib.nb_set_background(None, None, None, 2, 1.0) == nbgb.NB_EINVAL
    assert lib.nb_adjoint(None, None, None, None) == nbgb.NB_EINVAL
    assert lib.nb_fp64_peak_tflops(0, None) == nbgb.NB_EINVAL


@pytest.mark.skipif(gpu_available(), reason="checks the no-GPU error path")
def test_create_without_gpu_fails_cleanly():
    lib = nbgb.load()
    h = ctypes.c_void_p()
    rc = lib.nb_sim_create(ctypes.byref(h), 0, nbgb.NB_MIXED, None)
    assert rc == nbgb.NB_ECUDA
    assert not h.value
    with pytest.raises(nbgb.NbError):
        nbgb.Sim("mixed")
    # the FP64 peak probe reports an error and no rate
    x = ctypes.c_double(1.0)
    rc = lib.nb_fp64_peak_tflops(0, ctypes.byref(x))
    assert rc in (nbgb.NB_ECUDA, nbgb.NB_EINVAL)
    assert x.value == 0.0


def test_bounds_checked_build_exports_the_same_symbols():
    """The debug build (-DNB_CHECK=1) compiles, exports every declared
    symbol and says so in its version string."""
    path = _build.build(variant="check")
    assert path != _build.lib_path("release")
    lib = ctypes.CDLL(path)
    for name in sorted(declared_symbols()):
        assert hasattr(lib, name), name
    lib.nb_version.restype = ctypes.c_char_p
    assert lib.nb_version().decode().endswith("+check")
    rel = ctypes.CDLL(_build.lib_path("release"))
    rel.nb_version.restype = ctypes.c_char_p
    assert not rel.nb_version().decode().endswith("+check")
