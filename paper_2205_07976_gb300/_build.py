"""Compile libnbgb.so (the CUDA library behind include/nbgb.h) for sm_103a.

Every translation unit under csrc/ is compiled in parallel with nvcc and
linked into paper_2205_07976_gb300/_build/libnbgb.so.  A stamp file keyed
on the sources, flags and machine skips the rebuild when nothing changed.

build(variant="check") makes the debug build libnbgb_check.so: the same
sources with -DNB_CHECK=1, whose kernels check their table and image
indexing and report a failed check through the call's status (see
csrc/nbgb_internal.cuh).  nbgb.load() takes it when the environment
variable NBGB_VARIANT is "check".
"""
from __future__ import annotations

import concurrent.futures
import glob
import hashlib
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libnbgb.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr",
         "-I", INCLUDE]
# the plain FP64 form is evaluated in the order its definition is written
PER_FILE = {"spots_f64.cu": ["--fmad=false"]}


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stamp(extra_flags) -> str:
    h = hashlib.sha256()
    for f in _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
            os.path.join(INCLUDE, "nbgb.h")]:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS + list(extra_flags)).encode())
    h.update(repr(sorted(PER_FILE.items())).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


VARIANTS = {"release": ("libnbgb.so", ()),
            "check": ("libnbgb_check.so", ("-DNB_CHECK=1",))}


def lib_path(variant: str = "release") -> str:
    return os.path.join(BUILD, VARIANTS[variant][0])


def build(force: bool = False, extra_flags=(), verbose: bool = False,
          variant: str = "release") -> str:
    """Build (if needed) and return the path of libnbgb.so (or of the
    variant's library)."""
    name, vflags = VARIANTS[variant]
    lib = os.path.join(BUILD, name)
    objdir = BUILD if variant == "release" else os.path.join(BUILD, variant)
    os.makedirs(objdir, exist_ok=True)
    extra_flags = tuple(vflags) + tuple(extra_flags)
    stamp_file = os.path.join(BUILD, name[:-3] + ".stamp")
    stamp = _stamp(extra_flags)
    if (not force and os.path.exists(lib) and os.path.exists(stamp_file)
            and open(stamp_file).read() == stamp):
        return lib
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *PER_FILE.get(os.path.basename(src), []),
               *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=8) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
