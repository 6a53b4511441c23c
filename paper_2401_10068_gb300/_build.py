"""Build of the native libraries, in-tree.

* ``libvbh.so``       -- the CUDA path (``csrc/*.cu``, sm_103a only)
* ``libvbh_synth.so`` -- the device generator of synthetic inputs (``synth/synth.cu``)

Each translation unit is compiled by nvcc in parallel into ``_build/`` and
linked with ``nvcc -shared`` (static CUDA runtime), so the libraries load
without a GPU.  A library is rebuilt when any source or header is newer.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


LIBS = {
    "vbh": {
        "sources": lambda: sorted(glob.glob(os.path.join(PKG, "csrc", "*.cu"))),
        "deps": lambda: sorted(glob.glob(os.path.join(PKG, "csrc", "*.cuh")) + glob.glob(os.path.join(PKG, "csrc", "*.h"))
                               + glob.glob(os.path.join(INCLUDE, "vbh*.h"))),
        "out": os.path.join(PKG, "libvbh.so"),
    },
    "vbh_synth": {
        "sources": lambda: [os.path.join(PKG, "synth", "synth.cu")],
        "deps": lambda: [os.path.join(INCLUDE, "vbh_synth.h")],
        "out": os.path.join(PKG, "synth", "libvbh_synth.so"),
    },
}


def lib_path(name: str) -> str:
    return LIBS[name]["out"]


def _stale(out: str, inputs) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(p) > t for p in inputs)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build_lib(name: str, force: bool = False, verbose: bool = False, pool=None) -> str:
    spec = LIBS[name]
    srcs, deps, out = spec["sources"](), spec["deps"](), spec["out"]
    if not force and not _stale(out, srcs + deps):
        return out
    odir = os.path.join(BUILD, name)
    os.makedirs(odir, exist_ok=True)
    objs = [os.path.join(odir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    cmds = [[nvcc(), *ARCH, *CFLAGS, *(["-Xptxas", "-v"] if verbose else []), "-c", s, "-o", o]
            for s, o in zip(srcs, objs)]
    own = pool is None
    ex = pool or concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1)))
    try:
        logs = list(ex.map(_run, cmds))
    finally:
        if own:
            ex.shutdown()
    tmp = out + f".tmp{os.getpid()}"
    _run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, out)
    if verbose:
        for lg in logs:
            print(lg)
    return out


def build_all(force: bool = False, verbose: bool = False):
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        futs = [ex.submit(build_lib, n, force, verbose, None) for n in LIBS]
        return [f.result() for f in futs]
