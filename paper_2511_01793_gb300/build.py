"""Builds the sm_103a shared library ``_lib/libemagpie.so`` in-tree with nvcc.

The translation units compile in parallel; the link step produces one
shared object exporting the C ABI of ``include/emagpie.h``.  The build is
skipped when the sources and flags are unchanged since the last build.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB_NAME = "libemagpie.so"
SOURCES = ["emg_kernels.cu", "emg_capi.cu", "emg_tc.cu", "emg_metrics.cu"]
HEADERS = ["emg_fft.cuh", "emg_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -ftz=true: FP32 denormals flush to zero (the data never come near 1e-38).
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-ftz=true", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3"]


# Build variants, selected by the environment variable EMG_BUILD_VARIANT; each
# builds into its own directory under _lib/.  "boundscheck" adds the index
# checks of the kernels (emg_debug_bounds_errors reads what they record).
VARIANTS = {"": [], "boundscheck": ["-DEMG_BOUNDS_CHECK"]}


def variant() -> str:
    v = os.environ.get("EMG_BUILD_VARIANT", "")
    if v not in VARIANTS:
        raise RuntimeError(f"unknown EMG_BUILD_VARIANT {v!r}; known: {sorted(VARIANTS)}")
    return v


def out_dir() -> str:
    v = variant()
    return os.path.join(OUT_DIR, v) if v else OUT_DIR


def lib_path() -> str:
    return os.path.join(out_dir(), LIB_NAME)


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libemagpie.so")


def _digest(extra_flags) -> str:
    h = hashlib.sha256()
    for name in SOURCES + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    with open(os.path.join(ROOT, "include", "emagpie.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + CFLAGS + list(extra_flags)).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compiles the library if needed and returns its path.

    Extra nvcc flags come from ``extra_flags`` and the environment variable
    EMG_NVCC_EXTRA (whitespace-separated, e.g. tuning macros such as
    -DEMG_UPDATE_GROUP=8); both are part of the build stamp.
    """
    extra_flags = list(extra_flags) + os.environ.get("EMG_NVCC_EXTRA", "").split() + VARIANTS[variant()]
    odir = out_dir()
    os.makedirs(odir, exist_ok=True)
    stamp = os.path.join(odir, "build.sha256")
    digest = _digest(extra_flags)
    if not force and os.path.exists(lib_path()) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return lib_path()
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(odir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *ARCH, *CFLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    tmp = lib_path() + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib_path())
    with open(stamp, "w") as f:
        f.write(digest)
    return lib_path()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
