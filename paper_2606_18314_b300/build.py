"""Build libcert.so in-tree for sm_103a with nvcc (no JIT, no torch extension).

    python -m paper_2606_18314_b300.build [--force] [--verbose] [--debug]

--debug builds libcert_debug.so: the same sources with -DCERT_DEBUG_BOUNDS,
whose kernels check the indices the release build relies on by construction
and latch CERT_EINTERNAL on a violation (load it with CERT_LIB_VARIANT=debug).
"""
from __future__ import annotations

import concurrent.futures
import glob
import hashlib
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libcert.so")
LIB_DEBUG = os.path.join(HERE, "libcert_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC,-O2",
           "-shared", "-cudart=static", "--expt-relaxed-constexpr"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h"))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
                  glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h")))


def fingerprints() -> dict:
    """Per translation unit: the first 16 hex digits of the SHA-256 of its
    source and every header, in a fixed order.  The library reports them
    (cert_source_fingerprint), so a measurement taken on one build of a kernel
    can be told apart from the build that is running."""
    hh = hashlib.sha256()
    for h in headers():
        hh.update(os.path.basename(h).encode() + b"\0" + open(h, "rb").read())
    out = {}
    for src in sources():
        d = hh.copy()
        d.update(os.path.basename(src).encode() + b"\0" + open(src, "rb").read())
        out[os.path.splitext(os.path.basename(src))[0]] = d.hexdigest()[:16]
    return out


def fingerprint_defines() -> list:
    return [f"-DCERT_FP_{unit.upper()}=\"{fp}\"" for unit, fp in sorted(fingerprints().items())]


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in deps())


def _compile(nvcc, src, obj, extra, verbose):
    cmd = [nvcc, *ARCH, *[f for f in NVFLAGS if f not in ("-shared", "-cudart=static")], *extra,
           "-I", os.path.join(os.path.dirname(HERE), "include"), "-c", "-o", obj, src]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return subprocess.run(cmd, capture_output=True, text=True), cmd


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile every source to an object in parallel (one nvcc each; no
    relocatable device code crosses files), then link the shared library."""
    lib = LIB_DEBUG if debug else LIB
    if not force and not stale(lib):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    extra = (["-DCERT_DEBUG_BOUNDS"] if debug else []) + fingerprint_defines()
    srcs = sources()
    with tempfile.TemporaryDirectory(prefix="certbuild_") as tmp:
        objs = [os.path.join(tmp, os.path.basename(f) + ".o") for f in srcs]
        with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
            results = list(ex.map(lambda so: _compile(nvcc, so[0], so[1], extra, verbose), zip(srcs, objs)))
        for r, cmd in results:
            if verbose:
                print(" ".join(cmd), flush=True)
                sys.stdout.write(r.stdout + r.stderr)
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise subprocess.CalledProcessError(r.returncode, cmd)
        link = [nvcc, *ARCH, "-shared", "-cudart=static", "-Xcompiler", "-fPIC", "-o", lib + ".tmp", *objs]
        subprocess.run(link, check=True)
        os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, debug="--debug" in sys.argv))
