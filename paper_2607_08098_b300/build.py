"""Builds libevis.so in place with nvcc for sm_103a (no GPU needed to compile)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libevis.so")
MANIFEST = LIB + ".sources"   # the translation units of the last link, one name per line

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no fused multiply-add contraction anywhere; every float operation of the
# method is one rounded binary32 operation (bit-exact against an IEEE host).
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
                     "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libevis.so cannot be built")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(INCLUDE, "evis.h")]


def _newest(paths) -> float:
    return max(os.path.getmtime(p) for p in paths)


def _manifest() -> str:
    return "".join(os.path.basename(s) + "\n" for s in sources())


def _stale() -> bool:
    """The library is out of date when a source or header is newer, or when the set of
    translation units differs from the one it was linked from (a unit added or removed: a
    removed one's kernels would otherwise stay in a library newer than every source)."""
    if not os.path.exists(LIB) or not os.path.exists(MANIFEST):
        return True
    with open(MANIFEST) as f:
        if f.read() != _manifest():
            return True
    return _newest(sources() + _headers()) > os.path.getmtime(LIB)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every .cu under csrc/ (in parallel; an object is rebuilt when its source or
    any header is newer) and link libevis.so (static CUDA runtime)."""
    if not force and not _stale():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    hdr_t = _newest(_headers())
    jobs, objs = [], []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or ptxas_info or not os.path.exists(obj) or \
                os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_t):
            cmd = [cc] + NVCC_FLAGS + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", src, "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        return subprocess.run(cmd, capture_output=True, text=True)

    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as pool:
        results = list(pool.map(run, jobs))
    for cmd, r in zip(jobs, results):
        sys.stderr.write(r.stderr if (verbose or ptxas_info or r.returncode) else "")
        if r.returncode:
            raise subprocess.CalledProcessError(r.returncode, cmd, r.stdout, r.stderr)
    tmp = LIB + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    with open(MANIFEST + ".tmp", "w") as f:
        f.write(_manifest())
    os.replace(MANIFEST + ".tmp", MANIFEST)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas-info" in sys.argv)
    print(LIB)
