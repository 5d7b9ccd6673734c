"""Build the CUDA library libfos.so in-tree for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked
into ``paper_2002_00250_gb300/libfos.so`` (CUDA runtime linked statically).
No cmake; a clean build takes well under a minute.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
SO = os.path.join(PKG, "libfos.so")
# the range-checked variant (every kernel index checked, violations recorded)
BUILD_BOUNDS = os.path.join(PKG, "_build_bounds")
SO_BOUNDS = os.path.join(PKG, "libfos_bounds.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                 "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]
# PBAS arithmetic must round every operation once (bit-exact contract).
PER_FILE = {"pbas.cu": ["--fmad=false"], "pbas_joint.cu": ["--fmad=false"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return os.path.getmtime(src) > t or any(os.path.getmtime(h) > t for h in _headers())


def _compile(src: str, verbose: bool, bounds: bool = False) -> str:
    obj = os.path.join(BUILD_BOUNDS if bounds else BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if not _stale(obj, path):
        return obj
    cmd = [nvcc(), "-c", path, "-o", obj + ".tmp"] + COMMON + PER_FILE.get(src, [])
    if bounds:
        cmd.append("-DFOS_DEBUG_BOUNDS")
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compile and link libfos.so (bounds: the range-checked libfos_bounds.so);
    returns its path."""
    bdir, so = (BUILD_BOUNDS, SO_BOUNDS) if bounds else (BUILD, SO)
    os.makedirs(bdir, exist_ok=True)
    if force:
        for f in os.listdir(bdir):
            os.remove(os.path.join(bdir, f))
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(os.cpu_count() or 8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, bounds), srcs))
    if (not os.path.exists(so) or force or
            any(os.path.getmtime(o) > os.path.getmtime(so) for o in objs)):
        # -ldl: the NVTX ranges look their collector up with dlopen
        cmd = [nvcc(), "-shared", "-o", so + ".tmp"] + ARCH + objs + ["-Xcompiler", "-fPIC", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(so + ".tmp", so)
    return so


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv))
