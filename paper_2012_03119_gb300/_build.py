"""In-tree build of libgss.so for sm_103a (nvcc, one TU per kernel file, compiled in parallel)."""
from __future__ import annotations

import fcntl
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
# GSS_DEBUG_BOUNDS=1 selects a separate, bounds-checked build (the kernels check every index
# they gather with and count violations instead of reading out of range).
BOUNDS = os.environ.get("GSS_DEBUG_BOUNDS", "") not in ("", "0")
OUT_DIR = os.path.join(PKG, "_build_bounds" if BOUNDS else "_build")
LIB = os.path.join(PKG, "libgss_bounds.so" if BOUNDS else "libgss.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(ROOT, "include", "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile every .cu under csrc/ for sm_103a and link libgss.so next to this file."""
    os.makedirs(OUT_DIR, exist_ok=True)
    with open(os.path.join(OUT_DIR, "build.lock"), "w") as lf:
        fcntl.flock(lf, fcntl.LOCK_EX)
        if not force and up_to_date():
            return LIB
        flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
        if BOUNDS:
            flags += ["-DGSS_DEBUG_BOUNDS"]
        if ptxas_verbose:
            flags += ["-Xptxas", "-v"]

        def compile_one(src: str) -> tuple[str, str]:
            obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
            r = subprocess.run([NVCC, *flags, "-c", src, "-o", obj], capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            return obj, r.stderr

        with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            results = list(ex.map(compile_one, _sources()))
        if verbose or ptxas_verbose:
            for _, log in results:
                sys.stderr.write(log)
        tmp = LIB + f".tmp{os.getpid()}"
        r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv)
    print(LIB)
