"""Builds the CUDA library libgp.so in-tree for sm_103a (B300) with nvcc, and
its checked variant libgp_checked.so (the same sources with -DGP_CHECKED: every
gathered index tested in-kernel before the access, see include/gp.h).

The library is one translation unit (csrc/gp_api.cu includes the kernel
headers).  It is rebuilt when any source under csrc/ or include/ is newer
than the library.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libgp.so")
LIB_CHECKED = os.path.join(HERE, "libgp_checked.so")  # -DGP_CHECKED: in-kernel index tests
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu*")) + glob.glob(os.path.join(ROOT, "include", "*.h")))


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in sources())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds libgp.so, or with checked=True libgp_checked.so (the same sources with -DGP_CHECKED)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not stale(lib):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr",
           "-I", os.path.join(ROOT, "include"),
           "-o", tmp, os.path.join(HERE, "csrc", "gp_api.cu"), "-lcudart"]
    if checked:
        cmd.insert(1, "-DGP_CHECKED")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
