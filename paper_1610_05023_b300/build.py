"""Builds libdgh.so in-tree with nvcc for sm_103a (B300), and the checked
variant libdgh_checked.so (-DDGH_CHECKED: index checks in the stage kernels)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libdgh.so")
LIB_CHECKED = os.path.join(HERE, "libdgh_checked.so")
SOURCES = ["api.cu", "refelem.cpp", "meshsetup.cpp"]
HEADERS = [os.path.join("..", "..", "include", "dgh.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    deps += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h", ".cu", ".cpp"))]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False, extra=(), checked=False):
    """Compile libdgh.so (or, with checked=True, libdgh_checked.so) if missing
    or older than its sources; return its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    cmd = [NVCC, "-O3", "-std=c++17", "-lineinfo", "-shared", "-Xcompiler", "-fPIC,-O3",
           *ARCH, "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64",
           *(["-DDGH_CHECKED"] if checked else []),
           "-o", lib + ".tmp", *[os.path.join(CSRC, f) for f in SOURCES], *extra]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True, cwd=CSRC)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [], checked="--checked" in sys.argv)
