"""In-tree build of the CUDA library libpccp.so for sm_103a (nvcc, no cmake).

The library is the product: the Python binding loads it and nothing else
computes the method.  Built artefacts go to paper_2207_12116_gb300/_build/
(git-ignored)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpccp.so")
SOURCES = [os.path.join(CSRC, "pccp.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "pccp_device.cuh"), os.path.join(CSRC, "k_propagate.cuh"),
                  os.path.join(CSRC, "pccp_noalloc.inc"),
                  os.path.join(CSRC, "pccp_batch.inc"), os.path.join(CSRC, "k_solve_eps.cuh"),
                  os.path.join(ROOT, "include", "pccp.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and not stale():
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-Xptxas", "-v" if verbose else "-O3", *SOURCES, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
