"""In-tree build of the CUDA libraries for sm_103a (nvcc, no cmake).

libpccp.so is the product: the Python binding loads it and nothing else
computes the method.  libpccp_probe.so holds the roofline microbenchmarks
(include/pccp_probe.h).  Built artefacts go to paper_2207_12116_gb300/_build/
(git-ignored); the two libraries compile in parallel."""
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpccp.so")
PROBE_LIB = os.path.join(BUILD, "libpccp_probe.so")
SOURCES = [os.path.join(CSRC, "pccp.cu")]
PROBE_SOURCES = [os.path.join(CSRC, "roofline_probe.cu")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def deps():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(CSRC, "*.inc")) + glob.glob(os.path.join(ROOT, "include", "*.h")))


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in deps())


def _command(sources, out, verbose):
    return [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
            "-Xptxas", "-v" if verbose else "-O3", *sources, "-o", out]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile whichever library is missing or older than a source; returns
    the path of libpccp.so."""
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for sources, lib in ((SOURCES, LIB), (PROBE_SOURCES, PROBE_LIB)):
        if force or stale(lib):
            tmp = lib + f".{os.getpid()}.tmp"
            jobs.append((subprocess.Popen(_command(sources, tmp, verbose)), tmp, lib))
    failed = [lib for proc, _, lib in jobs if proc.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, f"nvcc for {', '.join(failed)}")
    for _, tmp, lib in jobs:
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
