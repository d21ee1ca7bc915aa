"""Compile libmbf.so in-tree for sm_103a (nvcc for .cu, g++ for .cpp, parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIBPATH = os.path.join(LIBDIR, "libmbf.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cpp")) + glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.hpp")) + glob.glob(
        os.path.join(os.path.dirname(HERE), "include", "*.h"))


def _cmd(src: str, obj: str):
    inc = [f"-I{CSRC}", f"-I{os.path.join(os.path.dirname(HERE), 'include')}", f"-I{CUDA_HOME}/include"]
    if src.endswith(".cu"):
        return [f"{CUDA_HOME}/bin/nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                "--expt-relaxed-constexpr", "-Xptxas", "-v", *inc, "-c", src, "-o", obj]
    return ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-fopenmp-simd", "-Wall", "-Wno-unused-function", *inc,
            "-c", src, "-o", obj]


def build(verbose: bool = False, force: bool = False) -> str:
    """Build (or reuse) the shared library; returns its path.  Raises on failure."""
    os.makedirs(os.path.join(LIBDIR, "obj"), exist_ok=True)
    srcs = _sources()
    hdr_t = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    jobs = []
    for s in srcs:
        obj = os.path.join(LIBDIR, "obj", os.path.basename(s) + ".o")
        stale = force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(s), hdr_t)
        if stale:
            jobs.append((s, obj))
    logs = {}
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        futs = {ex.submit(subprocess.run, _cmd(s, o), capture_output=True, text=True): s for s, o in jobs}
        for fu in cf.as_completed(futs):
            r = fu.result()
            logs[futs[fu]] = r.stdout + r.stderr
            if r.returncode != 0:
                raise RuntimeError(f"compile failed: {futs[fu]}\n{r.stdout}\n{r.stderr}")
    if verbose:
        for s, log in logs.items():
            if log.strip():
                print(f"--- {os.path.basename(s)}\n{log}")
    objs = [os.path.join(LIBDIR, "obj", os.path.basename(s) + ".o") for s in srcs]
    if force or jobs or not os.path.exists(LIBPATH):
        cmd = ["g++", "-shared", "-o", LIBPATH, *objs, f"-L{CUDA_HOME}/lib64", "-lcudart", "-pthread",
               f"-Wl,-rpath,{CUDA_HOME}/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed\n{r.stdout}\n{r.stderr}")
    return LIBPATH


if __name__ == "__main__":
    print(build(verbose=True))
