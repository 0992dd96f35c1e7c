"""Build libqcd_gb300.so in-tree with nvcc for sm_103a.

Each .cu translation unit is compiled to an object in parallel, then all are
linked into one shared library with a plain C ABI (include/qcd_gb300.h).
No torch headers are involved, so a build takes seconds per file.
"""

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB_NAME = "libqcd_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def lib_path():
    return os.path.join(BUILD, LIB_NAME)


def _compile(nvcc, src, obj, extra):
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
           "--expt-relaxed-constexpr", *extra, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{res.stdout}\n{res.stderr}")
    return res.stderr


def build(verbose=False, ptxas_info=False, force=False):
    """Compile every kernel source and link the shared library; returns its path.
    Concurrent callers (several ranks on one node) serialise on a lock file, so
    only the first compiles and the others find the library up to date."""
    os.makedirs(BUILD, exist_ok=True)
    import fcntl
    with open(os.path.join(BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            return _build_locked(verbose, ptxas_info, force)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(verbose, ptxas_info, force):
    nvcc = nvcc_path()
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(INCLUDE, "qcd_gb300.h"))
    newest_dep = max(os.path.getmtime(h) for h in headers)
    out = lib_path()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    objs = []
    jobs = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        for src in srcs:
            obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            stale = (force or ptxas_info or not os.path.exists(obj)
                     or os.path.getmtime(obj) < max(os.path.getmtime(src), newest_dep))
            if stale:
                jobs.append((src, ex.submit(_compile, nvcc, src, obj, extra)))
        for src, fut in jobs:
            log = fut.result()
            if verbose and log:
                sys.stderr.write(f"--- {os.path.basename(src)}\n{log}")
    if jobs or not os.path.exists(out):
        cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", out, "-lcudart"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    return out


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv, force="--force" in sys.argv))
