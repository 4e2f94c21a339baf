"""In-tree build of the package's native libraries.

* ``_build/libswgb.so``: the CUDA library behind ``include/swgb.h`` (host
  C-ABI + sm_103a kernels), compiled by nvcc for ``sm_103a`` only;
* ``_build/libswgb_workload.so``: the synthetic workload generator (plain C).

Both are rebuilt when a source is newer than the library.  Nothing here is
imported by the kernels' host code; it only runs compilers.
"""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")

SWGB_LIB = os.path.join(OUT, "libswgb.so")
WORKLOAD_LIB = os.path.join(OUT, "libswgb_workload.so")

CUDA_SOURCES = ["swgb_api.cu", "swgb_kernels.cu", "swgb_search.cu", "swgb_filter.cu",
                "swgb_server.cu"]
CUDA_HEADERS = ["swgb_internal.cuh", "swgb_host.cuh", "swgb_lane.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def swgb_commands(extra_flags=()):
    """nvcc commands: one object per translation unit, then the link."""
    nvcc = _nvcc()
    objs, cmds = [], []
    for src in CUDA_SOURCES:
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC,
                     *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj])
    link = [nvcc, *ARCH, "-shared", "-o", SWGB_LIB, *objs]
    return cmds, link


def build_swgb(force=False, verbose=False, extra_flags=()):
    """Compiles libswgb.so for sm_103a (translation units in parallel)."""
    sources = [os.path.join(CSRC, s) for s in CUDA_SOURCES + CUDA_HEADERS]
    sources.append(os.path.join(INCLUDE, "swgb.h"))
    if not force and not extra_flags and not _stale(SWGB_LIB, sources):
        return SWGB_LIB
    os.makedirs(OUT, exist_ok=True)
    cmds, link = swgb_commands(extra_flags)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for c in cmds]
    failed = []
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if verbose or p.returncode:
            print(out.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(c))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    subprocess.run(link, check=True)
    return SWGB_LIB


def build_workload(force=False):
    """Compiles libswgb_workload.so with gcc."""
    src = os.path.join(CSRC, "workload_gen.c")
    if not force and not _stale(WORKLOAD_LIB, [src]):
        return WORKLOAD_LIB
    os.makedirs(OUT, exist_ok=True)
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-Wall",
                    "-o", WORKLOAD_LIB, src, "-lm"], check=True)
    return WORKLOAD_LIB


def build_all(force=False, verbose=False):
    return build_swgb(force, verbose), build_workload(force)
