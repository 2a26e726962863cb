"""Builds the CUDA library libabm_gb300.so in-tree for sm_103a (GB300).

Each translation unit in csrc/ is compiled in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a), then linked into one shared
library next to this file.  The same sources compiled with -DABM_CHECKED
give libabm_gb300_checked.so, whose kernels check every layout-derived index
against its buffer and report ABM_ERR_BOUNDS instead of accessing outside
it.  Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libabm_gb300.so")
CHECKED_LIB = os.path.join(HERE, "libabm_gb300_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
              "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libabm_gb300.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Builds both libraries (every translation unit of both in one parallel
    pool); returns the path of the plain one."""
    targets = [(lib, flags, sub) for lib, flags, sub in ((LIB, [], "_build"), (CHECKED_LIB, ["-DABM_CHECKED"],
                                                                                    "_build_checked"))
               if force or not up_to_date(lib)]
    if not targets:
        return LIB
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    jobs = []
    for lib, flags, sub in targets:
        bdir = os.path.join(HERE, sub)
        os.makedirs(bdir, exist_ok=True)
        jobs += [(lib, flags, src, os.path.join(bdir, os.path.basename(src)[:-3] + ".o")) for src in sources()]

    def compile_one(job):
        lib, flags, src, obj = job
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *flags, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)} {' '.join(flags)}:\n{r.stderr}")
        return lib, obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose or ptxas_info:
        for _, _, err in results:
            if err:
                sys.stderr.write(err)
    for lib, _, _ in targets:
        objs = [o for l, o, _ in results if l == lib]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-Xlinker", "--no-undefined"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
