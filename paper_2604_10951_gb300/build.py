"""Builds ``_build/libfss.so`` (sm_103a) from ``csrc/`` with nvcc, and the
check build ``_build/libfss_check.so`` (device-side index checks and
workspace canaries, ``-DFSS_CHECK_BOUNDS=1``), which the binding loads
instead when the environment sets ``FSS_CHECK_BOUNDS=1``.

Each translation unit compiles in parallel; the binning unit is compiled
with ``-fmad=false`` so its binary32 operation order is never fused.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfss.so")
LIB_CHECK = os.path.join(OUT_DIR, "libfss_check.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-I", INCLUDE, "-I", CSRC]
UNITS = {
    "api.cu": [],
    "project.cu": ["-fmad=false"],
    "sort.cu": [],
    "render_fwd.cu": [],
    "render_topk_f32.cu": [],
    "render_topk_bf16.cu": [],
    "render_full.cu": [],
    "render_bwd.cu": [],
    "loss.cu": [],
    "static_scratch.cu": [],
    "query.cu": [],
    "color.cu": [],
}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "fss.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _fresh(lib: str) -> bool:
    return os.path.exists(lib) and os.path.getmtime(lib) >= _sources_mtime()


def build(force: bool = False, verbose: bool = False, extra: list | None = None, check: bool = True) -> str:
    """Compile every unit (in parallel) and link the shared library, and
    with ``check`` the check build beside it (both in one pool of
    compiles).  Returns the release library's path."""
    variants = [(LIB, os.path.join(OUT_DIR, "rel"), [])]
    if check:
        variants.append((LIB_CHECK, os.path.join(OUT_DIR, "check"), ["-DFSS_CHECK_BOUNDS=1"]))
    todo = [v for v in variants if force or not _fresh(v[0])]
    if not todo:
        return LIB
    nvcc = _nvcc()
    extra = list(extra or [])

    def compile_one(job):
        name, obj_dir, flags = job
        obj = os.path.join(obj_dir, name.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *COMMON, *UNITS[name], *flags, *extra, "-c", os.path.join(CSRC, name), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    jobs = []
    for lib, obj_dir, flags in todo:
        os.makedirs(obj_dir, exist_ok=True)
        jobs += [(n, obj_dir, flags) for n in UNITS]
    jobs.sort(key=lambda j: -os.path.getsize(os.path.join(CSRC, j[0])))  # longest first
    workers = min(len(jobs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(compile_one, jobs))
    for lib, obj_dir, _ in todo:
        mine = [o for o in objs if os.path.dirname(o) == obj_dir]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *mine]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import time

    t = time.time()
    print(build(force="--force" in sys.argv, verbose=True, extra=[a for a in sys.argv[1:] if a != "--force"]))
    print(f"built in {time.time() - t:.1f}s")
