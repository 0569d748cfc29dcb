"""Build libgrmhd.so in-tree with nvcc for sm_103a (no CMake; translation units compiled in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgrmhd.so")
BUILD_BC = os.path.join(HERE, "_build_bc")
LIB_BC = os.path.join(BUILD_BC, "libgrmhd.so")
ROOT = os.path.dirname(HERE)
SOURCES = ["grmhd_api.cu", "grmhd_fp64.cu", "grmhd_mixed.cu", "grmhd_batch.cu", "grmhd_noalloc.cu", "grmhd_mlp.cu",
           "grmhd_mlp_train.cu", "grmhd_mlp_tc.cu", "grmhd_peaks.cu", "grmhd_mlp_train_tc.cu"]
# The all-FP64 stage kernels round every double operation separately, as the FP64 reference does.
PER_SOURCE_FLAGS = {"grmhd_fp64.cu": ["-fmad=false"]}
HEADERS = ["grmhd_device.cuh", "grmhd_kernels.cuh", "grmhd_launch.h", "grmhd_mlp.cuh", "grmhd_face_ct.cuh",
           "grmhd_mesh.cuh", "grmhd_mesh_host.h", "grmhd_batch_launch.cuh",
           "grmhd_scalar.cuh", "grmhd_tc.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgrmhd.so")
    return path


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), bounds_check: bool = False) -> str:
    """Build libgrmhd.so (returns its path). bounds_check=True builds the bounds-check variant instead
    (-DGRMHD_BOUNDS_CHECK, in its own folder): the stage kernels check every global index and record the first
    out-of-range one (grmhd_bounds_fault) without trapping; a testing build."""
    if bounds_check:
        return _build_into(BUILD_BC, LIB_BC, force, verbose, tuple(extra_flags) + ("-DGRMHD_BOUNDS_CHECK",))
    return _build_into(BUILD, LIB, force, verbose, tuple(extra_flags))


def _build_into(BUILD, LIB, force, verbose, extra_flags):
    os.makedirs(BUILD, exist_ok=True)
    deps_common = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "grmhd.h"),
                                                              os.path.abspath(__file__)]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + deps_common):
            cmd = [nvcc(), *ARCH, *FLAGS, *PER_SOURCE_FLAGS.get(src, []), *extra_flags, "-c", s, "-o", o]
            jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
