"""Compile the CUDA/C++ sources under csrc/ into the in-tree shared library
`_lib/libmlbm.so` (sm_103a only).  Translation units compile in parallel;
a rebuild happens only when a source or header is newer than the library."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libmlbm.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
_LOCK = threading.Lock()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmlbm.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def common_flags():
    return ["-O3", "-lineinfo", "-std=c++17", ARCH, "-I", INCLUDE,
            "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off", "--expt-relaxed-constexpr"]


def build(force: bool = False, verbose: bool = False) -> str:
    with _LOCK:
        if not force and not _stale():
            return LIB
        os.makedirs(OUT_DIR, exist_ok=True)
        obj_dir = os.path.join(OUT_DIR, f"obj{os.getpid()}")
        os.makedirs(obj_dir, exist_ok=True)
        nv = nvcc()

        def compile_one(src):
            obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
            cmd = [nv, "-c", src, "-o", obj] + common_flags()
            if verbose:
                cmd += ["-Xptxas", "-v"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
            return obj, r.stderr

        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
            results = list(ex.map(compile_one, sources()))
        if verbose:
            for _, log in results:
                if log:
                    print(log)
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nv, "-shared", "-o", tmp] + [o for o, _ in results] + [ARCH, "-Xcompiler", "-fopenmp", "-lgomp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
        shutil.rmtree(obj_dir, ignore_errors=True)
        return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
