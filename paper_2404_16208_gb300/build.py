"""Builds the RANC CUDA library ``_lib/libranc.so`` in-tree for sm_103a.

The translation units are compiled in parallel with nvcc and linked into one
shared library against the shared CUDA runtime (the one PyTorch also loads).
"""

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libranc.so")
UNITS = ("ranc_api.cu", "ranc_plain.cu", "ranc_batched.cu", "ranc_multi.cu", "ranc_xbar.cu", "ranc_mlp.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the RANC CUDA library cannot be built")


def _cuda_lib_dir(nvcc):
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _sources_mtime():
    inc = os.path.join(ROOT, "include")
    paths = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(inc, f) for f in os.listdir(inc)] + [__file__]
    return max(os.path.getmtime(p) for p in paths)


def build(force=False, verbose=False):
    """Compile (if stale) and return the path of ``libranc.so``."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    objs = []

    def compile_one(unit):
        obj = os.path.join(OUT_DIR, unit.replace(".cu", f".{os.getpid()}.o"))
        cmd = [nvcc] + common + ["-c", os.path.join(SRC, unit), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {unit}:\n{r.stderr[-4000:]}")
        if verbose:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + f".tmp{os.getpid()}"
    libdir = _cuda_lib_dir(nvcc)
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", f"-rpath={libdir}", "-L", libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link of libranc.so failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
