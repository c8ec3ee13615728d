"""Builds the RANC CUDA library ``_lib/libranc.so`` in-tree for sm_103a.

The translation units are compiled in parallel with nvcc and linked into one
shared library against the shared CUDA runtime (the one PyTorch also loads).
``build(debug=True)`` makes the same library with device-side range checks
(``-DRANC_DEBUG``) as ``_lib/libranc_debug.so``, for the tests that run the
kernels under those checks; ``build_all()`` makes both.
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
LIB_DEBUG = os.path.join(OUT_DIR, "libranc_debug.so")
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


def build(force=False, verbose=False, debug=False):
    """Compile (if stale) and return the path of ``libranc.so`` (with debug:
    ``libranc_debug.so``, the kernels' range checks compiled in)."""
    lib = LIB_DEBUG if debug else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _sources_mtime():
        return lib
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if debug:
        common += ["-DRANC_DEBUG"]
    tag = ("dbg." if debug else "") + str(os.getpid())
    objs = []

    def compile_one(unit):
        obj = os.path.join(OUT_DIR, unit.replace(".cu", f".{tag}.o"))
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
    tmp = lib + f".tmp{os.getpid()}"
    libdir = _cuda_lib_dir(nvcc)
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", f"-rpath={libdir}", "-L", libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, lib)
    return lib


def build_all(force=False):
    """Both libraries, compiled side by side; returns (release, debug) paths."""
    with cf.ThreadPoolExecutor(2) as ex:
        rel, dbg = ex.submit(build, force), ex.submit(build, force, False, True)
        return rel.result(), dbg.result()


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
