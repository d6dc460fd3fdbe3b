"""Build step of the CUDA library ``libssm.so`` (sm_103a), in-tree.

Each ``csrc/*.cu`` translation unit is compiled by nvcc in parallel for
``-gencode arch=compute_103a,code=sm_103a`` and the objects are linked into
``paper_2105_09688_gb300/libssm.so``.  Rebuilds only when a source or header is
newer than the library.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libssm.so")
# The debug build (-DSSM_CHECK_BOUNDS: kernels check the indices they take from data
# and report SSM_EBOUNDS instead of touching memory outside an array), separate objects.
LIB_CHECK = os.path.join(PKG, "libssm_check.so")
BUILD_CHECK = os.path.join(PKG, "_build_check")
INCLUDE = os.path.join(ROOT, "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _compile(src, extra, build_dir=BUILD):
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, extra=(), check_bounds=False):
    """Compile libssm.so (or, with check_bounds, the debug build libssm_check.so) if
    missing or stale; returns its path."""
    lib_path, build_dir = (LIB_CHECK, BUILD_CHECK) if check_bounds else (LIB, BUILD)
    extra = list(extra) + (["-DSSM_CHECK_BOUNDS"] if check_bounds else [])
    deps = _deps()
    if (not force and os.path.exists(lib_path)
            and os.path.getmtime(lib_path) >= max(os.path.getmtime(p) for p in deps)):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        outs = list(ex.map(lambda s: _compile(s, extra, build_dir), _sources()))
    if verbose:
        for _, err in outs:
            if err.strip():
                sys.stderr.write(err)
    tmp = lib_path + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in outs] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(force="--force" in sys.argv, verbose=v,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [], check_bounds="--check-bounds" in sys.argv))
