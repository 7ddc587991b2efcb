"""Build libmpw.so (the C ABI of include/mpw.h) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into
``paper_2002_00088_gb300/libmpw.so``.  Host code is compiled with
``-ffp-contract=off`` so that the FP64 patch maps (and therefore the cover
flags) round the same way on every host architecture.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(PKG, "libmpw.so")
SOURCES = ["mpw_api.cu", "mpw_kernels.cu", "mpw_rhs.cu", "mpw_rhs32.cu", "mpw_shell.cu", "mpw_fill.cu", "mpw_noalloc.cu",
           "mpw_conv.cu", "mpw_surrogate.cu"]
GENCODE = "arch=compute_103a,code=sm_103a"


def nvcc_path() -> str:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmpw")
    return nvcc


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    inc = os.path.join(ROOT, "include")
    files += [os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h")]
    return files


def build_library(force: bool = False, verbose: bool = False) -> str:
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(f) for f in _inputs())):
        return LIB_PATH
    os.makedirs(BUILD, exist_ok=True)
    nvcc = nvcc_path()
    common = [nvcc, "-O3", "-std=c++17", "-gencode", GENCODE, "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(ROOT, "include")]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            print(log)
    objs = [o for o, _ in results]
    tmp = LIB_PATH + ".tmp"
    r = subprocess.run([nvcc, "-shared", "-gencode", GENCODE, "-o", tmp] + objs + ["-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of libmpw.so failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    import sys
    print(build_library(force=True, verbose="-v" in sys.argv))
