"""Build libpifepic.so (CUDA, sm_103a) in-tree with nvcc.

Translation units are compiled in parallel.  The FP64 particle cycle and the
set-up kernels are compiled with --fmad=false so that their arithmetic follows
the fixed operation order the FP64 parity tests rely on; host code is compiled
with -ffp-contract=off for the same reason (injection rates).
"""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpifepic.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, extra flags)
UNITS = [
    ("setup.cu", ["--fmad=false"]),
    ("particles.cu", ["--fmad=false"]),
    ("particles_mixed.cu", []),
    ("field.cu", []),
    ("pcg_coop.cu", []),
    ("pcg_mg.cu", []),
    ("pcg_cluster.cu", []),
    ("batch.cu", []),
    ("capi.cu", ["--fmad=false"]),
]


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def build_library(verbose=False, jobs=None):
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()

    def compile_one(u):
        src, extra = u
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags() + extra
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=jobs or len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-lcuda"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(verbose=True))
