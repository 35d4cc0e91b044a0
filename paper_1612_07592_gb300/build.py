"""Build libpe.so (the CUDA library behind include/pe.h) in-tree for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpe.so")
SOURCES = ["api.cu", "kernels.cu", "kernels_paired.cu", "kernels_f64.cu", "kernels_pic.cu", "kernels_pair.cu",
           "kernels_bw.cu", "kernels_diag.cu", "tables.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]
# single-precision division and square root at 2-ulp accuracy in the kernels (the FP64
# arithmetic is unaffected); the stated FP32 error budget includes this
KERNEL_FLAGS = ["-prec-div=false", "-prec-sqrt=false"]
# Every rounding as written where kernels must agree bit for bit: the FP64 step kernels (no
# multiply-add contraction: the plain and the persistent FP64 kernels round every operation
# alike, and the oracle builds the same way), and the paired FP32 kernels, whose single-run, batch
# and streaming instances inline the same emission branches (no contraction, IEEE division and
# square root: approximate forms lowered per instance made them differ in the last bit).
FILE_FLAGS = {"kernels_f64.cu": KERNEL_FLAGS + ["-fmad=false"],
              "kernels_paired.cu": ["-fmad=false", "-prec-div=true", "-prec-sqrt=true"]}


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False, lib: str | None = None, out_dir: str | None = None,
          defines: tuple = ()) -> str:
    """Compile the sources into `lib` (default: libpe.so beside the package).  `defines`
    are extra -D macros (e.g. PE_MIN_CTAS=3) for variant builds."""
    LIB_ = lib or LIB
    OUT = out_dir or OUT_DIR
    os.makedirs(OUT, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "pe.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB_) and os.path.getmtime(LIB_) >= newest:
        return LIB_
    nvcc = _nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(OUT, src + ".o")
        extra = FILE_FLAGS.get(src, KERNEL_FLAGS if src.startswith("kernels") else []) + \
            ["-D" + d for d in defines]
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, *FLAGS, "-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj] + ARCH
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_ + f".{os.getpid()}.tmp"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"], check=True)
    os.replace(tmp, LIB_)
    return LIB_


DEBUG_LIB = os.path.join(HERE, "libpe_debug.so")


def build_debug(force: bool = False) -> str:
    """The debug variant (PE_DEBUG: range checks of every table index, counted and clamped)."""
    return build(force=force, lib=DEBUG_LIB, out_dir=os.path.join(HERE, "_build_debug"), defines=("PE_DEBUG",))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
