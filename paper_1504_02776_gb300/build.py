"""Builds libmcv.so (the CUDA library behind include/mcv.h) in-tree, for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one shared library
with the CUDA runtime linked statically.  Nothing is installed outside the package folder.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmcv.so")
SOURCES = ["mcv_fp32.cu", "mcv_fp64.cu", "mcv_fp32_ev.cu", "mcv_fp64_ev.cu", "mcv_fp32_aux.cu",
           "mcv_fp64_aux.cu", "mcv_batch_fp32.cu", "mcv_batch_fp64.cu", "mcv_batch_fp32_ev.cu",
           "mcv_batch_fp64_ev.cu", "mcv_misc.cu", "mcv_api.cu", "mcv_batch.cu", "mcv_noalloc.cu",
           "mcv_phonon.cu", "mcv_bragg.cu"]
# per-file flags: the FP64 kernels round every operation separately (no FMA contraction)
_F64 = ["-fmad=false"]
_F32 = ["-prec-div=false", "-prec-sqrt=false"]
FILE_FLAGS = {f: (_F64 if "fp64" in f else _F32) for f in SOURCES if "_fp" in f or f.startswith("mcv_fp")}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "mcv.h"))
    return max(os.path.getmtime(f) for f in files)


def build(force=False, verbose=False, extra_flags=()):
    """Compile and link libmcv.so; returns its path.  Skipped when up to date."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + FLAGS + FILE_FLAGS.get(src, []) + list(extra_flags) + [
            "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for obj, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
