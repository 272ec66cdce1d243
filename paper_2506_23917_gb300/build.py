"""Build libsp.so (the CUDA library) in-tree for GB300 (sm_103a).

Each translation unit is compiled by nvcc in parallel and linked into
paper_2506_23917_gb300/libsp.so.  Only one -gencode target is built.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsp.so")
ROOT = os.path.dirname(HERE)
# (source, object, extra flags): sp_kern.cu is compiled once per precision
# mode.  The FP64 mode is compiled without FMA contraction (-fmad=false), so
# that every product and sum rounds as in the oracle (built with
# -ffp-contract=off) and no cell index or accept decision can differ by a
# fused rounding.
KERN = "sp_kern.cu"
SOURCES = [
    ("sp_api.cu", "sp_api.o", []),
    ("sp_common.cu", "sp_common.o", []),
    ("sp_noalloc.cu", "sp_noalloc.o", []),
    (KERN, "sp_kern_f64.o", ["-DSP_KT=double", "-DSP_KA=double", "-DSP_TAG=f64", "-fmad=false"]),
    (KERN, "sp_kern_f32.o", ["-DSP_KT=float", "-DSP_KA=double", "-DSP_TAG=f32"]),
    (KERN, "sp_kern_f32c.o", ["-DSP_KT=float", "-DSP_KA=float", "-DSP_TAG=f32c"]),
]
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code without FMA contraction (as the oracle): the O-grid's node
# coordinates and face lines, built on the host, must match the oracle's.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr", f"-I{os.path.join(ROOT, 'include')}"]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "sp.h"))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra=None) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or [])

    def cc(item):
        src, o, flags = item
        obj = os.path.join(BUILD, o)
        cmd = [NVCC, *ARCH, *FLAGS, *flags, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(cc, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(force="--force" in sys.argv, verbose=v,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
