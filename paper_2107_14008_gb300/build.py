"""Build libpsr.so in-tree for sm_103a (GB300).

Each translation unit is compiled in parallel (nvcc for .cu, g++ for .cpp),
then linked with nvcc into ``paper_2107_14008_gb300/_build/libpsr.so``
(static CUDA runtime).  Run ``python -m paper_2107_14008_gb300.build``.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.environ.get("PSR_SRC_DIR") or os.path.join(HERE, "csrc")
OUT = os.environ.get("PSR_BUILD_DIR") or os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpsr.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--ftz=true",
              "--prec-div=true", "--prec-sqrt=true", "--fmad=true", "-Xptxas", "-v",
              "-I" + os.path.join(ROOT, "include")]
# -ffp-contract=off: the builder's FP64 box tests must round the same way on
# every host (gcc contracts a*b+c into an FMA by default on aarch64).
CXX_FLAGS = ["-O3", "-std=c++17", "-fPIC", "-pthread", "-Wall", "-Wno-unused-function",
             "-ffp-contract=off",
             "-I" + os.path.join(ROOT, "include")]
CU_SOURCES = ["p2p_fwd_f32.cu", "p2p_fwd_f32_sc.cu", "p2p_fwd_f32_pk.cu", "p2p_fwd_blk.cu", "p2p_fwd_f64.cu",
              "p2p_adj.cu", "capi.cu", "noalloc.cu", "devbuild.cu", "pm.cu", "fmm.cu"]
CXX_SOURCES = ["builder.cpp"]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _needs(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _headers():
    hs = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(ROOT, "include", "psr.h")]


def build(force=False, verbose=False):
    """Compile and link libpsr.so; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    hdrs = _headers()
    jobs = []
    for f in CU_SOURCES:
        src = os.path.join(SRC, f)
        obj = os.path.join(OUT, f + ".o")
        if force or _needs(obj, [src] + hdrs):
            extra = os.environ.get("PSR_NVCC_EXTRA", "").split()
            jobs.append(([nvcc] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj], obj))
    for f in CXX_SOURCES:
        src = os.path.join(SRC, f)
        obj = os.path.join(OUT, f + ".o")
        if force or _needs(obj, [src] + hdrs):
            jobs.append((["g++"] + CXX_FLAGS + ["-c", src, "-o", obj], obj))
    logs = []

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, r in ex.map(lambda j: run(j[0]), jobs):
            logs.append((cmd, r.stdout + r.stderr))
            if r.returncode != 0:
                raise RuntimeError("compile failed: %s\n%s" % (" ".join(cmd), r.stdout + r.stderr))
    with open(os.path.join(OUT, "ptxas.log"), "a") as f:
        for cmd, txt in logs:
            f.write(" ".join(cmd) + "\n" + txt + "\n")
    objs = [os.path.join(OUT, f + ".o") for f in CU_SOURCES + CXX_SOURCES]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp%d" % os.getpid()
        cudalib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + [
            "-lpthread", "-L" + cudalib, "-lcufft", "-Xlinker", "-rpath=" + cudalib]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s" % (" ".join(cmd), r.stdout + r.stderr))
        os.replace(tmp, LIB)
    if verbose:
        for cmd, txt in logs:
            print(" ".join(cmd[:1] + cmd[-3:]))
            print(txt)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
