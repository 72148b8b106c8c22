"""In-tree build of libhpx.so (sm_103a) with nvcc: every translation unit is
compiled in parallel, then linked into paper_1904_10514_gb300/libhpx.so."""

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhpx.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
SOURCES = ["plan_math.cpp", "capi.cu", "k_ring.cu", "k_nufft.cu", "k_dense.cu", "k_rot.cu", "k_cl.cu", "k_adjoint.cu", "k_fused.cu", "k_fused_tc.cu", "group.cu", "k_cg.cu", "noalloc.cu", "k_nufft2.cu", "k_healpix.cu"]


def _compile(src, extra):
    obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC, "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17",
           "-Xcompiler", "-fPIC,-fopenmp", "-I" + CSRC] + extra
    if src.endswith(".cu"):
        cmd += ARCH + ["-lineinfo"]
    else:
        cmd = [NVCC, "-x", "c++"] + cmd[1:]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj, r.stderr


def build(verbose=False, extra=()):
    os.makedirs(OUT, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra)), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            if err.strip():
                sys.stderr.write(err)
    cmd = [NVCC, "-shared", "-o", LIB] + objs + ARCH + ["-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (r.stdout, r.stderr))
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(verbose=v or bool(extra), extra=extra))
