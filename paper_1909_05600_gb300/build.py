"""Build libffm_gb300.so (sm_103a) in-tree with nvcc.

Each translation unit under csrc/ is compiled in parallel to an object file, then the
objects are linked into paper_1909_05600_gb300/libffm_gb300.so.  Host code is compiled
with -ffp-contract=off so that the FP64 arithmetic which decides the octree (bounding
cubes, admissibility offsets) rounds exactly as written.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libffm_gb300.so")
SOURCES = ["tree.cu", "tables.cu", "farfield.cu", "nearfield.cu", "ffm_api.cu", "noalloc.cu", "autotune.cu",
           "nufft.cu", "bem.cu"]
ARCH = os.environ.get("FFM_CUDA_ARCH", "103a")

NVCC_FLAGS = ["-gencode", "arch=compute_%s,code=sm_%s" % (ARCH, ARCH), "-O3", "-lineinfo", "-std=c++17",
              "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC,-ffp-contract=off", "-Xptxas", "-warn-spills",
              "-I", os.path.join(HERE, "..", "include")]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src, os.path.join(CSRC, "ffm_internal.cuh"), os.path.join(HERE, "..", "include", "ffm.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=()):
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(o, s):
            jobs.append([nvcc, *NVCC_FLAGS, *extra, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for msg in ex.map(run, jobs):
            if verbose and msg:
                print(msg, file=sys.stderr)
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    if jobs or force or not os.path.exists(LIB):
        tmp = LIB + ".tmp%d" % os.getpid()
        run([nvcc, "-shared", "-gencode", "arch=compute_%s,code=sm_%s" % (ARCH, ARCH), "-o", tmp, *objs,
             "-lcudart", "-lcufft", "-Xlinker", "-rpath,/usr/local/cuda/lib64"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
