"""Compile libps.so (CUDA, sm_103a) in-tree with nvcc.

The translation units that form setup-phase quantities feeding integer
decisions (aggregation) are compiled with --fmad=false so that every a*b+c is
rounded twice, as in a plain IEEE evaluation of the same formula.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libps.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["util.cu", "gen.cu", "amg_setup.cu", "vcycle.cu", "flow_setup.cu", "flow_apply.cu", "krylov.cu",
           "api.cu", "noalloc.cu", "serve.cu", "rbm_setup.cu", "rbm_apply.cu", "newton.cu"]
NO_FMA = {"amg_setup.cu", "flow_setup.cu", "gen.cu", "rbm_setup.cu"}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(INCLUDE, "ps.h"))
    objs, jobs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [path] + headers + [__file__]):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "--extended-lambda", "-Xcompiler", "-fPIC",
                   "-I" + INCLUDE, "-c", path, "-o", obj]
            if src in NO_FMA:
                cmd.insert(1, "--fmad=false")
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, res):
            if verbose or r.returncode:
                print(" ".join(cmd))
                print(r.stdout, r.stderr)
            if r.returncode:
                raise RuntimeError("nvcc failed for %s" % cmd[-3])
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + ".%d.tmp" % os.getpid()
        # the CUDA runtime is linked shared, so that a process that already uses it (PyTorch) and the library
        # share one runtime instance: host memory pinned through the other's allocator is then seen as pinned
        # here too, and host-pointer copies take the direct DMA path
        cudalib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath," + cudalib, "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            print(r.stdout, r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
