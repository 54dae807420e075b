"""Build liblbm.so in-tree for GB300 (sm_103a).

Host sources compile with g++ and the CUDA kernels with nvcc, in parallel;
nvcc links the shared library against the shared CUDA runtime.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "liblbm.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_SRC = ["geometry.cpp", "mesh.cpp", "turbulence.cpp", "friction.cpp", "api.cpp"]
CUDA_SRC = ["kernels.cu", "mlp.cu"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "lbm.h"))
    return files


def up_to_date():
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force=False, verbose=False, extra_nvcc=()):
    if not force and up_to_date():
        return OUT
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I" + os.path.join(cuda, "include"), "-I" + CSRC]
    jobs = []
    for s in HOST_SRC:
        o = os.path.join(BUILD, s + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-Wall", "-c", os.path.join(CSRC, s), "-o", o] + inc)
    for s in CUDA_SRC:
        o = os.path.join(BUILD, s + ".o")
        jobs.append([nvcc] + ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-c",
                                     os.path.join(CSRC, s), "-o", o] + inc + list(extra_nvcc))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(BUILD, s + ".o") for s in HOST_SRC + CUDA_SRC]
    tmp = OUT + ".tmp.%d" % os.getpid()
    run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-Xcompiler", "-pthread", "-o", tmp] + objs + ["-lpthread"])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_nvcc=["-Xptxas", "-v"] if "--ptxas" in sys.argv else ()))
