"""Build libisg.so in-tree: nvcc for the sm_103a kernels and the C ABI, g++
(-ffp-contract=off) for the host FP64 arithmetic, linked with the static
CUDA runtime so that the library needs only the driver at run time.

    python -m paper_2503_14688_b300.build        # or __graft_entry__.build()
"""
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libisg.so")
CALIB_LIB = os.path.join(PKG, "libisg_calib.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["isg_kernels.cu", "isg_api.cu", "isg_noalloc.cu", "isg_ensemble.cu", "isg_server.cu",
              "isg_sw.cu", "isg_slab.cu"]
CPP_SOURCES = ["isg_host.cpp"]


def _sources():
    out = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    out.append(os.path.join(INCLUDE, "isg.h"))
    return out


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs = []
    inc = ["-I", INCLUDE, "-I", CSRC]
    for f in CU_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = [NVCC, "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", *inc, os.path.join(CSRC, f), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.run(cmd, check=True)
        objs.append(obj)
    for f in CPP_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-c", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
               *inc, "-I", os.path.join(CUDA_HOME, "include"), os.path.join(CSRC, f), "-o", obj]
        subprocess.run(cmd, check=True)
        objs.append(obj)
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.run([NVCC, "-shared", *ARCH, "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


def build_calib(force: bool = False) -> str:
    """Build the integer-throughput calibration kernels (libisg_calib.so), a
    measurement tool of the benchmark's roofline; not part of libisg."""
    src = os.path.join(CSRC, "isg_calib.cu")
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    if (not force and os.path.exists(CALIB_LIB)
            and all(os.path.getmtime(d) <= os.path.getmtime(CALIB_LIB) for d in deps)):
        return CALIB_LIB
    tmp = CALIB_LIB + ".tmp.%d" % os.getpid()
    subprocess.run([NVCC, "-shared", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
                    "-I", INCLUDE, "-I", CSRC, src, "-o", tmp], check=True)
    os.replace(tmp, CALIB_LIB)
    return CALIB_LIB


def clean():
    shutil.rmtree(BUILD, ignore_errors=True)
    for lib in (LIB, CALIB_LIB):
        if os.path.exists(lib):
            os.remove(lib)


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
