"""Build libcos.so (the CUDA kernels and their C ABI) in-tree for sm_103a."""
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libcos.so")
# measurement and verification instruments for the benchmark and the tests (not part of libcos)
INSTR_LIB = os.path.join(PKG, "libcos_instr.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def instr_sources():
    return sorted(glob.glob(os.path.join(CSRC, "instr", "*.cu")))


def deps():
    return (sources() + instr_sources() + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(INSTR_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(INSTR_LIB))
    return all(os.path.getmtime(d) <= t for d in deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu file to an object in parallel (one nvcc per file), then link."""
    if not force and up_to_date():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    nvcc = os.environ.get("NVCC", "nvcc")
    objdir = os.path.join(ROOT, "_build", "libcos")
    os.makedirs(objdir, exist_ok=True)
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if verbose:
        flags.insert(0, "-Xptxas=-v")

    def compile_one(src):
        obj = os.path.join(objdir, os.path.splitext(os.path.basename(src))[0] + ".o")
        subprocess.check_call([nvcc, *flags, "-c", "-o", obj, src])
        return obj

    srcs, isrcs = sources(), instr_sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs) + len(isrcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs + isrcs))
    for target, o in ((LIB, objs[:len(srcs)]), (INSTR_LIB, objs[len(srcs):])):
        tmp = target + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *o, "-lcudart"])
        os.replace(tmp, target)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
