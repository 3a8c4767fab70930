"""Compile the CUDA library ``libpc.so`` in-tree for sm_103a (GB300).

Each translation unit is compiled in parallel with its own flags, then linked:
``collide.cu``, ``project.cu``, ``fx_deposit.cu`` and the other units that carry
double-float or bit-exact arithmetic without implicit fused multiply-add (bit-exact
FP64 contact solve and response; double-float arithmetic and exact digit splits
that place every FMA explicitly); the others with the default contraction.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libpc.so")
BUILD = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
UNITS = {
    "pc_abi.cu": [],
    "bin.cu": [],
    "collide.cu": ["-fmad=false"],
    "project.cu": ["-fmad=false"],
    "noalloc.cu": [],
    "mixed.cu": ["-fmad=false"],
    "tc_deposit.cu": [],
    "fx_deposit.cu": ["-fmad=false"],
    "adjoint.cu": ["-fmad=false"],
    "curved.cu": ["-fmad=false"],
    "nodal.cu": ["-fmad=false"],
    "coupling.cu": ["-fmad=false"],
}


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".cuh"))] + \
        [os.path.join(INCLUDE, f) for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force=False, verbose=False, extra=()):
    """Build libpc.so if any source is newer; returns its path. Raises on failure.

    Each process compiles into its own object folder and replaces the library
    atomically, so processes that build at the same time do not mix objects."""
    if not force and up_to_date():
        return LIB
    objdir = os.path.join(BUILD, "p%d" % os.getpid())
    os.makedirs(objdir, exist_ok=True)
    try:
        return _compile_and_link(objdir, verbose, extra)
    finally:
        shutil.rmtree(objdir, ignore_errors=True)


def _compile_and_link(objdir, verbose, extra):
    nvcc = _nvcc()
    procs = []
    objs = []
    for unit, flags in UNITS.items():
        obj = os.path.join(objdir, unit.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + COMMON + list(flags) + list(extra) + ["-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    errors = []
    for unit, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append("%s:\n%s" % (unit, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed\n" + "\n".join(errors))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
