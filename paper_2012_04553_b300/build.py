"""Build the library (libpm_b300.so) in-tree with nvcc for sm_103a.

Usage: python paper_2012_04553_b300/build.py [--force] [-v] [--debug]
(run as a script: importing the package first would load the library it builds)

--debug builds libpm_b300_debug.so with PM_DEBUG defined: the kernels check
the indices they derive from data (list entries, shared and global counter
slots) before each access, skip an access that is out of range and set a
fault word that the host reports as an error.  The package loads it instead
of libpm_b300.so when the environment has PM_DEBUG=1.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpm_b300.so")
DEBUG_LIB = os.path.join(HERE, "libpm_b300_debug.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.hpp")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(ROOT, "include", "*.h")))


def needs_build(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in sources() + headers())


def build(force=False, verbose=False, debug=False):
    lib = DEBUG_LIB if debug else LIB
    if not force and not needs_build(lib):
        return lib
    objdir = os.path.join(HERE, "_build_debug" if debug else "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = []
    common = ["-O3", "-std=c++17", "-lineinfo", "-I", os.path.join(ROOT, "include"),
              "-Xcompiler", "-fPIC,-O3,-Wall"] + (["-DPM_DEBUG"] if debug else [])
    procs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [NVCC] + ARCH + common + ["-c", src, "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        else:
            cmd += ["-x", "c++"]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = False
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode())
        if p.returncode != 0:
            failed = True
    if failed:
        raise RuntimeError("nvcc compilation failed")
    tmp = lib + f".{os.getpid()}.tmp"
    subprocess.check_call([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
