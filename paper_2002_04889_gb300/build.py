"""Build the CUDA library libvolna_gb.so in-tree (paper_2002_04889_gb300/_build).

nvcc for the kernels (one -gencode for sm_103a, -lineinfo), g++ for the host
C++; translation units compile in parallel.  The FP64 step kernels are built
with --fmad=false and all host code with -ffp-contract=off, so FP64 results
round exactly as the expressions are written.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libvolna_gb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _sources():
    cu = sorted(f for f in os.listdir(SRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(SRC) if f.endswith(".cpp"))
    hdr = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    hdr += [os.path.join(INC, f) for f in os.listdir(INC) if f.endswith(".h")]
    return cu, cpp, hdr


def _stale(srcs) -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(verbose: bool = False, force: bool = False) -> str:
    cu, cpp, hdr = _sources()
    all_src = [os.path.join(SRC, f) for f in cu + cpp] + hdr + [os.path.abspath(__file__)]
    if not force and not _stale(all_src):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = "nvcc"
    jobs = []
    objs = []
    for f in cu:
        obj = os.path.join(OUT, f + ".o")
        flags = [nvcc, "-c", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xptxas", "-v",
                 "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", INC, "-o", obj, os.path.join(SRC, f)]
        if f.endswith("_f64.cu"):
            flags.insert(2, "--fmad=false")
        if f.endswith("_f32.cu"):
            flags[2:2] = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
        jobs.append(flags)
        objs.append(obj)
    for f in cpp:
        obj = os.path.join(OUT, f + ".o")
        jobs.append(["g++", "-c", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fopenmp", "-Wall",
                     "-I", INC, "-I", os.path.join(cuda, "include"), "-o", obj, os.path.join(SRC, f)])
        objs.append(obj)
    procs = []
    for cmd in jobs:
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    logs = []
    failed = False
    for cmd, p in procs:
        out, _ = p.communicate()
        logs.append(out)
        if p.returncode != 0:
            failed = True
            sys.stderr.write(f"FAILED: {' '.join(cmd)}\n{out}\n")
    with open(os.path.join(OUT, "ptxas.log"), "w") as fh:
        fh.write("\n".join(logs))
    if failed:
        raise RuntimeError("volna_gb build failed")
    link = [nvcc, "-shared", *ARCH, "-o", LIB + ".tmp", *objs, "-Xcompiler", "-fopenmp", "-lgomp",
            "-cudart", "static"]
    if verbose:
        print(" ".join(link), file=sys.stderr)
    subprocess.run(link, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
