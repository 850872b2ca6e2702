"""Build libimex.so in-tree for sm_103a (host setup in C++, kernels in CUDA).

    python -m paper_2310_14712_gb300.build [-v] [--ptxas-info]

Three translation units are compiled in parallel (g++ for the host setup,
nvcc for the step kernels with the C-ABI and for the FP64 pipe probe) and linked with nvcc into
paper_2310_14712_gb300/libimex.so.  Object files go to
paper_2310_14712_gb300/_build/.  No GPU is needed to build.
"""
import os
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libimex.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _run(cmd, results, key, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    p = subprocess.run(cmd, capture_output=True, text=True)
    results[key] = p


def build(verbose=False, ptxas_info=False):
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17"]
    cu = [nvcc, *ARCH, "-lineinfo", *common, "-Xcompiler", "-fPIC", "-c",
          os.path.join(CSRC, "imex.cu"), "-o", os.path.join(OUT, "imex.o")]
    if ptxas_info:
        cu.insert(1, "-Xptxas=-v")
    probe = [nvcc, *ARCH, "-lineinfo", *common, "-Xcompiler", "-fPIC", "-c",
             os.path.join(CSRC, "probe.cu"), "-o", os.path.join(OUT, "probe.o")]
    cpp = ["g++", *common, "-fPIC", "-pthread", "-Wall", "-Wno-unused-variable", "-c",
           os.path.join(CSRC, "setup.cpp"), "-o", os.path.join(OUT, "setup.o")]
    results = {}
    threads = [threading.Thread(target=_run, args=(cmd, results, k, verbose))
               for k, cmd in (("cu", cu), ("probe", probe), ("cpp", cpp))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for k in ("cu", "probe", "cpp"):
        r = results[k]
        if r.returncode != 0 or (verbose and (r.stdout or r.stderr)) or (ptxas_info and k == "cu"):
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"compilation of {k} failed")
    link = [nvcc, *ARCH, "-shared", os.path.join(OUT, "imex.o"), os.path.join(OUT, "probe.o"),
            os.path.join(OUT, "setup.o"),
            "-o", LIB + ".tmp", "-lpthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, ptxas_info="--ptxas-info" in sys.argv)
    print(LIB)
