"""In-tree build of libhdgmg.so (sm_103a) with nvcc, one object per source in
parallel, then a shared link.  No torch or CMake involved."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhdgmg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["refelem.cpp", "eigbasis.cpp", "k_condense.cu", "k_mg.cu", "k_ctail.cu", "k_krylov.cu", "hdgmg_api.cu",
           "hdgmg_batch.cpp", "umesh_plan.cpp", "umesh.cu"]
# the unstructured plan takes integer decisions from fp64 comparisons: no
# floating-point contraction, so that every host decides alike
FILE_FLAGS = {"umesh_plan.cpp": ["-Xcompiler", "-ffp-contract=off"]}
# k_edge_inst.cu is built once per (real type, trace modes per edge), plus
# once per ND for the BF16-storage matvec
EDGE_UNITS = [(t, nd) for nd in range(2, 10) for t in ("double", "float", "bf16")]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            return cand
        raise RuntimeError("nvcc not found")
    return exe


def _compile(unit, extra):
    if isinstance(unit, tuple):
        real, nd = unit
        src = "k_edge_inst.cu"
        obj = os.path.join(BUILD, f"k_edge_{real}_{nd}.o")
        if real == "bf16":
            extra = ["-DHDGMG_BF16", "-DHDGMG_REAL=float", f"-DHDGMG_ND={nd}", *extra]
        else:
            extra = [f"-DHDGMG_REAL={real}", f"-DHDGMG_ND={nd}",
                     f"-DHDGMG_REAL_IS_DOUBLE={int(real == 'double')}", *extra]
    else:
        src = unit
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        extra = [*FILE_FLAGS.get(src, []), *extra]
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-O3", "-I", os.path.join(HERE, "..", "include"), *extra,
           "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "cu")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stderr}")
    return obj, res.stderr


def build(verbose=False, extra=()):
    os.makedirs(BUILD, exist_ok=True)
    units = list(SOURCES) + EDGE_UNITS
    # the widest edge units take longest: start them first
    units.sort(key=lambda u: -(u[1] if isinstance(u, tuple) else 4))
    workers = max(2, min(len(units), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda u: _compile(u, list(extra)), units))
    objs = [r[0] for r in results]
    if verbose:
        for _, err in results:
            if err.strip():
                print(err)
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", LIB + ".tmp", *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
