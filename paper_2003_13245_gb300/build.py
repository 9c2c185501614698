"""Build step of libtdmrg.so: nvcc for sm_103a, one object per translation unit, in parallel.

The library is built in-tree (``paper_2003_13245_gb300/libtdmrg.so``) so that the Python
binding loads exactly the file compiled here."""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libtdmrg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["kernels_f64.cu", "qr_blocked.cu", "kernels_tc.cu", "bond_krylov.cu",
              "lanczos_step.cu", "engine.cu", "step_adjoint.cu", "capi.cu", "noalloc.cu",
              "fgr.cu"]
CXX_SOURCES = ["model.cpp", "small_exp.cpp"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtdmrg")


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libtdmrg.so."""
    os.makedirs(OBJ, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "tdmrg.h"))
    jobs = []
    objs = []
    for src in CU_SOURCES + CXX_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, os.path.splitext(src)[0] + ".o")
        objs.append(o)
        if force or _newer(o, [s] + headers):
            cmd = [nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                                   "-I" + os.path.join(ROOT, "include"), "-c", s, "-o", o]
            if src.endswith(".cpp"):
                cmd = [nvcc, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-x", "c++",
                       "-I" + os.path.join(ROOT, "include"), "-c", s, "-o", o]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _newer(LIB, objs):
        run([nvcc, "-shared"] + ARCH + ["-o", LIB] + objs +
            ["-lcudart", "-Xlinker", "--no-undefined"])
    return LIB


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
