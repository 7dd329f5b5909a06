"""Build the CUDA library ``_native/libchemgb.so`` in-tree (sm_103a only).

Five translation units compiled in parallel: the host mechanism compiler and the load-balance planner
(C++), the C ABI with its small kernels, the forward (rate, Jacobian, integration) kernels and the
adjoint kernels (CUDA).  Called by ``__graft_entry__.build()``; also runnable as a script.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_native")
LIB = os.path.join(OUT, "libchemgb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(ROOT, "include", "chem.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    cu_flags = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                *inc]
    if ptxas_info:
        cu_flags += ["-Xptxas", "-v"]
    host = [NVCC, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-x", "c++", *inc]
    jobs = [
        [*host, "-c", os.path.join(CSRC, "compile.cpp"), "-o", os.path.join(OUT, "compile.o")],
        [*host, "-c", os.path.join(CSRC, "balance.cpp"), "-o", os.path.join(OUT, "balance.o")],
        [*cu_flags, "-c", os.path.join(CSRC, "capi.cu"), "-o", os.path.join(OUT, "capi.o")],
        [*cu_flags, "-c", os.path.join(CSRC, "kern_forward.cu"), "-o", os.path.join(OUT, "kern_forward.o")],
        [*cu_flags, "-c", os.path.join(CSRC, "kern_adjoint.cu"), "-o", os.path.join(OUT, "kern_adjoint.o")],
    ]

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or (ptxas_info and r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("compilation failed: " + " ".join(cmd))

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    run([NVCC, *ARCH, "-shared", "-o", tmp, *(os.path.join(OUT, f + ".o") for f in
                                              ("compile", "balance", "capi", "kern_forward", "kern_adjoint"))])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True, ptxas_info="-v" in sys.argv))
