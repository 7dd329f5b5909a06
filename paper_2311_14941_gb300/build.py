"""Build the CUDA library ``_native/libchemgb.so`` in-tree (sm_103a only).

Translation units compiled in parallel: the host mechanism compiler, the load-balance planner and the
run-time specialisation (C++), the C ABI with its small kernels, the integration kernels of each
lane group and form (one warp, two warps, half a warp per cell), the rate and Jacobian kernels and the
adjoint kernels (CUDA).  The device headers of the integration kernels are embedded as text
(``_native/rtc_headers.inc``) for the run-time compiler.  Called by ``__graft_entry__.build()``; also
runnable as a script.
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
# kernel translation units besides capi.cu: the integration kernels per lane group, and the adjoint
# The integration kernels are held to 128 registers per thread: 16 warps per SM where shared memory allows
# it (small mechanisms), and no spills (ptxas -v).
REG_CAP = {f: ["-maxrregcount=128"] for f in ("kern_fwd_warp", "kern_fwd_warp_plain", "kern_fwd_pair", "kern_fwd_half")}
CUDA_UNITS = ("kern_fwd_warp", "kern_fwd_warp_plain", "kern_fwd_pair", "kern_fwd_half", "kern_rates",
              "kern_adjoint")
HOST_UNITS = ("compile", "balance", "specialize")
# device headers the run-time compiler sees, under the names integrate.cuh includes them by
RTC_HEADERS = ("mech.h", "elementary_tables.h", "scalar.cuh", "device.cuh", "integrate.cuh")
RTC_INC = os.path.join(OUT, "rtc_headers.inc")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(ROOT, "include", "chem.h")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _write_rtc_headers():
    names, texts = [], []
    for h in RTC_HEADERS:
        text = open(os.path.join(CSRC, h)).read()
        if ')CHEMRTC"' in text:
            raise RuntimeError(h + " contains the raw-string delimiter")
        names.append('"%s"' % h)
        texts.append('R"CHEMRTC(' + text + ')CHEMRTC"')
    body = ("// written by build.py from the device headers; not edited by hand\n"
            "static const char* const kRtcHeaderNames[] = {" + ", ".join(names) + "};\n"
            "static const char* const kRtcHeaderTexts[] = {\n" + ",\n".join(texts) + "};\n"
            "static const int kRtcHeaderCount = %d;\n" % len(RTC_HEADERS))
    if not os.path.exists(RTC_INC) or open(RTC_INC).read() != body:
        with open(RTC_INC, "w") as f:
            f.write(body)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    _write_rtc_headers()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", OUT]
    cu_flags = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                *inc]
    if ptxas_info:
        cu_flags += ["-Xptxas", "-v"]
    host = [NVCC, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-x", "c++", *inc]
    jobs = [
        *([*host, "-c", os.path.join(CSRC, f + ".cpp"), "-o", os.path.join(OUT, f + ".o")] for f in HOST_UNITS),
        [*cu_flags, "-c", os.path.join(CSRC, "capi.cu"), "-o", os.path.join(OUT, "capi.o")],
        *([*cu_flags, *REG_CAP.get(f, []), "-c", os.path.join(CSRC, f + ".cu"), "-o", os.path.join(OUT, f + ".o")]
          for f in CUDA_UNITS),
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
                                              (*HOST_UNITS, "capi", *CUDA_UNITS)), "-ldl"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True, ptxas_info="-v" in sys.argv))
