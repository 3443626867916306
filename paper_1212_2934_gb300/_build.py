"""Builds libff.so (the CUDA library behind include/ff.h) in-tree with nvcc.

The translation units are compiled in parallel for sm_103a only and linked
with the static CUDA runtime into paper_1212_2934_gb300/libff.so.  Objects go
to _build/ at the repository root.  A build is skipped when the library is
newer than every source and header.  The SIMT peak microbenchmark
(csrc/peak/simt_peak.cu, the roofline denominators of the arithmetic-bound
kernels) is built alongside it into libffpeak.so.
"""
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libff.so")
EXPORTS = os.path.join(CSRC, "libff.map")  # linker version script: only ff_* is exported
PEAK_SRC = os.path.join(CSRC, "peak", "simt_peak.cu")
PEAK_LIB = os.path.join(PKG, "libffpeak.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
           "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "ff.h"),
                                                                  EXPORTS, os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def _peak_up_to_date() -> bool:
    return (os.path.exists(PEAK_LIB)
            and os.path.getmtime(PEAK_LIB) >= max(os.path.getmtime(PEAK_SRC),
                                                   os.path.getmtime(os.path.abspath(__file__))))


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link libff.so (and libffpeak.so); returns the path of libff.so."""
    peak = None
    if force or not _peak_up_to_date():
        peak_tmp = PEAK_LIB + ".tmp%d" % os.getpid()
        peak = (peak_tmp, subprocess.Popen(
            [nvcc(), *ARCH, *NVFLAGS, "-shared", "-o", peak_tmp, PEAK_SRC, "-cudart", "static"],
            stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    if not force and up_to_date():
        _finish_peak(peak)
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.splitext(os.path.basename(src))[0] + ".o")
        objs.append(obj)
        cmd = [cc, *ARCH, *NVFLAGS, "-c", src, "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if out and (verbose or ptxas_info or p.returncode):
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed on: " + ", ".join(failed))
    _finish_peak(peak)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static",
           "-Xlinker", "--version-script=" + EXPORTS]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def _finish_peak(peak):
    if peak is None:
        return
    tmp, p = peak
    out, _ = p.communicate()
    if p.returncode:
        sys.stderr.write(out.decode(errors="replace"))
        raise RuntimeError("nvcc failed on: " + PEAK_SRC)
    os.replace(tmp, PEAK_LIB)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                ptxas_info="--ptxas" in sys.argv))
