"""Build libafmm.so in-tree with nvcc for sm_103a (no torch extension machinery).

Each translation unit is compiled in parallel, then linked into one shared library next
to this file.  The arithmetic-pipe peak probes the benchmark uses (csrc/peaks.cu) go into
a library of their own, libafmm_peaks.so.  ``python -m paper_2301_01179_gb300.build`` or
``build()``.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libafmm.so")
OBJDIR = os.path.join(HERE, "_build")
SOURCES = ["api.cu", "tree.cu", "nearfield.cu", "farfield.cu", "s2l_tc.cu", "fourier.cu"]
PEAKS_SRC = "peaks.cu"
PEAKS_OUT = os.path.join(HERE, "libafmm_peaks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale():
    if not os.path.exists(OUT) or not os.path.exists(PEAKS_OUT):
        return True
    t = min(os.path.getmtime(OUT), os.path.getmtime(PEAKS_OUT))
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "afmm.h"))
    deps.append(os.path.join(HERE, "..", "include", "afmm_peaks.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False):
    if not force and not _stale():
        return OUT
    os.makedirs(OBJDIR, exist_ok=True)
    procs = []
    objs = []
    ptmp = PEAKS_OUT + ".tmp%d" % os.getpid()
    plog = os.path.join(OBJDIR, "peaks.log")
    pcmd = [nvcc()] + ARCH + FLAGS + ["-shared", os.path.join(CSRC, PEAKS_SRC), "-o", ptmp]
    procs.append((PEAKS_SRC, subprocess.Popen(pcmd, stdout=open(plog, "w"), stderr=subprocess.STDOUT), plog))
    for src in SOURCES:
        obj = os.path.join(OBJDIR, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc()] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        log = open(obj + ".log", "w")
        procs.append((src, subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT), obj + ".log"))
    failed = []
    for src, pr, log in procs:
        if pr.wait() != 0:
            failed.append((src, log))
    if failed:
        msg = []
        for src, log in failed:
            msg.append("---- %s ----\n%s" % (src, open(log).read()))
        raise RuntimeError("nvcc failed:\n" + "\n".join(msg))
    if verbose:
        for src, _, log in procs:
            sys.stdout.write(open(log).read())
    tmp = OUT + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, OUT)
    os.replace(ptmp, PEAKS_OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
