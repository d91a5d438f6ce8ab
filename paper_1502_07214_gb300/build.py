"""Build the CUDA library ``libmuca.so`` in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel and linked into one
shared library beside this file.  Host code is compiled with
-ffp-contract=off so that the FP64 acceptance table and weight recursion round
exactly as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libmuca.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["sweep.cu", "scan.cu", "reweight.cu", "reweight_noalloc.cu", "peak.cu", "runtime.cu",
           "probe.cu", "bonds.cu"]
HEADERS = ["muca_internal.h", "philox.cuh", "scan_core.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
         "--expt-relaxed-constexpr"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    inc = [os.path.join(os.path.dirname(HERE), "include", h) for h in ("muca.h", "muca_probe.h")]
    return [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + inc + [__file__]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(OUT):
        if os.path.getmtime(OUT) >= max(os.path.getmtime(p) for p in _deps()):
            return OUT
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT, text=True)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out)
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = OUT + ".tmp"
    subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"], check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
