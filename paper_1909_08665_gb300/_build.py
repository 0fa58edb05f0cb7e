"""Compile the CUDA library ``libsnn_gb300.so`` in-tree for sm_103a.

Each translation unit is compiled in parallel with nvcc, then linked into one
shared library next to this file.  Host code is compiled with
``-ffp-contract=off`` and device code with ``-fmad=false`` so that no
floating-point expression is fused: the model's arithmetic is fixed to one
rounding per operation.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsnn_gb300.so")
SOURCES = ["capi.cu", "build_net.cu", "step.cu", "step_mode_plain.cu", "step_mode_paced.cu",
           "step_mode_sat.cu", "step_mode_sat_paced.cu", "noalloc.cu", "batch.cu", "grad.cu",
           "adjoint_part.cu", "deliver_cluster.cu", "deliver_words.cu", "deliver_stream.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-O2"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale(outputs, inputs):
    if not all(os.path.exists(o) for o in outputs):
        return True
    newest = max(os.path.getmtime(i) for i in inputs)
    return any(os.path.getmtime(o) < newest for o in outputs)


def build(force=False, verbose=False, extra=()):
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "snn.h"))
    objs, procs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(objdir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale([o], [s] + headers):
            cmd = [nvcc()] + ARCH + FLAGS + list(extra) + ["-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                stderr=subprocess.STDOUT, text=True)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: %s\n%s" % (" ".join(cmd), out))
        if verbose and out.strip():
            print(out, file=sys.stderr)
    if force or procs or _stale([LIB], objs):
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
