"""Builds libpcfadj.so for sm_103a in-tree (paper_2306_00165_gb300/_build/).

Each CUDA translation unit is compiled by nvcc in parallel, then linked with the shared
CUDA runtime so that the library and PyTorch use one runtime and one context.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpcfadj.so")
SOURCES = ["pcf_kernels.cu", "pcf_host.cu", "pcf_noalloc.cu", "pcf_dmd.cu", "pcf_cheb_tc.cu", "pcf_modes_split.cu",
           "pcf_fno.cu", "pcf_sym_dns.cu", "pcf_planes_warp.cu", "pcf_cheb_tc05.cu",
           "pcf_sweep.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-rdc=false"]


def _nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libpcfadj")
    return cand


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra_flags=(), out=None):
    """Compile every translation unit and link libpcfadj.so; returns its path.  ``out``: a
    build folder other than the in-tree default (e.g. for a build with other flags)."""
    OUT_ = out or OUT
    LIB_ = os.path.join(OUT_, "libpcfadj.so")
    os.makedirs(OUT_, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "pcfadj.h"))
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc, *ARCH, *FLAGS, *extra_flags, "-I", os.path.join(HERE, "..", "include"),
                         "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    if force or jobs or not os.path.exists(LIB_):
        run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", LIB_, *objs])
    return LIB_


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra_flags=("-Xptxas", "-v") if "--ptxas-v" in sys.argv else ())
    print(LIB)
