"""Build libss_gb300.so in-tree with nvcc for sm_103a (no torch extension machinery).

    python -m paper_1403_2056_gb300.build [--force]

Each .cu file under csrc/ compiles to an object in parallel, then one link.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
SO = os.path.join(OUT, "libss_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
ARCH_LTO = ["-gencode", "arch=compute_103a,code=lto_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
RDC_SOURCES = ("ss_sched.cu",)


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _stale(srcs, target) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = srcs + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    return any(os.path.getmtime(s) > t for s in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    os.makedirs(OUT, exist_ok=True)
    if not force and not _stale(srcs, SO):
        return SO
    procs = []
    objs = []
    rdc_objs = []
    for s in srcs:
        o = os.path.join(OUT, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        # the engine launches kernels from the device (its level scheduler):
        # relocatable device code as link-time-optimisable IR, compiled to
        # sm_103a with the whole engine in view by the device link below
        rdc = os.path.basename(s) in RDC_SOURCES
        if rdc:
            rdc_objs.append(o)
        cmd = [nvcc(), *(ARCH_LTO + ["-rdc=true"] if rdc else ARCH), *FLAGS, *extra, "-c", s, "-o", o]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    dlink = []
    if rdc_objs:
        dl = os.path.join(OUT, "device_link.o")
        cmd = [nvcc(), *ARCH, "-Xcompiler", "-fPIC", "-dlink", "-dlto", *rdc_objs, "-o", dl, "-lcudadevrt"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        dlink = [dl]
    tmp = SO + f".tmp{os.getpid()}"
    # the host linker joins the objects: the device code is final already (the
    # engine's in the device link above), so no further device link may run
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc()))), "lib64")
    link = [os.environ.get("CXX", "g++"), "-shared", "-o", tmp, *objs, *dlink, f"-L{cuda_lib}", "-lcudadevrt",
            "-lcudart", f"-Wl,-rpath,{cuda_lib}"]
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.check_call(link)
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(SO)
