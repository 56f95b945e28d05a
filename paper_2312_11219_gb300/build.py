"""Build the in-tree CUDA library lib/libg3aca.so for sm_103a.

Each CUDA translation unit is compiled by its own nvcc process (in
parallel); the host-only cluster-tree builder is compiled by g++ without
floating-point contraction so the block partition is bit-identical on every
host.  No cmake, one -gencode.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIB = os.path.join(LIBDIR, "libg3aca.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["g3_prep.cu", "g3_aca.cu", "g3_aca_slp.cu", "g3_aca_dlp.cu", "g3_aca_sep.cu", "g3_aca_gal.cu",
              "g3_aca_p1.cu", "g3_apply.cu",
              "g3_api.cu",
              "g3_probe.cu", "g3_mlp.cu", "g3_gcq.cu"]
# the compression-kernel instantiations of each kernel kind are compiled in
# this many parts (-DG3_ACA_PART=0..), one nvcc process each
ACA_PARTS = {"g3_aca_slp.cu": 4, "g3_aca_dlp.cu": 4, "g3_aca_sep.cu": 4, "g3_aca_gal.cu": 4, "g3_aca_p1.cu": 4}
CPP_SOURCES = ["g3_tree.cpp"]


def _run(cmd: list[str]) -> tuple[list[str], int, str]:
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    return cmd, p.returncode, p.stdout


def _stale(src_files: list[str], target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "g3aca.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps + src_files)


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link the library; returns its path.  Raises on failure."""
    os.makedirs(OBJDIR, exist_ok=True)
    srcs = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES]
    if not force and not _stale(srcs, LIB):
        return LIB
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    inc = ["-I", CSRC, "-I", os.path.join(HERE, "..", "include")]
    jobs = []
    objs = []
    for f in CU_SOURCES:
        parts = ACA_PARTS.get(f, 0)
        for part in range(max(parts, 1)):
            o = os.path.join(OBJDIR, f.replace(".cu", f"_{part}.o" if parts else ".o"))
            objs.append(o)
            cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, f), "-o", o]
            if parts:
                cmd.insert(1, f"-DG3_ACA_PART={part}")
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    cxx = shutil.which("g++") or "g++"
    for f in CPP_SOURCES:
        o = os.path.join(OBJDIR, f.replace(".cpp", ".o"))
        objs.append(o)
        jobs.append([cxx, "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off",
                     "-I", os.path.join(CUDA_HOME, "include"), *inc, "-c", os.path.join(CSRC, f), "-o", o])
    jobs.sort(key=lambda c: not any(a.startswith("-DG3_ACA_PART") for a in c))  # longest first
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 8))) as ex:
        results = list(ex.map(_run, jobs))
    for cmd, rc, out in results:
        if verbose or rc != 0 or ptxas_info:
            sys.stderr.write(" ".join(cmd) + "\n" + out)
        if rc != 0:
            raise RuntimeError(f"compilation failed: {' '.join(cmd)}\n{out}")
    tmp = LIB + ".tmp"
    cmd, rc, out = _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"])
    if rc != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{out}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, ptxas_info="--ptxas" in sys.argv))
