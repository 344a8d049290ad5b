"""Build libkmeans2.so in-tree with nvcc for sm_103a.

Each translation unit under ``csrc/`` is compiled in parallel into
``csrc/_build/`` and linked into ``paper_1108_1351_gb300/libkmeans2.so``.
Rebuilds only what changed (object older than its source or a header).
``build_probe()`` compiles the FP32 FMA throughput probe that the benchmark
uses as its roofline denominator (``probe/fp32_peak.cu`` ->
``libfp32peak.so``; not part of the library).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(CSRC, "_build")
LIB = os.path.join(HERE, "libkmeans2.so")
# debug build: device-side index checks (KM2_DEBUG_CHECKS) that report an
# error status instead of trapping; loaded when KMEANS2_DEBUG=1
OBJ_DEBUG = os.path.join(CSRC, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libkmeans2_debug.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fvisibility=hidden"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkmeans2")
    return cand


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(p) > t for p in deps)


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False,
          debug: bool = False) -> str:
    """Compile and link the library; returns the path of the shared object.
    debug=True builds libkmeans2_debug.so with the device-side index checks."""
    nvcc = _nvcc()
    OBJ = OBJ_DEBUG if debug else globals()["OBJ"]
    LIB = LIB_DEBUG if debug else globals()["LIB"]
    flags = NVCC_FLAGS + (["-DKM2_DEBUG_CHECKS"] if debug else [])
    os.makedirs(OBJ, exist_ok=True)
    # objects built on another host architecture (x86 here, aarch64 on the GPU
    # hosts) must not be linked: rebuild everything when the stamp differs
    stamp = os.path.join(OBJ, "host_arch.txt")
    arch = platform.machine()
    try:
        with open(stamp) as fh:
            if fh.read().strip() != arch:
                force = True
    except OSError:
        force = True
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = _headers()
    jobs = []
    for src in srcs:
        obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, [src] + hdrs):
            cmd = [nvcc, *ARCH, *flags, "-I", INCLUDE, "-c", src, "-o", obj]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            jobs.append((src, cmd))
    objs = [os.path.join(OBJ, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def run(job):
        src, cmd = job
        p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        return src, p.returncode, p.stdout

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for src, rc, out in ex.map(run, jobs):
                if verbose or ptxas_info or rc != 0:
                    print(f"[nvcc] {os.path.basename(src)}\n{out}", flush=True)
                if rc != 0:
                    raise RuntimeError(f"nvcc failed on {src}")
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if p.returncode != 0:
            print(p.stdout)
            raise RuntimeError("linking libkmeans2.so failed")
        os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(arch)
    return LIB


PROBE_SRC = os.path.join(HERE, "probe", "fp32_peak.cu")
PROBE_LIB = os.path.join(HERE, "libfp32peak.so")
PROBE_STAMP = os.path.join(HERE, "probe", "host_arch.txt")


def build_probe(force: bool = False) -> str:
    """Compile the FP32 FMA probe (one translation unit) for sm_103a."""
    arch = platform.machine()
    try:
        with open(PROBE_STAMP) as fh:
            force = force or fh.read().strip() != arch
    except OSError:
        force = True
    if force or _stale(PROBE_LIB, [PROBE_SRC]):
        tmp = PROBE_LIB + f".tmp{os.getpid()}"
        cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, "-shared", "-o", tmp, PROBE_SRC]
        p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if p.returncode != 0:
            print(p.stdout)
            raise RuntimeError("building libfp32peak.so failed")
        os.replace(tmp, PROBE_LIB)
        with open(PROBE_STAMP, "w") as fh:
            fh.write(arch)
    return PROBE_LIB


if __name__ == "__main__":
    import sys
    print(build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv))
