"""Compile the in-tree CUDA libraries for sm_103a (GB300).

``libwrs.so``            the product library (C ABI of include/wrs.h)
``libwrs_check.so``      the same sources with WRS_CHECK=1: bucket write
                         counts and index checks, for verification
``libwrs_workloads.so``  device-side generator of the seeded synthetic inputs

All are built with nvcc directly into this package directory (no cmake, no
torch extension machinery) and rebuilt only when a source is newer.
"""
from __future__ import annotations

import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared"]

# libwrs: no multiply-add contraction, so that the OS-ND binomial deviates
# (binary64 arithmetic) follow the written steps exactly.
EXTRA = {"libwrs.so": ["-fmad=false"], "libwrs_check.so": ["-fmad=false", "-DWRS_CHECK=1"]}

_WRS_HEADERS = ["wrs_device.cuh", "wrs_kernels.cuh", "wrs_batch.cuh", "wrs_twolevel.cuh", "wrs_osnd.cuh",
                "wrs_psaplus.cuh"]
TARGETS = {
    "libwrs.so": (["wrs.cu"], _WRS_HEADERS, [os.path.join(INCLUDE, "wrs.h")]),
    "libwrs_check.so": (["wrs.cu"], _WRS_HEADERS, [os.path.join(INCLUDE, "wrs.h")]),
    "libwrs_workloads.so": (["workloads.cu"], [], []),
}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> list[str]:
    procs = []
    outs = []
    for name, (srcs, hdrs, extra) in TARGETS.items():
        out = os.path.join(PKG, name)
        outs.append(out)
        src_paths = [os.path.join(CSRC, s) for s in srcs]
        deps = src_paths + [os.path.join(CSRC, h) for h in hdrs] + extra
        if not force and not _stale(out, deps):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *EXTRA.get(name, []), "-I", INCLUDE, "-o", tmp, *src_paths]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), tmp, out, cmd))
    errors = []
    for p, tmp, out, cmd in procs:
        log, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{' '.join(cmd)}\n{log.decode(errors='replace')}")
        else:
            os.replace(tmp, out)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    return outs


if __name__ == "__main__":
    for o in build(verbose=True):
        print(o)
