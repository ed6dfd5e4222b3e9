"""Build libwhff.so in-tree with nvcc for sm_103a (one -gencode, translation
units compiled in parallel).  Used by __graft_entry__.build() and by the
binding when the library is missing or older than its sources."""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
OUT = PKG / "libwhff.so"
OBJ = PKG / "_build"

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++17", "-O3", "-Xcompiler", "-fPIC", f"-I{ROOT / 'include'}", f"-I{CSRC}"]

CUDA_SOURCES = ["whff_runtime.cu", "whff_noalloc.cu", "wz2_r8.cu", "wz2_r12.cu", "wz2_r16.cu", "wz2_r20.cu",
                "wz2_r24.cu", "scaled.cu", "mma.cu", "scaled_mma.cu", "wz3.cu"]
HOST_SOURCES = ["whff_encode.cpp", "whff_serve.cpp"]


def sources():
    return [CSRC / s for s in CUDA_SOURCES + HOST_SOURCES]


def _deps():
    return sources() + list(CSRC.glob("*.cuh")) + list(CSRC.glob("*.h")) + [ROOT / "include" / "whff.h"]


def up_to_date() -> bool:
    return OUT.exists() and OUT.stat().st_mtime >= max(p.stat().st_mtime for p in _deps())


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and up_to_date():
        return OUT
    OBJ.mkdir(exist_ok=True)
    procs = []
    objs = []
    for s in CUDA_SOURCES:
        o = OBJ / (s + ".o")
        cmd = [NVCC, *COMMON, *ARCH, "-lineinfo", "-c", str(CSRC / s), "-o", str(o)]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(o)
    for s in HOST_SOURCES:
        o = OBJ / (s + ".o")
        cmd = [NVCC, *COMMON, "-Xcompiler", "-pthread", "-c", str(CSRC / s), "-o", str(o)]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(o)
    failed = False
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + out.decode(errors="replace"))
        failed |= p.returncode != 0
    if failed:
        raise RuntimeError("nvcc failed building libwhff")
    tmp = OUT.with_suffix(f".{os.getpid()}.tmp")
    link = [NVCC, "-shared", *ARCH, "-o", str(tmp), *map(str, objs), "-lcudart", "-Xcompiler", "-pthread"]
    subprocess.run(link, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
