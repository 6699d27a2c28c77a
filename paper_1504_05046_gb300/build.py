"""Build the bsmm shared library (C ABI over the sm_103a kernels) in-tree.

Every translation unit is compiled by nvcc for sm_103a only, in parallel, then
linked into ``_build/libbsmm.so`` next to this file. The CUDA runtime is linked
statically, so the library needs nothing but the driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libbsmm.so")
SOURCES = ["plan.cpp", "execute.cpp", "fp64.cu", "split.cu", "noalloc.cu", "mlp.cu", "batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, obj: str, extra) -> None:
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-I", os.path.join(HERE, "..", "include"), "-c", src, "-o", obj, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(OUT, exist_ok=True)
    srcs = [os.path.join(SRC, s) for s in SOURCES if os.path.exists(os.path.join(SRC, s))]
    deps = srcs + [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "bsmm.h"))
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(d) for d in deps)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    objs = [os.path.join(OUT, os.path.basename(s) + ".o") for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        futs = [ex.submit(_compile, s, o, list(extra)) for s, o in zip(srcs, objs)]
        for f in futs:
            f.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(LIB)
    return LIB


_KIND_PROBE = r"""
#include <cstdint>
__global__ void probe(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n\t}\n"
               :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
"""


def tcgen05_kind_supported(kind: str):
    """Whether the toolchain accepts one tcgen05.mma of the given kind (f16, tf32, f8f6f4,
    i8, ...) for sm_103a: compiles a one-instruction kernel. Returns (accepted, message)."""
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "probe.cu")
        with open(src, "w") as f:
            f.write(_KIND_PROBE.replace("KIND", kind))
        r = subprocess.run([nvcc(), *ARCH, "-c", src, "-o", os.path.join(d, "probe.o")], capture_output=True,
                           text=True)
        msg = " ".join(m.group(1) for m in re.finditer(r"error\s*:\s*(.*)", r.stderr))
        return r.returncode == 0, msg


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
