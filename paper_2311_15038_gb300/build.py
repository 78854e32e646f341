"""Build libmctp.so in-tree: nvcc for sm_103a, one object per .cu, in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmctp.so")
LIB_CHECKED = os.path.join(BUILD, "checked", "libmctp_checked.so")  # kernels compiled with MCTP_CHECKED
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I", os.path.join(ROOT, "include")]


def _compile(src: str, verbose_ptxas: bool, checked: bool = False) -> tuple[str, str]:
    out = os.path.join(BUILD, "checked") if checked else BUILD
    obj = os.path.join(out, os.path.basename(src).replace(".cu", ".o"))
    cmd = ["nvcc", *NVCC_FLAGS, *(["-DMCTP_CHECKED"] if checked else []), "-c", src, "-o", obj]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose_ptxas: bool = False, checked: bool = True) -> str:
    """Compile every csrc/*.cu and link libmctp.so (and, with checked, the
    bounds-tested libmctp_checked.so from the same sources); returns the
    path of libmctp.so."""
    os.makedirs(os.path.join(BUILD, "checked"), exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs = [(src, False) for src in srcs] + ([(src, True) for src in srcs] if checked else [])
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), 2 * (os.cpu_count() or 4))) as ex:
        results = list(ex.map(lambda j: _compile(j[0], verbose_ptxas and not j[1], j[1]), jobs))
    objs = [o for (o, _), (_, chk) in zip(results, jobs) if not chk]
    if verbose_ptxas:
        with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
            for (_, log), (src, chk) in zip(results, jobs):
                if not chk:
                    f.write(f"== {os.path.basename(src)}\n{log}\n")
    for lib, these in ((LIB, objs), (LIB_CHECKED, [o for (o, _), (_, chk) in zip(results, jobs) if chk])):
        if not these:
            continue
        tmp = lib + ".tmp"
        subprocess.check_call(["nvcc", "-shared", *ARCH, "-o", tmp, *these])
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose_ptxas="-v" in sys.argv))
