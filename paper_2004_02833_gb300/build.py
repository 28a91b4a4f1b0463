"""Build librtpn.so in-tree for sm_103a (nvcc, one -gencode, translation units in parallel).

Usage:  python -m paper_2004_02833_gb300.build   (or __graft_entry__.build())
Output: paper_2004_02833_gb300/lib/librtpn.so (git-ignored; rebuilt on every machine).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "lib")
BUILD_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "librtpn.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


VARIANT_SRC = "window.cu"  # compiled once per (order, class) listed in window_variants.h
STAGE_SRC = "stage.cu"     # compiled once per (order, tile, depth, box size) listed in stage_variants.h
FUSED_SRC = "fused.cu"     # compiled once per order listed in fused_variants.h


def window_orders() -> list[int]:
    text = open(os.path.join(CSRC, "window_variants.h")).read()
    line = [l for l in text.splitlines() if l.startswith("#define RTPN_WINDOW_ORDERS")][0]
    return [int(v) for v in re.findall(r"X\((\d+)\)", line)]


def fused_orders() -> list[int]:
    text = open(os.path.join(CSRC, "fused_variants.h")).read()
    line = [l for l in text.splitlines() if l.startswith("#define RTPN_FUSED_ORDERS")][0]
    return [int(v) for v in re.findall(r"X\((\d+)\)", line)]


def stage_variants() -> list[tuple[int, int, int, int, int, int]]:
    text = open(os.path.join(CSRC, "stage_variants.h")).read()
    line = [l for l in text.splitlines() if l.startswith("#define RTPN_STAGE_VARIANTS")][0]
    return [tuple(int(v) for v in m) for m in
            re.findall(r"X\((\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)", line)]


def units() -> list[tuple[str, list[str], str]]:
    """(source, defines, object name) of every translation unit."""
    out = []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith((".cu", ".cpp")) or f in (VARIANT_SRC, STAGE_SRC, FUSED_SRC):
            continue
        out.append((os.path.join(CSRC, f), [], f + ".o"))
    for n in window_orders():
        for cls in (0, 1):
            out.append((os.path.join(CSRC, VARIANT_SRC), [f"-DRTPN_WN={n}", f"-DRTPN_WCLS={cls}"],
                        f"window_N{n}_c{cls}.o"))
    for n in fused_orders():
        out.append((os.path.join(CSRC, FUSED_SRC), [f"-DRTPN_FN={n}"], f"fused_N{n}.o"))
    for n, tx, ty, tz, nb, em in stage_variants():
        out.append((os.path.join(CSRC, STAGE_SRC),
                    [f"-DRTPN_SN={n}", f"-DRTPN_STX={tx}", f"-DRTPN_STY={ty}", f"-DRTPN_STZ={tz}",
                     f"-DRTPN_SNB={nb}", f"-DRTPN_SEM={em}"],
                    f"stage_N{n}_{tx}x{ty}x{tz}_b{nb}_e{em}.o"))
    return out


def _compile(unit, extra: list[str]) -> str:
    src, defines, name = unit
    obj = os.path.join(BUILD_DIR, name)
    deps = [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(INCLUDE, "rtpn.h"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    cmd = [_nvcc()] + ARCH + COMMON + defines + extra + ["-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(verbose: bool = False, extra: list[str] | None = None, jobs: int | None = None) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = list(extra or [])
    todo = units()
    # longest units first so the parallel build ends sooner
    todo.sort(key=lambda u: -max([int(d.split("=")[1]) for d in u[1]
                                  if d.startswith(("-DRTPN_WN", "-DRTPN_SN", "-DRTPN_FN"))] or [0]))
    jobs = jobs or min(len(todo), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda u: _compile(u, extra), todo))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = [_nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB] + objs + [
            "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
