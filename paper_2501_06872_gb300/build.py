"""Builds libgt.so (the C-ABI library) and libgtgen.so (input generators) in-tree
for sm_103a with nvcc.  Translation units compile in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgt")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                   "-I", os.path.join(PKG, "csrc")] + list(extra)


def _compile(src: str, obj: str, extra=()) -> None:
    cmd = [nvcc()] + _flags(extra) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _link(objs, out: str) -> None:
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed for {out}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)


def build_lib(name: str, sources, headers, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    out = os.path.join(BUILD, f"lib{name}.so")
    objs = [os.path.join(BUILD, f"{name}_{os.path.splitext(os.path.basename(s))[0]}.o") for s in sources]
    todo = [(s, o) for s, o in zip(sources, objs) if _stale(o, [s] + headers)]
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(todo))) as ex:
            list(ex.map(lambda so: _compile(so[0], so[1], extra), todo))
    if todo or _stale(out, objs):
        _link(objs, out)
    return out


def build_generators() -> str:
    """libgtgen.so alone (the seeded input generators), without the CUDA
    library of the method."""
    gen_dir = os.path.join(PKG, "inputs")
    return build_lib("gtgen", sorted(glob.glob(os.path.join(gen_dir, "*.cu"))),
                     glob.glob(os.path.join(gen_dir, "*.h")))


def build(force: bool = False) -> dict:
    if force and os.path.isdir(BUILD):
        shutil.rmtree(BUILD)
    csrc = os.path.join(PKG, "csrc")
    headers = glob.glob(os.path.join(csrc, "*.h")) + glob.glob(os.path.join(csrc, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    srcs = sorted(glob.glob(os.path.join(csrc, "*.cu")))
    gen_dir = os.path.join(PKG, "inputs")
    gen_srcs = sorted(glob.glob(os.path.join(gen_dir, "*.cu")))
    out = {}
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        f1 = ex.submit(build_lib, "gt", srcs, headers)
        f2 = ex.submit(build_lib, "gtgen", gen_srcs, glob.glob(os.path.join(gen_dir, "*.h"))) if gen_srcs else None
        out["gt"] = f1.result()
        if f2 is not None:
            out["gtgen"] = f2.result()
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
