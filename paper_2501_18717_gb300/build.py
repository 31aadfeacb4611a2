"""Build libbk.so (the C-ABI CUDA library) in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into
paper_2501_18717_gb300/libbk.so. Run ``python -m paper_2501_18717_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libbk.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["bk_api.cu", "k_ops.cu", "k_block.cu", "k_rng.cu", "bk_static.cu", "k_gemm.cu", "k_krylov.cu",
           "bk_krylov_api.cu", "k_batch.cu", "bk_batch_api.cu", "k_tc.cu", "k_tsm.cu", "k_pcg.cu", "k_rbf.cu", "k_bf16.cu",
           "k_ozaki.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the block-CG library needs the CUDA toolkit to build")


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    deps.append(os.path.join(HERE, "..", "include", "bk.h"))
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def _stamp() -> str:
    import platform
    return f"{platform.machine()} {' '.join(ARCH + FLAGS)}"


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    extra = list(extra or [])
    stamp_path = os.path.join(BUILD, "stamp.txt")
    old = open(stamp_path).read() if os.path.exists(stamp_path) else ""
    if old != _stamp():
        # objects from another machine or flag set: rebuild everything
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
        if os.path.exists(OUT):
            os.remove(OUT)
        with open(stamp_path, "w") as fh:
            fh.write(_stamp())

    def compile_one(src: str) -> str:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if _stale(o, s) or extra:
            cmd = [cc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), flush=True)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and r.stderr:
                print(r.stderr, flush=True)
        return o

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if not os.path.exists(OUT) or any(os.path.getmtime(o) > os.path.getmtime(OUT) for o in objs):
        tmp = OUT + ".tmp"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, extra=[a for a in sys.argv[1:] if a != "-v"]))
