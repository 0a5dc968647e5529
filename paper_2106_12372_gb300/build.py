"""Builds the CUDA library ``libnrc.so`` in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into one shared
library with a C ABI (``include/nrc.h``).  No PyTorch headers are involved.

Variants (``build(variant=...)``, ``python build.py --variant V``), each its
own library ``libnrc_V.so`` and object folder:
  san    the host code compiled and linked with AddressSanitizer and
         UndefinedBehaviorSanitizer (load it with libasan preloaded);
  debug  ``-DNRC_DEBUG``: device-side bounds checks that set the error word
         (NRC_ERR_BOUNDS through nrc_check_error) instead of accessing out of
         range.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnrc.so")
VARIANTS = {
    "": [],
    # (one sanitizer per -Xcompiler: nvcc splits its values at commas)
    "san": ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined", "-Xcompiler",
            "-fno-omit-frame-pointer", "-Xcompiler", "-fno-sanitize-recover=undefined"],
    "debug": ["-DNRC_DEBUG"],
}


def lib_path(variant: str = "") -> str:
    return LIB if not variant else os.path.join(HERE, f"libnrc_{variant}.so")
SOURCES = ["nrc_api.cu", "k_simt.cu", "k_tc.cu", "k_plain.cu", "nrc_noalloc.cu", "nrc_batch.cu", "nrc_serve.cu", "k_shampoo.cu", "k_paths.cu", "k_frame.cu", "k_tc128.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def flags(verbose: bool = False) -> list[str]:
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")] + ARCH
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, p) for p in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "nrc.h"), __file__]
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, variant: str | None = None) -> str:
    """Compile (if stale) and return the path of libnrc.so (or of a variant;
    by default the one NRC_LIB_VARIANT names)."""
    if variant is None:
        variant = os.environ.get("NRC_LIB_VARIANT", "")
    if variant not in VARIANTS:
        raise ValueError(f"unknown build variant {variant!r}")
    lib = lib_path(variant)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    obj_dir = BUILD if not variant else BUILD + "_" + variant
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    extra = VARIANTS[variant]

    def compile_one(src: str) -> str:
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + flags(verbose) + extra
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        if verbose:
            sys.stderr.write(res.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    res = subprocess.run([cc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC", "-lpthread"] + extra,
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = sys.argv[sys.argv.index("--variant") + 1] if "--variant" in sys.argv else None
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, variant=v))
