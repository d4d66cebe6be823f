"""Build the CUDA library libdfscf.so in-tree with nvcc for sm_103a (GB300).

Each .cu file is compiled to an object in parallel, then linked with -shared.  The
result lands next to this file; a stamp of source hashes avoids needless rebuilds.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libdfscf.so")
BUILD_DIR = os.path.join(HERE, "_build")
# The checking variant (kernels bound-check their computed indices, see DF_IX in the
# sources) builds next to the normal library and loads when DFSCF_VARIANT=bounds.
VARIANTS = {"": (LIB, BUILD_DIR, []),
            "bounds": (os.path.join(HERE, "libdfscf_bounds.so"), os.path.join(HERE, "_build_bounds"),
                       ["-DDFSCF_BOUNDS_CHECK"])}


def variant_path(variant: str = "") -> str:
    return VARIANTS[variant][0]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC] + ARCH


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _digest() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)) + [os.path.join(INCLUDE, "dfscf.h")]:
        p = f if os.path.isabs(f) else os.path.join(CSRC, f)
        with open(p, "rb") as fh:
            h.update(p.encode() + fh.read())
    h.update(" ".join(NVCC_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None, variant: str = "") -> str:
    lib_path, build_dir, vflags = VARIANTS[variant]
    os.makedirs(build_dir, exist_ok=True)
    stamp = os.path.join(build_dir, "stamp")
    extra = list(vflags) + list(extra_flags or [])
    dig = _digest() + " ".join(extra)
    if not force and os.path.exists(lib_path) and os.path.exists(stamp) and open(stamp).read() == dig:
        return lib_path
    cc = nvcc()
    flags = NVCC_FLAGS + extra

    def compile_one(src: str) -> str:
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, "-c", src, "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, variant="bounds" if "--bounds" in sys.argv else ""))
