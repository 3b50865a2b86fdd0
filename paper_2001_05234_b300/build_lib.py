"""Build the in-tree CUDA library libcans.so for sm_103a (nvcc cross-compiles without a GPU)."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SO = os.path.join(HERE, "libcans.so")
SOURCES = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))
DEPS = SOURCES + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + [os.path.join(ROOT, "include", "cans.h")]
OBJDIR = os.path.join(HERE, "_build")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _obj(src: str) -> str:
    return os.path.join(OBJDIR, os.path.basename(src) + ".o")


def _stale_objects() -> list[str]:
    """Objects left behind by sources that no longer exist."""
    want = {_obj(s) for s in SOURCES}
    return [o for o in glob.glob(os.path.join(OBJDIR, "*.o")) if o not in want]


def _out_of_date(src: str) -> bool:
    """An object is rebuilt when its source or any shared header is newer than it."""
    obj = _obj(src)
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in [src, *DEPS[len(SOURCES):]])


def needs_build() -> bool:
    if not os.path.exists(SO) or _stale_objects():
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(d) > t for d in DEPS)


def _compile(src: str, verbose: bool) -> str:
    obj = _obj(src)
    cmd = [nvcc(), *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-c", "-o", obj, src]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the out-of-date translation units in parallel, then link one shared library (static
    cudart)."""
    if force or needs_build():
        from concurrent.futures import ThreadPoolExecutor

        os.makedirs(OBJDIR, exist_ok=True)
        for o in _stale_objects():
            os.remove(o)
        todo = [s for s in SOURCES if force or verbose or _out_of_date(s)]
        with ThreadPoolExecutor(max_workers=max(1, min(len(todo) or 1, os.cpu_count() or 1))) as ex:
            list(ex.map(lambda s: _compile(s, verbose), todo))
        objs = [_obj(s) for s in SOURCES]
        cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-cudart", "static",
               "-o", SO + ".tmp", *objs]
        subprocess.check_call(cmd)
        os.replace(SO + ".tmp", SO)
    return SO


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(SO)
