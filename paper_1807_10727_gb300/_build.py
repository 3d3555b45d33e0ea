"""In-tree build of the native libraries (no cmake, no torch extension machinery).

* ``libsynth.so``  - host C input generators (``csrc/synth.c``), built with gcc.
* ``liblc.so``     - the CUDA connected-components library behind ``include/lc.h``
                     (``csrc/*.cu``), built with nvcc for sm_103a only.

Objects are compiled in parallel and relinked only when a source is newer than
the library, so a second ``build()`` is a no-op.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
CSRC = os.path.join(PKG_DIR, "csrc")
INCLUDE = os.path.join(REPO_DIR, "include")
LIB_DIR = os.path.join(PKG_DIR, "_lib")
OBJ_DIR = os.path.join(LIB_DIR, "obj")

SYNTH_SO = os.path.join(LIB_DIR, "libsynth.so")
LC_SO = os.path.join(LIB_DIR, "liblc.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
LC_SOURCES = ["lc_abi.cu", "lc_round.cu", "lc_sort.cu", "lc_merge.cu"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd: list[str]) -> None:
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("build failed: %s\n%s\n%s" % (" ".join(cmd), res.stdout, res.stderr))


def build_synth() -> str:
    os.makedirs(LIB_DIR, exist_ok=True)
    src = os.path.join(CSRC, "synth.c")
    if _newer(SYNTH_SO, [src]):
        tmp = SYNTH_SO + ".tmp"
        _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", src, "-o", tmp, "-lm"])
        os.replace(tmp, SYNTH_SO)
    return SYNTH_SO


def _headers() -> list[str]:
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs


def build_lc(extra_flags: list[str] | None = None) -> str:
    os.makedirs(OBJ_DIR, exist_ok=True)
    nvcc = _nvcc()
    headers = _headers()
    flags = NVCC_FLAGS + ARCH_FLAGS + ["-I", INCLUDE, "-I", CSRC] + (extra_flags or [])
    objs, jobs = [], []
    for s in LC_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OBJ_DIR, s.replace(".cu", ".o"))
        objs.append(obj)
        if _newer(obj, [src] + headers):
            jobs.append([nvcc] + flags + ["-c", src, "-o", obj])
    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(_run, jobs))
    if _newer(LC_SO, objs):
        tmp = LC_SO + ".tmp"
        _run([nvcc] + ARCH_FLAGS + ["-shared", "-cudart", "static", "-o", tmp] + objs)
        os.replace(tmp, LC_SO)
    return LC_SO


def build_all() -> None:
    build_synth()
    build_lc()
