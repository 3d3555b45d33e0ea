"""CPU oracle for the LocalContraction round loop -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (``paper_1807_10727_gb300``)
never imports it and shares no code with it: the oracle is plain single-threaded
C++ in ``lc_oracle.cpp`` (see that file's header for every reading of the paper
it fixes), built here with g++ and called through ctypes.

Pins (what each function is checked against, in ``tests/test_oracle_pins.py``):

* ``splitmix64_next`` / ``rank``: published SplitMix64 output values for a
  fixed seed (``tests/golden/splitmix64.txt``) and the stream composition.
* ``uf_labels``: scipy's connected components and BFS on tiny graphs.
* ``lc_run`` labels: union-find and scipy on every generated input; brute force
  over every graph on <= 5 vertices.
* ``lc_run`` per-phase sizes (forest variant): an independent per-phase
  construction in the tests (arborescences found as connected components of the
  parent graph, no pointer jumping), local-minimum counts, and closed forms
  for complete graphs, stars and paths.
* two-hop and tree variants: the same independent per-phase construction from
  their own definitions (labels over N(N(v)); weakly connected components of
  the open-neighbourhood parent graph).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "lc_oracle.cpp")
_SO = os.path.join(_DIR, "_build", "liblc_oracle.so")

FOREST, TWO_HOP, TREE = 0, 1, 2
_lib = None


def build() -> str:
    """Compile the oracle with g++ (plain -O2, no architecture flags)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp"
        res = subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", _SRC, "-o", tmp],
                             capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + res.stderr)
        os.replace(tmp, _SO)
    return _SO


def _bind(lib):
    u32, u64, i32, p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
    lib.oracle_splitmix64_next.argtypes = [ctypes.POINTER(u64)]
    lib.oracle_splitmix64_next.restype = u64
    lib.oracle_round_key.argtypes = [u64, u32]
    lib.oracle_round_key.restype = u64
    lib.oracle_rank.argtypes = [u64, u32, u32]
    lib.oracle_rank.restype = u32
    lib.oracle_ranks.argtypes = [u64, u32, u32, u32, p]
    lib.oracle_ranks.restype = None
    lib.oracle_uf_labels.argtypes = [u32, p, p, u64, p]
    lib.oracle_uf_labels.restype = i32
    lib.oracle_node_names.argtypes = [i32, u32, p, p, u64, u64, u32, p, p]
    lib.oracle_node_names.restype = i32
    lib.oracle_lc_run.argtypes = [u32, p, p, u64, u64, i32, u64, p, u32, u32, p, p, p, p, p, p, u32]
    lib.oracle_lc_run.restype = i32
    return lib


def _L():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily route every oracle call to another build of lc_oracle.cpp
    (the tests use this to check that deliberately broken copies of the oracle
    fail the pins)."""
    global _lib
    saved = _L()
    _lib = _bind(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def splitmix64_next(state: int) -> tuple[int, int]:
    """Returns (output, new_state) of one SplitMix64 step."""
    s = ctypes.c_uint64(state)
    out = _L().oracle_splitmix64_next(ctypes.byref(s))
    return int(out), int(s.value)


def round_key(seed: int, i: int) -> int:
    return int(_L().oracle_round_key(seed, i))


def rank(seed: int, i: int, v: int) -> int:
    return int(_L().oracle_rank(seed, i, v))


def ranks(seed: int, i: int, v0: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint32)
    _L().oracle_ranks(seed, i, v0, count, out.ctypes.data)
    return out


def uf_labels(n: int, src, dst) -> np.ndarray:
    src, dst = _u32(src), _u32(dst)
    out = np.empty(n, dtype=np.uint32)
    rc = _L().oracle_uf_labels(n, src.ctypes.data, dst.ctypes.data, src.size, out.ctypes.data)
    if rc:
        raise ValueError("uf_labels: vertex id out of range")
    return out


def node_names(variant: int, n: int, src, dst, seed: int, i: int) -> tuple[np.ndarray, int]:
    src, dst = _u32(src), _u32(dst)
    out = np.empty(n, dtype=np.uint32)
    J = ctypes.c_uint32(0)
    rc = _L().oracle_node_names(variant, n, src.ctypes.data, dst.ctypes.data, src.size, seed, i,
                                out.ctypes.data, ctypes.byref(J))
    if rc:
        raise ValueError("node_names: invalid input")
    return out, int(J.value)


class Result:
    def __init__(self, labels, rounds, n_i, m_i, mp_i, J_i):
        self.labels, self.rounds = labels, rounds
        self.n_i, self.m_i, self.mp_i, self.J_i = n_i, m_i, mp_i, J_i

    def sizes(self) -> list[tuple[int, int]]:
        return [(int(a), int(b)) for a, b in zip(self.n_i, self.m_i)]


def lc_run(n: int, src, dst, seed: int, variant: int = FOREST, finish_edges: int = 0,
           max_rounds: int = 1 << 20, cap: int = 4096, merge_alpha=()) -> Result:
    """merge_alpha[i] > 0: MergeToLarge step with parameter alpha_i in phase i."""
    src, dst = _u32(src), _u32(dst)
    alpha = np.ascontiguousarray(np.asarray(merge_alpha, dtype=np.uint32).reshape(-1))
    labels = np.empty(n, dtype=np.uint32)
    n_i = np.zeros(cap, dtype=np.uint64)
    m_i = np.zeros(cap, dtype=np.uint64)
    mp_i = np.zeros(cap, dtype=np.uint64)
    J_i = np.zeros(cap, dtype=np.uint32)
    R = ctypes.c_uint32(0)
    rc = _L().oracle_lc_run(n, src.ctypes.data, dst.ctypes.data, src.size, seed, variant,
                            finish_edges, alpha.ctypes.data if alpha.size else None, alpha.size,
                            max_rounds, labels.ctypes.data, ctypes.byref(R),
                            n_i.ctypes.data, m_i.ctypes.data, mp_i.ctypes.data, J_i.ctypes.data,
                            cap)
    if rc == 1:
        raise ValueError("lc_run: invalid input")
    if rc == 2:
        raise RuntimeError("lc_run: more phases than cap")
    if rc == 3:
        raise RuntimeError("lc_run: no convergence within max_rounds")
    r = int(R.value)
    return Result(labels, r, n_i[:r].copy(), m_i[:r].copy(), mp_i[:r].copy(), J_i[:r].copy())
