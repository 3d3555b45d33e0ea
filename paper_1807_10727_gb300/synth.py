"""Seeded synthetic inputs shaped like the paper's workloads (Section 6, Empirical study, Table 1).

The paper evaluates on social and web graphs (Orkut, Friendster, Clueweb and two
non-public graphs) that are not available here; these generators stand in for
them: R-MAT for the skewed social/web graphs, Erdos-Renyi G(n, m) for the random
graph class of Section 5, and a permuted 2D grid mixed with power-law-sized
random components for the high-diameter lower-bound case of Section 6.

This module builds inputs only.  It holds none of the method's arithmetic (no
vertex ranking, no minimum, no contraction), so both the CPU oracle and the GPU
path consume exactly the same edge lists from it.  All randomness is a counter
hash of (seed, index) computed in ``csrc/synth.c``.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field

import numpy as np

from . import _build

_lib = None


def _synth():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build_synth())
        u64, i32, dbl = ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        p = ctypes.c_void_p
        lib.synth_er.argtypes = [u64, u64, u64, p, p, i32]
        lib.synth_rmat.argtypes = [i32, u64, u64, dbl, dbl, dbl, u64, u64, p, p, i32]
        lib.synth_permute_ids.argtypes = [u64, u64, p, u64, i32]
        lib.synth_perm_one.argtypes = [u64, u64, ctypes.c_uint32]
        lib.synth_perm_one.restype = ctypes.c_uint32
        lib.synth_grid_edges.argtypes = [u64, u64]
        lib.synth_grid_edges.restype = u64
        lib.synth_grid.argtypes = [u64, u64, u64, p, p, i32]
        lib.synth_powerlaw_sizes.argtypes = [u64, ctypes.c_uint32, ctypes.c_uint32, dbl, u64, p]
        lib.synth_components.argtypes = [u64, p, p, p, u64, u64, p, p, i32]
        lib.synth_draws.argtypes = [u64, u64, p]
        for name in ("synth_er", "synth_rmat", "synth_permute_ids", "synth_grid",
                     "synth_powerlaw_sizes", "synth_components"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError("%s: invalid arguments (code %d)" % (what, rc))


@dataclass
class Graph:
    """One undirected graph as a uint32 COO edge list (loops and duplicates kept)."""
    n: int
    src: np.ndarray
    dst: np.ndarray
    name: str = ""
    seed: int = 0          # rank seed the workload is quoted with
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def er(n: int, m: int, seed: int, nthreads: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """G(n, m): m endpoint pairs drawn uniformly from [0, n) with replacement."""
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    _check(_synth().synth_er(n, m, seed, _ptr(src), _ptr(dst), nthreads), "er")
    return src, dst


def rmat(scale: int, m: int, seed: int, perm_seed: int = 0, a: float = 0.57,
         b: float = 0.19, c: float = 0.19, n_keep: int | None = None,
         nthreads: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """R-MAT with `scale` levels; ids >= n_keep are redrawn; perm_seed != 0
    applies a seeded bijection of [0, n_keep) to both endpoints."""
    n_keep = (1 << scale) if n_keep is None else n_keep
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    _check(_synth().synth_rmat(scale, n_keep, m, a, b, c, seed, perm_seed,
                               _ptr(src), _ptr(dst), nthreads), "rmat")
    return src, dst


def permute_ids(x: np.ndarray, n: int, perm_seed: int, nthreads: int = 0) -> None:
    """In place: x[j] <- pi(x[j]) for a seeded bijection pi of [0, n)."""
    assert x.dtype == np.uint32 and x.flags.c_contiguous
    _check(_synth().synth_permute_ids(n, perm_seed, _ptr(x), x.size, nthreads), "permute")


def perm_one(n: int, perm_seed: int, v: int) -> int:
    return int(_synth().synth_perm_one(n, perm_seed, v))


def grid(w: int, h: int, off: int = 0, nthreads: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """w x h 4-neighbour grid with vertex (x, y) = off + y*w + x."""
    m = int(_synth().synth_grid_edges(w, h))
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    _check(_synth().synth_grid(w, h, off, _ptr(src), _ptr(dst), nthreads), "grid")
    return src, dst


def powerlaw_sizes(count: int, smin: int, smax: int, alpha: float, seed: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint32)
    _check(_synth().synth_powerlaw_sizes(count, smin, smax, alpha, seed, _ptr(out)), "sizes")
    return out


def draws(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _synth().synth_draws(seed, count, _ptr(out))
    return out


def uniforms(seed: int, count: int) -> np.ndarray:
    """count floats in [0, 1) from the top 53 bits of the counter stream."""
    return (draws(seed, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)


def grid_mix(grid_w: int, grid_h: int, n_comp: int, alpha: float = 2.1, smin: int = 2,
             smax: int = 1 << 14, edges_per_vertex: float = 1.5, seed: int = 303,
             perm_seed: int = 304, nthreads: int = 0) -> Graph:
    """A grid unioned with n_comp ER components of power-law sizes, each with
    ceil(edges_per_vertex * s) edges drawn inside it, all ids permuted."""
    sizes = powerlaw_sizes(n_comp, smin, smax, alpha, seed)
    ecount = np.ceil(sizes.astype(np.float64) * edges_per_vertex).astype(np.uint64)
    voff = np.zeros(n_comp + 1, dtype=np.uint64)
    np.cumsum(sizes, out=voff[1:])
    eoff = np.zeros(n_comp + 1, dtype=np.uint64)
    np.cumsum(ecount, out=eoff[1:])
    n_grid = grid_w * grid_h
    n = n_grid + int(voff[-1])
    if n > 0xFFFFFFFF:
        raise ValueError("grid_mix: too many vertices")
    m_grid = int(_synth().synth_grid_edges(grid_w, grid_h))
    m = m_grid + int(eoff[-1])
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    if m_grid:
        _check(_synth().synth_grid(grid_w, grid_h, 0, _ptr(src), _ptr(dst), nthreads), "grid")
    cs, cd = src[m_grid:], dst[m_grid:]
    _check(_synth().synth_components(n_comp, _ptr(sizes), _ptr(voff), _ptr(eoff), n_grid,
                                     seed + 1, _ptr(cs), _ptr(cd), nthreads), "components")
    permute_ids(src, n, perm_seed, nthreads)
    permute_ids(dst, n, perm_seed, nthreads)
    return Graph(n, src, dst, meta={"grid": (grid_w, grid_h), "components": n_comp})


# ------------------------------------------------------------- workloads

RMAT_ABC = (0.57, 0.19, 0.19)


def workload(name: str, nthreads: int = 0) -> Graph:
    """The named single-graph workloads.

    er16      G(n=2^16, m=2^19), gen seed 101, rank seed 1
    rmat26    R-MAT scale 26, m=2^30, (a,b,c,d)=(.57,.19,.19,.05), permuted ids,
              gen seed 202, perm seed 203, rank seed 7
    gridmix   8192x8192 grid + 2^20 power-law (alpha 2.1, sizes 2..2^14) ER
              components with 1.5 edges per vertex (average degree 3), permuted,
              gen seed 303, perm seed 304, rank seed 3
    rmatS / gridmixS   reduced versions of the same recipes for fast tests,
              e.g. rmat18 (scale 18, m = 16 * 2^18) and gridmix_small
              (512x512 grid + 2^12 components).
    """
    if name == "er16":
        s, d = er(1 << 16, 1 << 19, 101, nthreads)
        return Graph(1 << 16, s, d, name, seed=1)
    if name.startswith("rmat"):
        scale = int(name[4:])
        m = 1 << (scale + 4)
        s, d = rmat(scale, m, 202, 203, *RMAT_ABC, nthreads=nthreads)
        return Graph(1 << scale, s, d, name, seed=7)
    if name == "gridmix":
        g = grid_mix(8192, 8192, 1 << 20, nthreads=nthreads)
        g.name, g.seed = name, 3
        return g
    if name == "gridmix_small":
        g = grid_mix(512, 512, 1 << 12, nthreads=nthreads)
        g.name, g.seed = name, 3
        return g
    if name.startswith("er_"):
        # er_<log2 n>_<log2 m>
        _, ln, lm = name.split("_")
        s, d = er(1 << int(ln), 1 << int(lm), 101, nthreads)
        return Graph(1 << int(ln), s, d, name, seed=1)
    raise KeyError(name)


@dataclass
class Batch:
    """Many independent graphs packed back to back: graph g owns local vertex
    ids [0, n[g]) and edges [eoff[g], eoff[g+1]) of src/dst."""
    n: np.ndarray       # uint32 [k]
    eoff: np.ndarray    # uint64 [k+1]
    src: np.ndarray     # uint32 [sum m]
    dst: np.ndarray
    seeds: np.ndarray   # uint64 [k] rank seeds

    @property
    def k(self) -> int:
        return int(self.n.shape[0])

    def graph(self, g: int) -> Graph:
        lo, hi = int(self.eoff[g]), int(self.eoff[g + 1])
        return Graph(int(self.n[g]), self.src[lo:hi], self.dst[lo:hi], "batch%d" % g,
                     seed=int(self.seeds[g]))


def batch(k: int = 4096, lo_exp: float = 6.0, hi_exp: float = 16.0, seed: int = 404,
          nthreads: int = 0) -> Batch:
    """k graphs, n_g = floor(2^U), U ~ U[lo_exp, hi_exp]; even g: ER with m = 2n
    (average degree 4); odd g: R-MAT at scale ceil(log2 n) with ids >= n redrawn,
    m = 8n (average degree 16); rank seed of graph g = g."""
    u = uniforms(seed, k)
    n = np.floor(np.exp2(lo_exp + (hi_exp - lo_exp) * u)).astype(np.uint64)
    n = np.maximum(n, 2)
    m = np.where(np.arange(k) % 2 == 0, 2 * n, 8 * n).astype(np.uint64)
    eoff = np.zeros(k + 1, dtype=np.uint64)
    np.cumsum(m, out=eoff[1:])
    src = np.empty(int(eoff[-1]), dtype=np.uint32)
    dst = np.empty(int(eoff[-1]), dtype=np.uint32)
    lib = _synth()
    for g in range(k):
        lo, hi = int(eoff[g]), int(eoff[g + 1])
        ng = int(n[g])
        gs, gd = src[lo:hi], dst[lo:hi]
        gseed = seed * 1000003 + g
        if g % 2 == 0:
            _check(lib.synth_er(ng, hi - lo, gseed, _ptr(gs), _ptr(gd), nthreads), "er")
        else:
            scale = max(1, int(math.ceil(math.log2(ng))))
            _check(lib.synth_rmat(scale, ng, hi - lo, *RMAT_ABC, gseed, 0,
                                  _ptr(gs), _ptr(gd), nthreads), "rmat")
    return Batch(n.astype(np.uint32), eoff, src, dst, np.arange(k, dtype=np.uint64))


@dataclass
class Request:
    rid: int
    arrival_s: float
    kind: str
    graph: Graph


def serving_stream(rate: float, count: int, lo_exp: float = 10.0, hi_exp: float = 22.0,
                   seed: int = 505, nthreads: int = 0) -> list[Request]:
    """Poisson arrivals at `rate` req/s; each request an ER, R-MAT or permuted 2D
    grid (uniform over the three) with n = floor(2^U), U ~ U[lo_exp, hi_exp],
    average degree uniform in [4, 32] (m = deg * n / 2), rank seed = request id."""
    u = uniforms(seed, 4 * count).reshape(count, 4)
    t = np.cumsum(-np.log1p(-u[:, 0]) / rate)
    out = []
    for r in range(count):
        kind = ("er", "rmat", "grid")[min(2, int(u[r, 1] * 3))]
        n = max(4, int(math.floor(2.0 ** (lo_exp + (hi_exp - lo_exp) * u[r, 2]))))
        deg = 4.0 + 28.0 * u[r, 3]
        gseed = seed * 1000003 + r
        if kind == "er":
            m = max(1, int(deg * n / 2))
            s, d = er(n, m, gseed, nthreads)
        elif kind == "rmat":
            m = max(1, int(deg * n / 2))
            scale = max(1, int(math.ceil(math.log2(n))))
            s, d = rmat(scale, m, gseed, gseed + 1, *RMAT_ABC, n_keep=n, nthreads=nthreads)
        else:
            w = max(2, int(math.isqrt(n)))
            n = w * w
            s, d = grid(w, w, 0, nthreads)
            permute_ids(s, n, gseed, nthreads)
            permute_ids(d, n, gseed, nthreads)
        out.append(Request(r, float(t[r]), kind, Graph(n, s, d, "req%d" % r, seed=r)))
    return out
