"""An independent per-phase construction of LocalContraction, used to pin the
oracle.  It shares no code with ``oracle/lc_oracle.cpp`` and computes each
phase a different way:

* forest: the parent f(v) is the minimum-key vertex of the closed
  neighbourhood (Section 2 N(v)); the arborescences are found as connected
  components of the graph whose edges are {v, f(v)} (scipy), not by pointer
  jumping, and each is named by its unique fixed point f(r) = r;
* two-hop: the label is the minimum key over the radius-2 ball, read off the
  sparsity pattern of (A + I)^2 (Section 3, LocalContraction);
* tree: f(v) over the open neighbourhood; the weakly connected components of
  the f-graph (scipy) are named by the lower-key vertex of their 2-cycle
  (Section 3, TreeContraction; Lemmas lem:cycle, lem:wccs);
* MergeToLarge (Section 5): node sizes and priorities from Python lists of
  member keys, the radius-2 ball of every node of the contracted graph read
  off the sparsity pattern of (A_H + I)^2;
* contraction with Python sets (relabel, drop loops, deduplicate), new ids by
  sorting the surviving names.

Only the vertex ranks come from the oracle (``oracle.ranks``), which the
published SplitMix64 values pin separately.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import oracle

FOREST, TWO_HOP, TREE = 0, 1, 2


def keys(seed: int, i: int, n: int) -> np.ndarray:
    r = oracle.ranks(seed, i, 0, n).astype(np.uint64)
    return (r << np.uint64(32)) | np.arange(n, dtype=np.uint64)


def _sym(n, s, d, loops=True):
    s = np.asarray(s, dtype=np.int64)
    d = np.asarray(d, dtype=np.int64)
    if not loops:
        s, d = s[s != d], d[s != d]
    A = sp.coo_matrix((np.ones(len(s), dtype=np.int8), (s, d)), shape=(n, n)).tocsr()
    A = ((A + A.T) > 0).astype(np.int8)
    if loops:
        A = A + sp.identity(n, dtype=np.int8, format="csr")
    return (A > 0).astype(np.int8).tocsr()


def _row_argmin(M: sp.csr_matrix, key: np.ndarray, empty) -> np.ndarray:
    out = np.empty(M.shape[0], dtype=np.int64)
    for v in range(M.shape[0]):
        cols = M.indices[M.indptr[v]:M.indptr[v + 1]]
        out[v] = empty(v) if cols.size == 0 else int(cols[np.argmin(key[cols])])
    return out


def names_forest(n, s, d, key):
    N = _sym(n, s, d, loops=True)
    f = _row_argmin(N, key, lambda v: v)
    F = sp.coo_matrix((np.ones(n), (np.arange(n), f)), shape=(n, n))
    nc, comp = connected_components(F, directed=False)
    root_of = {}
    for v in range(n):
        if f[v] == v:
            assert comp[v] not in root_of, "two fixed points in one arborescence"
            root_of[comp[v]] = v
    return np.array([root_of[comp[v]] for v in range(n)], dtype=np.int64)


def names_two_hop(n, s, d, key):
    N = _sym(n, s, d, loops=True)
    N2 = ((N @ N) > 0).astype(np.int8).tocsr()
    return _row_argmin(N2, key, lambda v: v)


def names_tree(n, s, d, key):
    N = _sym(n, s, d, loops=False)
    f = _row_argmin(N, key, lambda v: v)
    H = sp.coo_matrix((np.ones(n), (np.arange(n), f)), shape=(n, n))
    nc, comp = connected_components(H, directed=True, connection="weak")
    name_of = {}
    for x in range(n):
        y = int(f[x])
        if y != x and f[y] == x:
            nm = x if key[x] < key[y] else y
            assert name_of.get(comp[x], nm) == nm
            name_of[comp[x]] = nm
    return np.array([name_of.get(comp[v], v) for v in range(n)], dtype=np.int64)


def merge_to_large(n, s, d, name, key, alpha):
    """Replace each vertex's node name by the name of the large node its node
    joins (nodes with >= alpha members are large; priority = the alpha-th
    largest member key; a small node joins the highest-priority large node at
    distance <= 2 in the contracted graph)."""
    members = {}
    for v in range(n):
        members.setdefault(int(name[v]), []).append(int(key[v]))
    prio = {x: sorted(k, reverse=True)[alpha - 1] for x, k in members.items() if len(k) >= alpha}
    a = np.asarray([int(name[u]) for u in s], dtype=np.int64)
    b = np.asarray([int(name[u]) for u in d], dtype=np.int64)
    keep = a != b
    AH = sp.coo_matrix((np.ones(int(keep.sum()), dtype=np.int8), (a[keep], b[keep])),
                       shape=(n, n)).tocsr()
    AH = (((AH + AH.T) > 0).astype(np.int8) + sp.identity(n, dtype=np.int8, format="csr"))
    B2 = ((AH @ AH) > 0).tocsr()
    target = {}
    for x in members:
        if x in prio:
            continue
        ball = B2.indices[B2.indptr[x]:B2.indptr[x + 1]]
        cand = [(prio[int(y)], int(y)) for y in ball if int(y) in prio]
        if cand:
            target[x] = max(cand)[1]
    return np.array([target.get(int(name[v]), int(name[v])) for v in range(n)], dtype=np.int64)


def run(n, s, d, seed, variant=FOREST, finish_edges=0, merge_alpha=()):
    """Returns (labels, [(n_i, m_i)], [mp_i])."""
    s = np.asarray(s, dtype=np.int64)
    d = np.asarray(d, dtype=np.int64)
    # labels: the plain definition (smallest id per weakly connected component)
    if n:
        A = sp.coo_matrix((np.ones(len(s)), (s, d)), shape=(n, n))
        nc, comp = connected_components(A, directed=True, connection="weak")
        first = {}
        for v in range(n):
            first.setdefault(comp[v], v)
        labels = np.array([first[comp[v]] for v in range(n)], dtype=np.uint32)
    else:
        labels = np.zeros(0, dtype=np.uint32)
    sizes, mps = [], []
    ni, es, ed = n, s, d
    i = 0
    namers = {FOREST: names_forest, TWO_HOP: names_two_hop, TREE: names_tree}
    while len(es) > 0:
        if finish_edges and len(es) <= finish_edges:
            A = sp.coo_matrix((np.ones(len(es)), (es, ed)), shape=(ni, ni))
            _, comp = connected_components(A, directed=True, connection="weak")
            rep = {}
            for v in range(ni):
                rep.setdefault(comp[v], v)
            name = np.array([rep[comp[v]] for v in range(ni)], dtype=np.int64)
        else:
            k = keys(seed, i, ni)
            name = namers[variant](ni, es, ed, k)
        mp = int(np.count_nonzero(name[es] != name[ed]))
        if not (finish_edges and len(es) <= finish_edges) and i < len(merge_alpha) \
                and merge_alpha[i] > 0:
            name = merge_to_large(ni, es, ed, name, k, int(merge_alpha[i]))
        rel = [(min(a, b), max(a, b)) for a, b in zip(name[es], name[ed]) if a != b]
        uniq = sorted(set(rel))
        keep = sorted({x for e in uniq for x in e})
        newid = {r: k for k, r in enumerate(keep)}
        sizes.append((ni, len(es)))
        mps.append(mp)
        ni = len(keep)
        es = np.array([newid[a] for a, _ in uniq], dtype=np.int64)
        ed = np.array([newid[b] for _, b in uniq], dtype=np.int64)
        i += 1
    return labels, sizes, mps
