"""Pins of the CPU oracle against facts fixed outside it (published values,
closed forms, brute force, library connected components, an independent
per-phase construction).  CPU only."""
import itertools
import os
import random
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import oracle
from tests import phase_ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MASK64 = (1 << 64) - 1


def scipy_labels(n, s, d):
    A = sp.coo_matrix((np.ones(len(s)), (np.asarray(s), np.asarray(d))), shape=(n, n))
    _, comp = connected_components(A, directed=True, connection="weak")
    first = {}
    return np.array([first.setdefault(c, v) for v, c in enumerate(comp)], dtype=np.uint32)


def random_graph(rng, n, m, loops=True):
    s = rng.integers(0, n, m).astype(np.uint32)
    d = rng.integers(0, n, m).astype(np.uint32)
    if not loops:
        keep = s != d
        s, d = s[keep], d[keep]
    return s, d


# ------------------------------------------------------------- ranking

def read_golden_splitmix():
    seed, outs = None, []
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("seed"):
                seed = int(line.split()[1])
            else:
                outs.append(int(line))
    return seed, outs


def check_splitmix_vector():
    seed, outs = read_golden_splitmix()
    state = seed
    got = []
    for _ in outs:
        o, state = oracle.splitmix64_next(state)
        got.append(o)
    return got == outs


def test_splitmix64_published_values():
    assert check_splitmix_vector()


def check_rank_composition(seeds=(0, 1, 7, 12345678901234), phases=(0, 1, 5), ids=(0, 1, 2, 1000, 2**32 - 2)):
    """rank_i(v) = high half of output v+1 of the stream seeded with output
    i+1 of the stream seeded with the run seed (streams stepped with the
    pinned generator)."""
    for seed in seeds:
        state = seed
        for i in range(max(phases) + 1):
            rk, state = oracle.splitmix64_next(state)
            if i not in phases:
                continue
            for v in ids:
                # output v+1 of the stream seeded with rk: state rk + (v+1)*gamma
                o, _ = oracle.splitmix64_next((rk + v * 0x9E3779B97F4A7C15) & MASK64)
                if oracle.rank(seed, i, v) != (o >> 32):
                    return False
    return True


def test_rank_is_splitmix_stream_composition():
    assert check_rank_composition()


def test_vectorised_ranks_match_scalar():
    r = oracle.ranks(99, 3, 2**32 - 100, 99)
    assert all(int(r[j]) == oracle.rank(99, 3, 2**32 - 100 + j) for j in range(99))


def test_ranks_look_uniform():
    r = oracle.ranks(5, 0, 0, 1 << 16).astype(np.float64) / 2**32
    assert abs(r.mean() - 0.5) < 0.01
    hist = np.histogram(r, bins=16, range=(0, 1))[0]
    assert hist.min() > 0.9 * (1 << 12) and hist.max() < 1.1 * (1 << 12)


# ------------------------------------------------------- labels (exact)

def test_uf_labels_match_scipy():
    rng = np.random.default_rng(3)
    for n, m in [(1, 0), (5, 0), (10, 4), (100, 80), (1000, 600), (5000, 20000)]:
        s, d = random_graph(rng, n, m)
        assert np.array_equal(oracle.uf_labels(n, s, d), scipy_labels(n, s, d))


def bfs_labels(n, edges):
    adj = {v: set() for v in range(n)}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    lab = [-1] * n
    for v in range(n):
        if lab[v] >= 0:
            continue
        stack, lab[v] = [v], v
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if lab[y] < 0:
                    lab[y] = v
                    stack.append(y)
    return np.array(lab, dtype=np.uint32)


@pytest.mark.parametrize("variant", [oracle.FOREST, oracle.TWO_HOP, oracle.TREE])
def test_every_graph_on_up_to_5_vertices(variant):
    """Brute force: every simple graph on n <= 5 labelled vertices, 2 seeds:
    labels against BFS, per-phase sizes against the independent construction."""
    for n in range(1, 6):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            edges = [pairs[k] for k in range(len(pairs)) if mask >> k & 1]
            s = np.array([a for a, _ in edges], dtype=np.uint32)
            d = np.array([b for _, b in edges], dtype=np.uint32)
            for seed in (1, 2):
                r = oracle.lc_run(n, s, d, seed, variant)
                assert np.array_equal(r.labels, bfs_labels(n, edges))
                if mask % 7 == 0 or n < 5:
                    _, sizes, mps = phase_ref.run(n, s, d, seed, variant)
                    assert r.sizes() == sizes and list(r.mp_i) == mps, (n, edges, seed)


@pytest.mark.parametrize("variant", [oracle.FOREST, oracle.TWO_HOP, oracle.TREE])
def test_phases_match_independent_construction(variant):
    rng = np.random.default_rng(11 + variant)
    cases = [(8, 12), (30, 30), (60, 200), (200, 300), (300, 1500), (500, 400)]
    for n, m in cases:
        for seed in (0, 5):
            s, d = random_graph(rng, n, m)
            r = oracle.lc_run(n, s, d, seed, variant)
            labels, sizes, mps = phase_ref.run(n, s, d, seed, variant)
            assert np.array_equal(r.labels, labels)
            assert r.sizes() == sizes
            assert list(r.mp_i) == mps


def test_finish_matches_independent_construction():
    rng = np.random.default_rng(21)
    for n, m, fin in [(200, 300, 50), (400, 1200, 400), (100, 90, 1000)]:
        s, d = random_graph(rng, n, m)
        r = oracle.lc_run(n, s, d, 4, oracle.FOREST, finish_edges=fin)
        labels, sizes, mps = phase_ref.run(n, s, d, 4, oracle.FOREST, finish_edges=fin)
        assert np.array_equal(r.labels, labels)
        assert r.sizes() == sizes and list(r.mp_i) == mps
        assert int(r.m_i[-1]) <= fin


@pytest.mark.parametrize("variant", [oracle.FOREST, oracle.TWO_HOP, oracle.TREE])
def test_merge_to_large_matches_independent_construction(variant):
    """MergeToLarge (Section 5) against the radius-2-ball construction."""
    rng = np.random.default_rng(41 + variant)
    for n, m in [(12, 20), (40, 60), (80, 240), (200, 300), (300, 1200)]:
        for alpha in ([2], [3, 2], [4, 4, 4], [0, 3], [6, 1, 2]):
            s, d = random_graph(rng, n, m)
            r = oracle.lc_run(n, s, d, 7, variant, merge_alpha=alpha)
            labels, sizes, mps = phase_ref.run(n, s, d, 7, variant, merge_alpha=alpha)
            assert np.array_equal(r.labels, labels)
            assert r.sizes() == sizes and list(r.mp_i) == mps, (n, m, alpha)


def test_merge_to_large_degenerate_parameters():
    """alpha = 1 makes every node large (nobody moves); alpha above the vertex
    count makes none large: both give the run without the step."""
    rng = np.random.default_rng(43)
    for n, m in [(50, 80), (300, 900)]:
        s, d = random_graph(rng, n, m)
        for variant in (oracle.FOREST, oracle.TWO_HOP, oracle.TREE):
            plain = oracle.lc_run(n, s, d, 2, variant)
            for alpha in ([1] * 8, [n + 1] * 8):
                r = oracle.lc_run(n, s, d, 2, variant, merge_alpha=alpha)
                assert r.sizes() == plain.sizes() and np.array_equal(r.labels, plain.labels)


def test_merge_to_large_coarsens_the_first_phase():
    """The step only merges nodes, so G_1 never has more vertices or edges
    than without it, and labels do not change."""
    rng = np.random.default_rng(47)
    for t in range(30):
        n = int(rng.integers(20, 400))
        s, d = random_graph(rng, n, int(rng.integers(n, 4 * n)))
        plain = oracle.lc_run(n, s, d, t, oracle.FOREST)
        r = oracle.lc_run(n, s, d, t, oracle.FOREST, merge_alpha=[int(rng.integers(2, 8))])
        assert np.array_equal(r.labels, plain.labels)
        if plain.rounds > 1:
            assert r.rounds == 1 or (r.n_i[1] <= plain.n_i[1] and r.m_i[1] <= plain.m_i[1])


def test_merge_to_large_random_graph_lemma():
    """Lemma lem:random: for G ~ G(n, alpha/n) with alpha >= (4 + 4c) ln n, one
    phase of LocalContraction (two-hop label) with MergeToLarge parameter
    alpha / 4 leaves at most n / alpha vertices w.h.p. (c = 1 here)."""
    import math
    for n, seed in [(2048, 1), (4096, 2), (8192, 3)]:
        alpha = 8 * math.log(n)
        m = int(round(alpha / n * n * (n - 1) / 2))
        rng = np.random.default_rng(seed)
        s, d = rng.integers(0, n, m), rng.integers(0, n, m)
        r = oracle.lc_run(n, s, d, seed, oracle.TWO_HOP, merge_alpha=[int(alpha / 4)])
        assert r.rounds == 1 or r.n_i[1] <= n / alpha


def test_workload_labels_match_union_find_and_scipy():
    from paper_1807_10727_gb300 import synth
    for name in ("er16", "rmat14", "gridmix_small"):
        g = synth.workload(name)
        ref = scipy_labels(g.n, g.src, g.dst)
        assert np.array_equal(oracle.uf_labels(g.n, g.src, g.dst), ref)
        for variant in (oracle.FOREST, oracle.TWO_HOP, oracle.TREE):
            assert np.array_equal(oracle.lc_run(g.n, g.src, g.dst, g.seed, variant).labels, ref)


def test_er_workload_phases_match_independent_construction():
    """A 4096-vertex slice of the ER recipe checked phase by phase."""
    from paper_1807_10727_gb300 import synth
    s, d = synth.er(4096, 1 << 15, 101)
    r = oracle.lc_run(4096, s, d, 1)
    _, sizes, mps = phase_ref.run(4096, s, d, 1)
    assert r.sizes() == sizes and list(r.mp_i) == mps


# --------------------------------------------------------- closed forms

def keys_of(seed, i, n):
    return [(oracle.rank(seed, i, v) << 32) | v for v in range(n)]


def test_empty_and_loop_only_inputs():
    r = oracle.lc_run(7, [], [], 1)
    assert r.rounds == 0 and list(r.labels) == list(range(7))
    r = oracle.lc_run(5, [0, 3, 3], [0, 3, 3], 1)
    assert r.rounds == 1 and r.sizes() == [(5, 3)] and list(r.mp_i) == [0]
    assert list(r.labels) == list(range(5))


@pytest.mark.parametrize("n", [2, 3, 10, 40])
def test_complete_graph_one_phase(n):
    pairs = list(itertools.combinations(range(n), 2))
    s = [a for a, _ in pairs]
    d = [b for _, b in pairs]
    for seed in range(4):
        r = oracle.lc_run(n, s, d, seed)
        assert r.rounds == 1 and r.sizes() == [(n, len(pairs))]
        assert list(r.labels) == [0] * n


@pytest.mark.parametrize("k", [1, 2, 5, 31])
def test_star_closed_form(k):
    """Star with centre 0: the leaves ranked below the centre are roots; the
    global minimum's tree takes the centre; phase 1 is a star on those leaves."""
    s = [0] * k
    d = list(range(1, k + 1))
    for seed in range(12):
        key = keys_of(seed, 0, k + 1)
        low = sum(1 for v in range(1, k + 1) if key[v] < key[0])
        r = oracle.lc_run(k + 1, s, d, seed)
        if low <= 1:
            assert r.rounds == 1
        else:
            assert r.sizes()[1] == (low, low - 1)


@pytest.mark.parametrize("n", [2, 3, 9, 50, 301])
def test_path_and_cycle_local_minima(n):
    """On a path or cycle the trees are runs between local minima: phase 1 has
    one node per local minimum, joined as a path (cycle)."""
    for cyc in (False, True):
        if cyc and n < 3:
            continue
        s = list(range(n - 1)) + ([n - 1] if cyc else [])
        d = list(range(1, n)) + ([0] if cyc else [])
        for seed in range(6):
            key = keys_of(seed, 0, n)

            def nb(v):
                out = [v]
                if v > 0 or cyc:
                    out.append((v - 1) % n)
                if v < n - 1 or cyc:
                    out.append((v + 1) % n)
                return out

            minima = sum(1 for v in range(n) if min(nb(v), key=lambda u: key[u]) == v)
            r = oracle.lc_run(n, s, d, seed)
            if minima == 1:
                assert r.rounds == 1
            else:
                n1, m1 = r.sizes()[1]
                assert n1 == minima
                assert m1 == (minima if cyc and minima >= 3 else minima - 1)


# ------------------------------------------------------------ invariants

def test_invariants_on_generated_graphs():
    from paper_1807_10727_gb300 import synth
    for name in ("er16", "rmat16", "gridmix_small"):
        g = synth.workload(name)
        r = oracle.lc_run(g.n, g.src, g.dst, g.seed)
        assert r.rounds <= g.n
        for i in range(r.rounds):
            assert r.mp_i[i] <= r.m_i[i]
            if i + 1 < r.rounds:
                assert r.m_i[i + 1] <= r.mp_i[i]
                assert r.n_i[i + 1] < r.n_i[i]
        # after phase 0 the edges are simple, so every phase removes at least
        # the parent edge of each non-root
        for i in range(1, r.rounds - 1):
            assert r.m_i[i + 1] < r.m_i[i]


def test_first_phase_shrinks_er_vertices():
    """Section 4's counting argument: a phase keeps at most 3/4 of the
    vertices in expectation; on the ER workload the forest reading keeps far
    fewer (the roots are local minima)."""
    from paper_1807_10727_gb300 import synth
    g = synth.workload("er16")
    r = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    assert r.n_i[1] <= 0.75 * r.n_i[0]


# ------------------------------------------------------ planted mistakes

MUTANTS = {
    "dropped +1 in the hashed id": ("((uint64_t)v + 1) * GAMMA", "((uint64_t)v) * GAMMA"),
    "no deduplication": ("E1.erase(std::unique(E1.begin(), E1.end()), E1.end());", ""),
    "one pointer-jumping step only": ("      if (!changed) break;\n      p.swap(q);\n      ++*J;\n    }\n    return p;",
                                      "      p.swap(q);\n      ++*J;\n      break;\n    }\n    return p;"),
    "isolated nodes kept": ("for (const auto& e : E1) keep[e.first] = keep[e.second] = 1;",
                            "for (uint32_t r = 0; r < ni; ++r) keep[r] = name[r] == r;"),
    "wrong SplitMix constant": ("0x94D049BB133111EBULL", "0x94D049BB133111EAULL"),
    "two-hop reads one hop": ("std::vector<uint64_t> mk2 = closed_min(n, E, mk1);",
                              "std::vector<uint64_t> mk2 = mk1;"),
    "merge priority = alpha-th smallest key": ("[](uint64_t a, uint64_t b) { return a > b; }",
                                               "[](uint64_t a, uint64_t b) { return a < b; }"),
    "merge looks one hop only": ("  h2 = h1;\n  for (uint32_t x = 0; x < n; ++x)\n    for (uint32_t y : adj[x]) h2[x] = std::max(h2[x], h1[y]);",
                                 "  h2 = h1;"),
    "merge moves large nodes too": ("if (prio[x] == 0 && h2[x] != 0)", "if (h2[x] != 0 && h2[x] != prio[x])"),
    "merge size counts one short": ("k.size() < alpha", "k.size() <= alpha"),
}


def pins_pass():
    rng = np.random.default_rng(5)
    if not check_splitmix_vector() or not check_rank_composition():
        return False
    for variant in (oracle.FOREST, oracle.TWO_HOP):
        for n, m in [(40, 50), (200, 600)]:
            s, d = random_graph(rng, n, m)
            r = oracle.lc_run(n, s, d, 3, variant)
            labels, sizes, mps = phase_ref.run(n, s, d, 3, variant)
            if not (np.array_equal(r.labels, labels) and r.sizes() == sizes and list(r.mp_i) == mps):
                return False
    for variant in (oracle.FOREST, oracle.TREE):
        for n, m, alpha in [(80, 240, [3, 2]), (200, 300, [4]), (300, 1200, [2, 3])]:
            s, d = random_graph(rng, n, m)
            r = oracle.lc_run(n, s, d, 7, variant, merge_alpha=alpha)
            labels, sizes, mps = phase_ref.run(n, s, d, 7, variant, merge_alpha=alpha)
            if not (np.array_equal(r.labels, labels) and r.sizes() == sizes and list(r.mp_i) == mps):
                return False
    return True


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(mutant, tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    src = open(os.path.join(os.path.dirname(oracle.__file__), "lc_oracle.cpp")).read()
    old, new = MUTANTS[mutant]
    assert old in src, "mutant anchor not found"
    path = tmp_path / "mut.cpp"
    path.write_text(src.replace(old, new, 1))
    so = str(tmp_path / "libmut.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", str(path), "-o", so], check=True)
    assert pins_pass()  # the real oracle passes
    with oracle.using_library(so):
        assert not pins_pass(), "planted mistake not caught: " + mutant
