// CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded restatement of the LocalContraction
// connected-components round loop of "Connected Components at Scale via Local
// Contractions" (Lacki, Mirrokni, Wlodarczyk; arXiv 1807.10727).  Only the test
// suite, the smoke check and the benchmark's CPU-baseline leg may load it; the
// GPU library never does, and the two share no code.
//
// Readings of the paper that this file fixes (the paper leaves them open):
//  * rank: SplitMix64 (Steele, Lea, Flood 2014).  Round key
//    k_i = mix(seed + (i+1)*GAMMA) is the (i+1)-th output of a SplitMix64 stream
//    seeded with `seed`; rank_i(v) = mix(k_i + (v+1)*GAMMA) >> 32 is the high half
//    of the (v+1)-th output of the stream seeded with k_i.  The paper asks only
//    for a uniform random priority per vertex, redrawn every phase (Section 3).
//  * ties: key_i(v) = rank_i(v) << 32 | v, so the order is total and ties go to
//    the smaller current id (the paper assumes a one-to-one ordering).
//  * the hashed id in phase i is the vertex's dense id in G_i.
//  * forest variant (default): parent f(v) = argmin of key over the CLOSED
//    neighbourhood N(v), which contains v (Section 2 defines N(v) that way); the
//    relation is "same arborescence of f"; each arborescence is named by its
//    root, found by pointer jumping (Theorem thm:tree-rounds).
//  * two-hop variant: label l(v) = argmin of key over N(N(v)) (Section 3,
//    LocalContraction); vertices with equal label merge; the node is named by
//    the label vertex.
//  * tree variant: f(v) = argmin over N(v) \ {v} (Section 3, TreeContraction);
//    the relation is "same weakly connected component of the f-graph", named by
//    the lower-key vertex of its terminal 2-cycle (Lemmas lem:cycle, lem:wccs).
//    A vertex with no neighbour other than itself is its own node.
//  * contraction: edges are relabelled through the node map, self-loops
//    dropped, duplicates removed (proof of the O(1)-round contraction lemma);
//    nodes left without an edge are isolated and dropped (Section 6, Empirical study); surviving
//    nodes get new dense ids in ascending order of their name.
//  * the loop runs while edges remain (Section 3); R = number of phases run.
//  * final label of v = the smallest original id in v's component, found by
//    composing the per-phase maps c_i (Section 6, Empirical study).
//  * optional finish (off by default): once 0 < m_i <= finish_edges, the phase
//    merges each connected component of G_i into one node by union-find, as the
//    paper's small-graph optimisation does on one machine (Section 6, Empirical study); that
//    phase is counted as a phase.
//  * optional MergeToLarge step (off by default; Section 5, the step used by
//    the O(log log n) analysis on random graphs): with parameter alpha_i for
//    phase i, a node of the contracted graph H is large when at least alpha_i
//    vertices of G_i were merged into it; its priority is the alpha_i-th
//    largest phase-i key among those vertices.  Every node that is not large
//    and has a large node at distance 1 or 2 in H joins the large node of
//    highest priority; large nodes never move (the paper merges small nodes
//    into large ones).  Keys are distinct, so priorities are.  The step is
//    part of phase i (it does not count as a phase) and is skipped in a
//    union-find finish phase.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

namespace {

const uint64_t GAMMA = 0x9E3779B97F4A7C15ULL;

// SplitMix64 output function.
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t round_key(uint64_t seed, uint32_t i) { return mix64(seed + (uint64_t)(i + 1) * GAMMA); }

uint32_t rank_of(uint64_t rk, uint32_t v) { return (uint32_t)(mix64(rk + ((uint64_t)v + 1) * GAMMA) >> 32); }

uint64_t key_of(uint64_t rk, uint32_t v) { return ((uint64_t)rank_of(rk, v) << 32) | v; }

enum { FOREST = 0, TWO_HOP = 1, TREE = 2 };

// Closed-neighbourhood minimum of key over N(v), for every v (Section 2 N(v)).
std::vector<uint64_t> closed_min(uint32_t n, const std::vector<std::pair<uint32_t, uint32_t>>& E,
                                 const std::vector<uint64_t>& val) {
  std::vector<uint64_t> mk(val);
  for (const auto& e : E) {
    mk[e.first] = std::min(mk[e.first], val[e.second]);
    mk[e.second] = std::min(mk[e.second], val[e.first]);
  }
  return mk;
}

// Node name of every vertex of G_i under the chosen variant.  Also reports the
// number of synchronous pointer-jumping steps J (forest and tree variants).
std::vector<uint32_t> node_names(int variant, uint32_t n,
                                 const std::vector<std::pair<uint32_t, uint32_t>>& E,
                                 uint64_t rk, uint32_t* J) {
  std::vector<uint64_t> key(n);
  for (uint32_t v = 0; v < n; ++v) key[v] = key_of(rk, v);
  *J = 0;
  if (variant == FOREST) {
    // f(v) = argmin_{u in N(v)} key(u)
    std::vector<uint64_t> mk = closed_min(n, E, key);
    std::vector<uint32_t> p(n);
    for (uint32_t v = 0; v < n; ++v) p[v] = (uint32_t)mk[v];
    // pointer jumping: after step t, p(v) = f^(2^t)(v); stop when nothing moves
    for (;;) {
      std::vector<uint32_t> q(n);
      bool changed = false;
      for (uint32_t v = 0; v < n; ++v) {
        q[v] = p[p[v]];
        if (q[v] != p[v]) changed = true;
      }
      if (!changed) break;
      p.swap(q);
      ++*J;
    }
    return p;
  }
  if (variant == TWO_HOP) {
    // l(v) = argmin over N(N(v)) = min over u in N(v) of (min over N(u))
    std::vector<uint64_t> mk1 = closed_min(n, E, key);
    std::vector<uint64_t> mk2 = closed_min(n, E, mk1);
    std::vector<uint32_t> l(n);
    for (uint32_t v = 0; v < n; ++v) l[v] = (uint32_t)mk2[v];
    return l;
  }
  // TREE: f(v) = argmin over N(v) \ {v}; vertices without another neighbour keep f(v) = v
  const uint64_t NONE = ~0ULL;
  std::vector<uint64_t> mk(n, NONE);
  for (const auto& e : E) {
    if (e.first == e.second) continue;
    mk[e.first] = std::min(mk[e.first], key[e.second]);
    mk[e.second] = std::min(mk[e.second], key[e.first]);
  }
  std::vector<uint32_t> f(n);
  for (uint32_t v = 0; v < n; ++v) f[v] = mk[v] == NONE ? v : (uint32_t)mk[v];
  // pointer jumping to the terminal 2-cycle: p <- p o p until stable (f^(2^t))
  std::vector<uint32_t> p(f);
  for (;;) {
    std::vector<uint32_t> q(n);
    bool changed = false;
    for (uint32_t v = 0; v < n; ++v) {
      q[v] = p[p[v]];
      if (q[v] != p[v]) changed = true;
    }
    if (!changed) break;
    p.swap(q);
    ++*J;
  }
  // p(v) now lies on v's terminal 2-cycle {x, f(x)}; name = lower key of the pair
  std::vector<uint32_t> name(n);
  for (uint32_t v = 0; v < n; ++v) {
    uint32_t x = p[v], y = f[x];
    name[v] = key[x] <= key[y] ? x : y;
  }
  return name;
}

// MergeToLarge (Section 5) applied to the node names of one phase: H is G_i
// contracted by `name`; name[v] is replaced by the name of the large node
// that v's node joins.
void merge_to_large(uint32_t n, const std::vector<std::pair<uint32_t, uint32_t>>& E,
                    std::vector<uint32_t>& name, uint64_t rk, uint32_t alpha) {
  // members of every node of H (a node is identified by its name)
  std::vector<std::vector<uint64_t>> member_keys(n);
  for (uint32_t v = 0; v < n; ++v) member_keys[name[v]].push_back(key_of(rk, v));
  // priority + 1 of each large node (0: not large): the alpha-th largest key
  std::vector<uint64_t> prio(n, 0);
  for (uint32_t x = 0; x < n; ++x) {
    std::vector<uint64_t>& k = member_keys[x];
    if (alpha == 0 || k.size() < alpha) continue;
    std::sort(k.begin(), k.end(), [](uint64_t a, uint64_t b) { return a > b; });
    prio[x] = k[alpha - 1] + 1;
  }
  // adjacency of H without loops
  std::vector<std::vector<uint32_t>> adj(n);
  for (const auto& e : E) {
    uint32_t a = name[e.first], b = name[e.second];
    if (a == b) continue;
    adj[a].push_back(b);
    adj[b].push_back(a);
  }
  // best priority within distance 1 (h1) and within distance 2 (h2)
  std::vector<uint64_t> h1(prio), h2;
  for (uint32_t x = 0; x < n; ++x)
    for (uint32_t y : adj[x]) h1[x] = std::max(h1[x], prio[y]);
  h2 = h1;
  for (uint32_t x = 0; x < n; ++x)
    for (uint32_t y : adj[x]) h2[x] = std::max(h2[x], h1[y]);
  // a priority is a member's key, whose low half is that member's id
  std::vector<uint32_t> target(n);
  for (uint32_t x = 0; x < n; ++x) {
    target[x] = x;
    if (prio[x] == 0 && h2[x] != 0) target[x] = name[(uint32_t)(h2[x] - 1)];
  }
  for (uint32_t v = 0; v < n; ++v) name[v] = target[name[v]];
}

// Union-find with path halving; find returns the set's root.
struct UF {
  std::vector<uint32_t> par;
  explicit UF(uint32_t n) : par(n) {
    for (uint32_t v = 0; v < n; ++v) par[v] = v;
  }
  uint32_t find(uint32_t x) {
    while (par[x] != x) {
      par[x] = par[par[x]];
      x = par[x];
    }
    return x;
  }
  void unite(uint32_t a, uint32_t b) {
    a = find(a);
    b = find(b);
    if (a == b) return;
    if (a < b) par[b] = a; else par[a] = b;
  }
};

}  // namespace

extern "C" {

// One output of the SplitMix64 stream: advance *state by GAMMA, return mix64.
uint64_t oracle_splitmix64_next(uint64_t* state) {
  *state += GAMMA;
  return mix64(*state);
}

uint64_t oracle_round_key(uint64_t seed, uint32_t i) { return round_key(seed, i); }

uint32_t oracle_rank(uint64_t seed, uint32_t i, uint32_t v) { return rank_of(round_key(seed, i), v); }

// out[j] = rank of vertex v0 + j in phase i, for j < count.
void oracle_ranks(uint64_t seed, uint32_t i, uint32_t v0, uint32_t count, uint32_t* out) {
  uint64_t rk = round_key(seed, i);
  for (uint32_t j = 0; j < count; ++j) out[j] = rank_of(rk, v0 + j);
}

// Component labels by union-find: labels[v] = smallest vertex id in v's
// component (the plain definition of the result, Section 2).
int oracle_uf_labels(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t m,
                     uint32_t* labels) {
  for (uint64_t j = 0; j < m; ++j)
    if (src[j] >= n || dst[j] >= n) return 1;
  UF uf(n);
  for (uint64_t j = 0; j < m; ++j) uf.unite(src[j], dst[j]);
  // with union by smaller id, every root is its set's minimum
  for (uint32_t v = 0; v < n; ++v) labels[v] = uf.find(v);
  return 0;
}

// Per-phase node names for one phase on the given graph (diagnostic access for
// tests: phase index i selects the rank).
int oracle_node_names(int variant, uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t m,
                      uint64_t seed, uint32_t i, uint32_t* names, uint32_t* J) {
  std::vector<std::pair<uint32_t, uint32_t>> E(m);
  for (uint64_t j = 0; j < m; ++j) {
    if (src[j] >= n || dst[j] >= n) return 1;
    E[j] = {src[j], dst[j]};
  }
  std::vector<uint32_t> nm = node_names(variant, n, E, round_key(seed, i), J);
  std::copy(nm.begin(), nm.end(), names);
  return 0;
}

// The whole round loop; alpha[i] (i < alpha_count, 0 = off) is the
// MergeToLarge parameter of phase i.  Outputs: labels[n]; *rounds = R; n_i, m_i, mp_i
// (edges after relabel and loop removal, before deduplication) and J_i for
// i < min(R, cap).  Returns 0 on success, 1 on invalid input, 2 when R > cap
// (outputs up to cap are valid, labels are not written), 3 when max_rounds is
// exceeded.
int oracle_lc_run(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t m, uint64_t seed,
                  int variant, uint64_t finish_edges, const uint32_t* alpha,
                  uint32_t alpha_count, uint32_t max_rounds, uint32_t* labels,
                  uint32_t* rounds, uint64_t* n_i, uint64_t* m_i, uint64_t* mp_i, uint32_t* J_i,
                  uint32_t cap) {
  if (variant < FOREST || variant > TREE) return 1;
  std::vector<std::pair<uint32_t, uint32_t>> E(m);
  for (uint64_t j = 0; j < m; ++j) {
    if (src[j] >= n || dst[j] >= n) return 1;
    E[j] = {src[j], dst[j]};
  }
  // Per phase: name[v] of every vertex of G_i, and newid[name] (or DROPPED).
  const uint32_t DROPPED = 0xFFFFFFFFu;
  std::vector<std::vector<uint32_t>> names, newids;
  uint32_t ni = n;
  uint32_t i = 0;
  while (!E.empty()) {
    if (i >= max_rounds) return 3;
    uint32_t J = 0;
    bool merge = false;
    std::vector<uint32_t> name;
    if (finish_edges > 0 && E.size() <= finish_edges) {
      UF uf(ni);
      for (const auto& e : E) uf.unite(e.first, e.second);
      name.resize(ni);
      for (uint32_t v = 0; v < ni; ++v) name[v] = uf.find(v);
    } else {
      name = node_names(variant, ni, E, round_key(seed, i), &J);
      merge = i < alpha_count && alpha[i] > 0;
    }
    // m'_i: edges that the phase's contraction leaves, loops dropped, before
    // deduplication (and before a MergeToLarge step, which works on the
    // contracted graph)
    uint64_t mprime = 0;
    for (const auto& e : E) mprime += name[e.first] != name[e.second] ? 1 : 0;
    if (merge) merge_to_large(ni, E, name, round_key(seed, i), alpha[i]);
    // relabel every edge through the names, drop self-loops (the contraction)
    std::vector<std::pair<uint32_t, uint32_t>> E1;
    E1.reserve(E.size());
    for (const auto& e : E) {
      uint32_t a = name[e.first], b = name[e.second];
      if (a == b) continue;
      E1.push_back({std::min(a, b), std::max(a, b)});
    }
    // remove duplicates
    std::sort(E1.begin(), E1.end());
    E1.erase(std::unique(E1.begin(), E1.end()), E1.end());
    // surviving nodes: names that appear in an edge; dense ids by ascending name
    std::vector<uint32_t> newid(ni, DROPPED);
    std::vector<char> keep(ni, 0);
    for (const auto& e : E1) keep[e.first] = keep[e.second] = 1;
    uint32_t next = 0;
    for (uint32_t r = 0; r < ni; ++r)
      if (keep[r]) newid[r] = next++;
    for (auto& e : E1) e = {newid[e.first], newid[e.second]};
    if (i < cap) {
      n_i[i] = ni;
      m_i[i] = E.size();
      mp_i[i] = mprime;
      J_i[i] = J;
    }
    names.push_back(std::move(name));
    newids.push_back(std::move(newid));
    E.swap(E1);
    ni = next;
    ++i;
  }
  *rounds = i;
  if (i > cap) return 2;
  // compose the maps c_i: follow each vertex until its node is dropped; the
  // final node is (phase, name); its label is the smallest original id in it
  std::vector<std::vector<uint32_t>> minid(names.size());
  for (size_t k = 0; k < names.size(); ++k) minid[k].assign(names[k].size(), DROPPED);
  std::vector<uint32_t> id_minlabel(n, DROPPED);  // components finished before phase 0 (no phases)
  for (uint32_t v = 0; v < n; ++v) {
    uint32_t x = v;
    size_t k = 0;
    bool done = false;
    while (k < names.size()) {
      uint32_t r = names[k][x];
      if (newids[k][r] == DROPPED) {
        if (minid[k][r] == DROPPED) minid[k][r] = v;  // v ascending: first visitor is the minimum
        labels[v] = minid[k][r];
        done = true;
        break;
      }
      x = newids[k][r];
      ++k;
    }
    if (!done) labels[v] = v;  // R = 0: every vertex is its own component
  }
  return 0;
}

}  // extern "C"
