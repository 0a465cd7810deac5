// CPU oracle for round-synchronous contraction-hierarchy construction and
// CH s-t queries.
//
// TEST INFRASTRUCTURE. This file is the reference the CUDA path is checked
// against. Only the test suite, the smoke check and the benchmark's CPU
// baseline leg load it; the library's product path never does. It shares no
// code, header, table or helper with the CUDA path.
//
// It is deliberately plain: single-threaded (a build with -DORACLE_THREADS
// runs each phase's witness searches on all host threads, with identical
// results), ordered std::map adjacency,
// every step applied literally in the order the paper gives it, no blocking,
// no fusion; the one cut inside a search (labels that cannot decide
// anything) is stated where it is made. Where the paper leaves a detail open
// the reading taken is stated next to the code.
//
// Paper passages followed (arXiv 2412.18008):
//   Sec. 2 notation: N_in, N_out, N over the overlay graph G_O.
//   Alg. 2  round loop: LocalSearch -> Score -> Select -> Contract, then the
//           affected set becomes N(V_F); Postprocess at the end.
//   Alg. 3  LocalSearch: searches batched per source s, with target set
//           V_n = union of N_out(u) over u in N_out(s) and u in the affected set.
//   Alg. 4  Score: P[u] = -(edges of u) + #{(v1, v2) : a shortcut is needed}.
//   Alg. 5  Select: u is chosen iff its score is below every neighbour's,
//           ties broken by a per-vertex label.
//   Alg. 6  Contract: in-edges of u go to the downward set, out-edges to the
//           upward set, surviving in x out pairs become shortcuts, u and its
//           edges leave the overlay.
//   Sec. 4  duplicate shortcuts (u-c1-v and u-c2-v) keep the smallest weight.
//   Sec. 3.5 Postprocess: vertices ordered by level, then by score.
//   Sec. 5  Query: upward search from s on the upward edges, upward search
//           from t on the reversed downward edges, answer = min over meeting
//           vertices of d_s(v) + d_t(v).
//
// Readings of points the paper leaves open:
//   * Witness search: the paper bounds each Dijkstra by a settled-vertex cap
//     whose value it never gives. Here the witness distance is the hop-limited
//     distance d_H(a, b) = least weight of a walk a -> b with at most H edges
//     in the current overlay graph (INF if none), which is exact and does not
//     depend on any visiting order. The contracted vertex itself is not
//     excluded from the search. An optional ball bound stands in for the
//     cap: the search from a stops after the first hop level h at which more
//     than `ball` vertices hold a label below a's heaviest candidate weight,
//     and d_h replaces d_H (still an upper bound on a real walk, so the
//     distances stay exact; only more shortcuts may be kept). Unbounded by
//     default.
//   * Level-work bound (optional): a hop-limited search does not run a
//     level, from the second on, whose frontier (the vertices whose label
//     dropped in the level before) has more out-edges in total than the
//     bound; the labels of the level before are its result. Like the ball
//     bound it only drops witnesses, so distances stay exact. It keeps
//     searches from expanding hubs of power-law graphs.
//   * Settled-vertex cap (optional, theta > 0): the search of Alg. 3 as
//     written, a Dijkstra from the source that stops when all its targets or
//     theta vertices are settled; an unsettled target's distance is INF.
//     Equal labels are settled in id order, which makes the cap exact: the
//     settled set is the first theta vertices in (distance, id) order. The
//     hop limit and the ball bound do not apply in this mode.
//   * Pruning (optional): after the searches of a round's LocalSearch, every
//     overlay edge (s, v) heavier than the distance recorded for (s, v) is
//     deleted (Alg. 3), before Score; the searches all see the overlay as it
//     was before any deletion.
//   * Memoisation (optional): the distance map outlives the phase (Alg. 3's
//     dist); a pair already in it is not searched again, and a source none
//     of whose targets is new is not searched at all. Each search drops
//     labels at or above the heaviest weight it has to decide (its new
//     targets' candidate weights and, with pruning, the direct edges to
//     them), so the value kept is the label the search held, else INF. The
//     map is cleared at the end of a round that leaves more entries than a
//     given limit (the paper clears its table lazily, once it is filled to
//     a constant fraction). An old value is the weight of a walk in an
//     earlier overlay, so it bounds the distance from above and the
//     argument below still holds.
//   * Shortcut predicate: a candidate (v1, u, v2) with v1 != v2 is kept iff
//     w(v1,u) + w(u,v2) <= d_H(v1, v2). For H >= 2 this is the paper's
//     "equals the witness distance" test; for H < 2 it is its natural
//     extension (the pair's distance is not known, so the shortcut stays).
//   * Edge term of the score: the prose defines edge difference with the
//     number of edges incident to u, so P[u] subtracts |N_in(u)| + |N_out(u)|.
//   * Tie-break label: either the vertex id itself, or the MurmurHash3 32-bit
//     finaliser of (id XOR seed), a bijection on 32-bit words, so that a chain
//     or a row-major grid does not get a single local minimum per round.
//   * Rescoring: only the affected set A_r = N(V_F of round r-1) is rescored,
//     other scores stay as they were. Contraction decisions use fresh
//     witness distances on the overlay of the current round.
//   * Merge: among kept candidates with the same (v1, v2), the smallest
//     weight wins, ties to the smallest contracted vertex id; it is inserted
//     when (v1, v2) is not an overlay edge or its weight is strictly smaller
//     than the existing edge's, which it then replaces. Each such insertion
//     is one shortcut.
//   * Saturation: sums are computed exactly and any sum >= 2^32 - 1 is INF. A
//     candidate whose via-weight is INF is never kept: it cannot lie on a
//     path shorter than INF, so no representable distance needs it.
//   * Rank: by (level, score at contraction, id), all ascending.
//   * Candidate bound Cmax (partial hierarchy): a rescored vertex u with
//     |N_in(u)| * |N_out(u)| > Cmax is not eligible: it is not scored (no
//     witness search; its score becomes INT32_MAX - 1) and never selected,
//     until a later rescoring finds it within the bound. When a round finds
//     no eligible vertex, the live vertices form the core: they all get that
//     round's index as their level, their overlay out- and in-edges become
//     E_up and E_down as if contracted (no shortcuts), and construction
//     stops; that last round has no statistics row. The upward searches of
//     a query then also run every core-core edge in their direction, which
//     is a full search inside the core. Cmax = 2^64 - 1 contracts every
//     vertex.
//
// Why the result preserves every distance, for any H, tie-break or score:
// take a shortest path in the round-r overlay between two vertices that
// survive the round. Each contracted vertex u on it has its predecessor a and
// successor b outside V_F (V_F is independent) and a != b (weights are >= 1),
// and w(a,u) + w(u,b) = dist(a, b) <= d_H(a, b), so (a, b) is kept, and the
// edge (a, b) of the next overlay weighs at most that. Every shortcut weighs
// as much as a real walk, so no distance can drop below the true one. A
// pruned edge (s, v) weighs more than dist(s, v), so it lies on no shortest
// path, and deleting any number of such edges at once changes no distance.

#include <algorithm>
#include <array>
#ifdef ORACLE_THREADS
#include <thread>
#endif
#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <queue>
#include <stdexcept>
#include <tuple>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

constexpr uint32_t INF = 0xFFFFFFFFu;

constexpr int ORC_OK = 0;
constexpr int ORC_EINVAL = -1;

enum StatField {
    ST_AFFECTED = 0,      // |A_r|
    ST_SCORE_SOURCES,     // |N_in(A_r)|
    ST_SELECTED,          // |V_F|
    ST_CONTRACT_SOURCES,  // |N_in(V_F)|
    ST_CANDIDATES,        // in x out pairs of V_F with v1 != v2
    ST_KEPT,              // candidates passing the witness test
    ST_MERGED,            // distinct (v1, v2) among kept
    ST_INSERTED,          // shortcuts written into the overlay
    ST_VO_AFTER,          // live vertices after the round
    ST_EO_AFTER,          // live directed edges after the round
    NSTAT
};

uint32_t sat_add(uint32_t a, uint32_t b) {
    uint64_t s = uint64_t(a) + uint64_t(b);
    return s >= INF ? INF : uint32_t(s);
}

// MurmurHash3 fmix32 (Appleby): a bijection on 32-bit words.
uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

using Adj = std::map<uint32_t, uint32_t>;  // neighbour -> weight

struct Overlay {
    std::vector<Adj> out, in;
    std::vector<char> alive;
};

bool validate(uint32_t n, uint64_t m, const uint64_t* off, const uint32_t* tgt,
              const uint32_t* w) {
    if (n == 0) return m == 0;
    if (!off || off[0] != 0 || off[n] != m) return false;
    for (uint32_t u = 0; u < n; ++u)
        if (off[u] > off[u + 1]) return false;
    for (uint64_t e = 0; e < m; ++e) {
        if (tgt[e] >= n) return false;
        if (w[e] == 0 || w[e] == INF) return false;
    }
    return true;
}

// Input normalisation: drop self-loops, merge parallel edges by min weight.
void load(Overlay& g, uint32_t n, const uint64_t* off, const uint32_t* tgt,
          const uint32_t* w) {
    g.out.assign(n, Adj());
    g.in.assign(n, Adj());
    g.alive.assign(n, 1);
    for (uint32_t u = 0; u < n; ++u) {
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint32_t v = tgt[e];
            if (v == u) continue;
            auto it = g.out[u].find(v);
            if (it == g.out[u].end() || w[e] < it->second) {
                g.out[u][v] = w[e];
                g.in[v][u] = w[e];
            }
        }
    }
}

// Hop-limited distances from one source: d_k(y) = min(d_{k-1}(y),
// min_x d_{k-1}(x) + w(x, y)), k = 1..H, starting from d_0 = {s: 0}. Every
// level re-relaxes all edges out of every vertex reached so far using the
// previous level's values, exactly as the recurrence reads.
struct HopSearch {
    std::vector<uint32_t> prev, cur, mark;
    std::vector<char> seen;
    std::vector<uint32_t> reached, front, next;
    uint64_t work = 0;  // out-edges of the frontier vertices of every level run, summed

    explicit HopSearch(uint32_t n) : prev(n, INF), cur(n, INF), mark(n, 0), seen(n, 0) {}

    // Levels 1..H of a hop-synchronous search from s that keeps only labels
    // below `bound` (a walk at or above the bound cannot decide a candidate:
    // keep(via, d) holds for every via <= bound whenever d >= bound). After
    // each level, if more than `ball` vertices (s included) hold a label, the
    // search stops there and the labels of that level are its result. The
    // frontier of a level is s (level 1) or the vertices whose label dropped
    // in the level before; only their out-edges can lower a label. With a
    // finite `level_work`, a level from the second on whose frontier has
    // more than that many out-edges in total is not run, and the labels of
    // the level before are the result.
    void run(const std::vector<Adj>& out, uint32_t s, uint32_t H, uint32_t bound = INF,
             uint64_t ball = ~uint64_t(0), uint64_t level_work = ~uint64_t(0)) {
        for (uint32_t x : reached) {
            prev[x] = cur[x] = INF;
            seen[x] = 0;
            mark[x] = 0;
        }
        reached.clear();
        prev[s] = cur[s] = 0;
        seen[s] = 1;
        reached.push_back(s);
        front.assign(1, s);
        for (uint32_t k = 1; k <= H; ++k) {
            uint64_t wk = 0;
            for (uint32_t x : front) wk += out[x].size();
            if (k >= 2 && wk > level_work) break;
            work += wk;
            next.clear();
            size_t R = reached.size();
            for (size_t i = 0; i < R; ++i) {
                uint32_t x = reached[i];
                uint32_t dx = prev[x];
                for (const auto& [y, wy] : out[x]) {
                    uint32_t nd = sat_add(dx, wy);
                    if (nd < bound && nd < cur[y]) {
                        cur[y] = nd;
                        if (!seen[y]) {
                            seen[y] = 1;
                            reached.push_back(y);
                        }
                        if (mark[y] != k) {
                            mark[y] = k;
                            next.push_back(y);
                        }
                    }
                }
            }
            for (uint32_t x : reached) prev[x] = cur[x];
            front.swap(next);
            if (reached.size() > ball) break;
        }
    }
    uint32_t dist(uint32_t v) const { return seen[v] ? cur[v] : INF; }
};

// Alg. 3's witness search as the paper states it: Dijkstra from s that stops
// once every target is settled or once theta vertices (s included) are
// settled. The heap is ordered by (distance, id), so with weights >= 1 the
// vertices are settled in ascending (dist(s, v), v) order: the settled set is
// the first theta vertices of that order, whatever the targets. A target
// that was not settled gets INF.
struct SettleSearch {
    std::vector<uint32_t> d;
    std::vector<char> done, want;
    std::vector<uint32_t> touched;

    explicit SettleSearch(uint32_t n) : d(n, INF), done(n, 0), want(n, 0) {}

    void run(const std::vector<Adj>& out, uint32_t s, const std::vector<uint32_t>& targets,
             uint64_t theta) {
        for (uint32_t x : touched) {
            d[x] = INF;
            done[x] = 0;
            want[x] = 0;
        }
        touched.clear();
        uint64_t remaining = 0;
        for (uint32_t v : targets)
            if (!want[v]) {
                want[v] = 1;
                touched.push_back(v);
                ++remaining;
            }
        using QE = std::pair<uint32_t, uint32_t>;  // (label, vertex)
        std::priority_queue<QE, std::vector<QE>, std::greater<QE>> pq;
        d[s] = 0;
        touched.push_back(s);
        pq.push({0, s});
        uint64_t settled = 0;
        while (!pq.empty() && remaining > 0 && settled < theta) {
            auto [du, u] = pq.top();
            pq.pop();
            if (done[u]) continue;
            done[u] = 1;
            ++settled;
            if (want[u]) {
                want[u] = 0;
                --remaining;
            }
            for (const auto& [v, wv] : out[u]) {
                uint32_t nd = sat_add(du, wv);
                if (nd < d[v]) {
                    if (d[v] == INF) touched.push_back(v);
                    d[v] = nd;
                    pq.push({nd, v});
                }
            }
        }
    }
    uint32_t dist(uint32_t v) const { return done[v] ? d[v] : INF; }
};

// Per-thread state of one witness search of either kind.
struct Searcher {
    HopSearch hop;
    SettleSearch settle;
    explicit Searcher(uint32_t n) : hop(n), settle(n) {}
};

// How the witness distances of a phase are computed: the hop-limited search
// (optionally with the ball bound), or, with theta > 0, the settled-vertex
// cap of Alg. 3.
struct Witness {
    uint32_t H = 0;
    uint64_t ball = ~uint64_t(0);
    uint64_t level_work = ~uint64_t(0);
    uint64_t theta = 0;
    bool prune = false;  // the recorded distances also decide edge deletions
    bool memo = false;   // the distance map persists across phases and rounds
};

bool keep(uint32_t via, uint32_t dh) { return via != INF && via <= dh; }

uint64_t pair_key(uint32_t a, uint32_t b) { return (uint64_t(a) << 32) | b; }

// Alg. 3: for every source s with an out-neighbour u in `middle`, search from
// s and record the witness distance for every target v in N_out(u), v != s
// (the set V_n of s). With the d_H reading the search keeps labels below the
// heaviest candidate weight of s and, with a finite ball bound, stops after
// the first level at which it holds more than `ball` vertices (the settled-
// vertex cap read per hop level). With theta > 0 it is the capped Dijkstra
// of Alg. 3 itself. Returns the number of sources searched.
uint64_t local_search(const Overlay& g, const std::vector<char>& middle,
                      const std::vector<uint32_t>& middle_list, const Witness& wit,
                      Searcher& hs, std::unordered_map<uint64_t, uint32_t>& dist,
                      std::vector<Searcher>* per_thread = nullptr,
                      uint64_t* searched = nullptr) {
    std::vector<uint32_t> sources;
    for (uint32_t u : middle_list)
        for (const auto& [v1, w1] : g.in[u]) sources.push_back(v1);
    std::sort(sources.begin(), sources.end());
    sources.erase(std::unique(sources.begin(), sources.end()), sources.end());
    // Without memoisation each phase starts from an empty map. With it, the
    // map holds every distance recorded since it was last cleared, and a
    // target whose pair is already there is not searched for again (Alg. 3:
    // (s, v) in dist is skipped); a source with no target left is not
    // searched at all. Every recorded value is the weight of a real walk
    // (or INF), so an old value is still an upper bound on the distance.
    if (!wit.memo) dist.clear();
    // One source's searches and its (pair, distance) records.
    auto search = [&](uint32_t s, Searcher& h, std::vector<std::pair<uint64_t, uint32_t>>& outp) {
        uint32_t bound = 0;  // heaviest candidate weight of s (targets to search)
        uint32_t direct = 0;  // heaviest overlay edge (s, v) to a target v
        std::vector<uint32_t> targets;
        for (const auto& [u, w1] : g.out[s]) {
            if (!middle[u]) continue;
            for (const auto& [v, w2] : g.out[u])
                if (v != s && !(wit.memo && dist.count(pair_key(s, v)))) {
                    bound = std::max(bound, sat_add(w1, w2));
                    targets.push_back(v);
                    auto e = g.out[s].find(v);
                    if (e != g.out[s].end()) direct = std::max(direct, e->second);
                }
        }
        if (targets.empty()) return;  // no candidate from s, or all memoised
        outp.push_back({~uint64_t(0), 0});  // marks one search run
        if (wit.theta) {
            h.settle.run(g.out, s, targets, wit.theta);
            for (uint32_t v : targets) outp.push_back({pair_key(s, v), h.settle.dist(v)});
        } else {
            // Without a ball bound a label at or above the bound cannot
            // change a decision, so the recorded value is exact d_H wherever
            // it is used; with pruning that includes every d_H(s, v) below
            // w(s, v), hence the wider bound. With a ball bound the
            // candidate bound is part of the definition and stays.
            const bool unbounded = wit.ball == ~uint64_t(0);
            h.hop.run(g.out, s, wit.H, unbounded && wit.prune ? std::max(bound, direct) : bound,
                      wit.ball, wit.level_work);
            for (uint32_t v : targets) outp.push_back({pair_key(s, v), h.hop.dist(v)});
        }
    };
#ifdef ORACLE_THREADS
    // Threaded build: the sources are split over host threads, each with its
    // own search state; every record depends on its source alone, so the map
    // is the same as the sequential one.
    std::vector<Searcher> local;
    if (!per_thread) {
        per_thread = &local;
        const unsigned nt = std::max(1u, std::thread::hardware_concurrency());
        for (unsigned t = 0; t < nt; ++t) local.emplace_back(uint32_t(g.out.size()));
    }
    const size_t nt = per_thread->size();
    std::vector<std::vector<std::pair<uint64_t, uint32_t>>> parts(nt);
    std::vector<std::thread> pool;
    for (size_t t = 0; t < nt; ++t)
        pool.emplace_back([&, t] {
            for (size_t i = t; i < sources.size(); i += nt) search(sources[i], (*per_thread)[t], parts[t]);
        });
    for (auto& th : pool) th.join();
    uint64_t runs = 0;
    for (const auto& p : parts)
        for (const auto& [k, v] : p) {
            if (k == ~uint64_t(0)) ++runs;
            else dist[k] = v;
        }
    (void)hs;
#else
    (void)per_thread;
    // The records of a source go in after its search; a record only ever
    // concerns its own source's pairs, so no search of the phase sees
    // another's.
    uint64_t runs = 0;
    std::vector<std::pair<uint64_t, uint32_t>> recs;
    for (uint32_t s : sources) {
        recs.clear();
        search(s, hs, recs);
        for (const auto& [k, v] : recs) {
            if (k == ~uint64_t(0)) ++runs;
            else dist[k] = v;
        }
    }
#endif
    if (searched) *searched += runs;
    return sources.size();
}

// The (s, v) pairs a phase with these middles needs, v in N_out(u) for an
// out-neighbour u of s among the middles, v != s; sorted, no repeats.
std::vector<uint64_t> phase_pairs(const Overlay& g, const std::vector<char>& middle,
                                  const std::vector<uint32_t>& middle_list) {
    std::vector<uint64_t> pairs;
    for (uint32_t u : middle_list)
        for (const auto& [s, w1] : g.in[u])
            for (const auto& [v, w2] : g.out[u])
                if (v != s) pairs.push_back(pair_key(s, v));
    std::sort(pairs.begin(), pairs.end());
    pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
    (void)middle;
    return pairs;
}

struct Shortcut {
    uint32_t round, v1, v2, w, via;
};

struct CH {
    uint32_t n = 0;
    uint32_t H = 0;
    std::vector<uint32_t> level, rank;
    std::vector<int32_t> P;
    std::vector<Shortcut> shortcuts;
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> up;    // E_up: u -> (x, w)
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> down;  // E_down into u: (x, w) for (x,u)
    std::vector<std::array<uint64_t, NSTAT>> stats;
    // Per-vertex bookkeeping behind the features of the learned priority:
    // edge difference at the last rescoring, incident edges removed by
    // contractions so far, hierarchy depth (1 + the largest depth among
    // contracted neighbours, 0 if none), times rescored, degree in the
    // normalised input, and the training label (edge difference at
    // contraction plus depth at contraction).
    std::vector<int32_t> ed_last, depth, label;
    std::vector<uint32_t> cn, rescore, orig_deg;
    // One row per rescoring: round, vertex, then the 12 integer features.
    std::vector<std::array<int64_t, 14>> trace;
    // Overlay edges deleted by the pruning of Alg. 3: (round, s, v, w).
    std::vector<std::array<uint32_t, 4>> pruned;
    uint64_t searches = 0;  // witness searches run (sources with a target to search)
    uint64_t witness_work = 0;  // hop-limited searches: frontier out-edges of the levels run
};

}  // namespace

struct orc_ch {
    CH ch;
};

namespace {

uint64_t select_key(int32_t p, uint32_t u, uint32_t tie_mode, uint32_t seed) {
    uint32_t hi = uint32_t(p) ^ 0x80000000u;  // order-preserving map of int32 onto uint32
    uint32_t lo = tie_mode == 0 ? fmix32(u ^ seed) : u;
    return (uint64_t(hi) << 32) | lo;
}

// Alg. 4 for one vertex, given the round's witness distances.
int32_t score_one(const Overlay& g, uint32_t u,
                  const std::unordered_map<uint64_t, uint32_t>& dist) {
    int64_t p = -int64_t(g.in[u].size() + g.out[u].size());
    for (const auto& [v1, w1] : g.in[u])
        for (const auto& [v2, w2] : g.out[u]) {
            if (v1 == v2) continue;
            auto it = dist.find(pair_key(v1, v2));
            uint32_t dh = it == dist.end() ? INF : it->second;
            if (keep(sat_add(w1, w2), dh)) ++p;
        }
    return int32_t(p);
}

// The 12 integer features of u on the current overlay (learned priority; the
// paper has no counterpart): kept pairs S, |N_in|, |N_out|, distinct
// neighbours, edge difference, removed incident edges, depth, round,
// |N_in|*|N_out|, input degree, times rescored before, mean incident weight
// (integer division; 0 without edges).
std::array<int64_t, 12> features(const Overlay& g, const CH& ch, uint32_t u, int32_t ed, uint32_t r) {
    const int64_t in = g.in[u].size(), out = g.out[u].size();
    int64_t common = 0;
    uint64_t wsum = 0;
    for (const auto& [x, wx] : g.in[u]) {
        if (g.out[u].count(x)) ++common;
        wsum += wx;
    }
    for (const auto& [x, wx] : g.out[u]) wsum += wx;
    std::array<int64_t, 12> f{};
    f[0] = int64_t(ed) + in + out;
    f[1] = in;
    f[2] = out;
    f[3] = in + out - common;
    f[4] = ed;
    f[5] = ch.cn[u];
    f[6] = ch.depth[u];
    f[7] = r;
    f[8] = in * out;
    f[9] = ch.orig_deg[u];
    f[10] = ch.rescore[u];
    f[11] = (in + out) ? int64_t(wsum / uint64_t(in + out)) : 0;
    return f;
}

// Priorities to use instead of the edge difference, keyed by (round, vertex).
using Replay = std::map<std::pair<uint32_t, uint32_t>, int32_t>;

constexpr int32_t P_INELIGIBLE = 2147483646;  // INT32_MAX - 1

// The composite score (Sec. 3.2 names edge difference, vertex degree, hop
// distance and hierarchy depth, without weights): 4 * ED + (|N_in| + |N_out|)
// + 8 * depth, the edge difference weighted highest and depth at twice its
// weight, clamped to +-2^30. Hop counts per overlay edge are not kept, so
// the hop-distance term is left out.
int32_t composite_score(int32_t ed, size_t n_in, size_t n_out, int32_t depth) {
    int64_t p = 4 * int64_t(ed) + int64_t(n_in) + int64_t(n_out) + 8 * int64_t(depth);
    p = std::min<int64_t>(std::max<int64_t>(p, -(int64_t(1) << 30)), int64_t(1) << 30);
    return int32_t(p);
}

void build(CH& ch, uint32_t n, const uint64_t* off, const uint32_t* tgt,
           const uint32_t* w, uint32_t H, uint32_t tie_mode, uint32_t seed,
           bool want_trace = false, const Replay* replay = nullptr,
           uint64_t cmax = ~uint64_t(0), uint64_t ball = ~uint64_t(0), uint64_t theta = 0,
           bool prune = false, uint64_t memo_limit = 0, uint64_t level_work = ~uint64_t(0),
           bool composite = false) {
    Overlay g;
    load(g, n, off, tgt, w);
    ch.ed_last.assign(n, 0);
    ch.depth.assign(n, 0);
    ch.label.assign(n, 0);
    ch.cn.assign(n, 0);
    ch.rescore.assign(n, 0);
    ch.orig_deg.assign(n, 0);
    for (uint32_t u = 0; u < n; ++u) ch.orig_deg[u] = uint32_t(g.in[u].size() + g.out[u].size());
    ch.n = n;
    ch.H = H;
    ch.level.assign(n, INF);
    ch.P.assign(n, 0);
    ch.up.assign(n, {});
    ch.down.assign(n, {});
    Witness wit;
    wit.H = H;
    wit.ball = ball;
    wit.theta = theta;
    wit.prune = prune;
    wit.memo = memo_limit > 0;
    wit.level_work = level_work;
    Searcher hs(n);
    std::unordered_map<uint64_t, uint32_t> dist;
    std::vector<Searcher>* per_thread = nullptr;
#ifdef ORACLE_THREADS
    std::vector<Searcher> hs_pool;
    for (unsigned t = 0, nt = std::max(1u, std::thread::hardware_concurrency()); t < nt; ++t)
        hs_pool.emplace_back(n);
    per_thread = &hs_pool;
#endif

    // the frontier work of the searches so far, collected from every searcher
    auto take_work = [&]() {
        uint64_t w = hs.hop.work;
        hs.hop.work = 0;
        if (per_thread)
            for (auto& t : *per_thread) {
                w += t.hop.work;
                t.hop.work = 0;
            }
        return w;
    };
    uint64_t live = n;
    uint64_t live_edges = 0;
    for (uint32_t u = 0; u < n; ++u) live_edges += g.out[u].size();

    std::vector<uint32_t> A(n);
    for (uint32_t u = 0; u < n; ++u) A[u] = u;
    std::vector<char> inA(n, 0), inF(n, 0), eligible(n, 1);

    for (uint32_t r = 0; live > 0; ++r) {
        std::array<uint64_t, NSTAT> st{};
        st[ST_AFFECTED] = A.size();

        // Eligibility under the candidate bound; only eligible members of A
        // are scored.
        std::vector<uint32_t> Ae;
        for (uint32_t u : A) {
            const uint64_t prod = uint64_t(g.in[u].size()) * uint64_t(g.out[u].size());
            eligible[u] = prod <= cmax;
            if (eligible[u]) Ae.push_back(u);
            else ch.P[u] = P_INELIGIBLE;
        }

        // Step 1: LocalSearch for the affected set.
        for (uint32_t u : Ae) inA[u] = 1;
        st[ST_SCORE_SOURCES] = local_search(g, inA, Ae, wit, hs, dist, per_thread, &ch.searches);
        ch.witness_work += take_work();

        // Pruning (Alg. 3, last step): an overlay edge (s, v) heavier than the
        // witness distance just recorded for (s, v) is deleted. That distance
        // is the weight of a walk s -> v that cannot use (s, v) itself (it
        // weighs less), so every distance survives; deleting all such edges
        // at once is safe too, since each is replaced by a walk of strictly
        // lighter edges. All searches of the step see the overlay as it was
        // before any deletion; Score and the rest of the round see it after.
        if (prune) {
            for (uint64_t key : phase_pairs(g, inA, Ae)) {
                const uint32_t s = uint32_t(key >> 32), v = uint32_t(key);
                const uint32_t d = dist.at(key);
                auto it = g.out[s].find(v);
                if (it == g.out[s].end() || !(it->second > d)) continue;
                ch.pruned.push_back({r, s, v, it->second});
                g.out[s].erase(it);
                g.in[v].erase(s);
                --live_edges;
            }
        }

        // Step 2: Score (edge difference), or the replayed priority; the
        // features are taken from the same overlay.
        for (uint32_t u : Ae) {
            const int32_t ed = score_one(g, u, dist);
            if (want_trace) {
                const auto f = features(g, ch, u, ed, r);
                std::array<int64_t, 14> row{};
                row[0] = r;
                row[1] = u;
                for (int k = 0; k < 12; ++k) row[2 + k] = f[k];
                ch.trace.push_back(row);
            }
            ch.ed_last[u] = ed;
            ++ch.rescore[u];
            if (replay) {
                auto it = replay->find({r, u});
                if (it == replay->end()) throw std::runtime_error("replay has no priority");
                ch.P[u] = it->second;
            } else if (composite) {
                ch.P[u] = composite_score(ed, g.in[u].size(), g.out[u].size(), ch.depth[u]);
            } else {
                ch.P[u] = ed;
            }
        }
        for (uint32_t u : Ae) inA[u] = 0;

        // Step 3: Select (strict local minimum of the key over N(u)).
        std::vector<uint32_t> F;
        for (uint32_t u = 0; u < n; ++u) {
            if (!g.alive[u] || !eligible[u]) continue;
            uint64_t ku = select_key(ch.P[u], u, tie_mode, seed);
            bool minimal = true;
            for (const auto& [v, wv] : g.out[u])
                if (select_key(ch.P[v], v, tie_mode, seed) <= ku) minimal = false;
            for (const auto& [v, wv] : g.in[u])
                if (select_key(ch.P[v], v, tie_mode, seed) <= ku) minimal = false;
            if (minimal) F.push_back(u);
        }
        st[ST_SELECTED] = F.size();

        // No eligible vertex left: the live vertices are the core.
        if (F.empty()) {
            for (uint32_t u = 0; u < n; ++u) {
                if (!g.alive[u]) continue;
                ch.level[u] = r;
                for (const auto& [x, wx] : g.out[u]) ch.up[u].push_back({x, wx});
                for (const auto& [x, wx] : g.in[u]) ch.down[u].push_back({x, wx});
                ch.label[u] = ch.ed_last[u] + ch.depth[u];
            }
            break;
        }

        // Step 4: Contract. Witness distances for the candidates of V_F on
        // the same overlay.
        for (uint32_t u : F) inF[u] = 1;
        st[ST_CONTRACT_SOURCES] = local_search(g, inF, F, wit, hs, dist, per_thread, &ch.searches);
        ch.witness_work += take_work();

        std::map<std::pair<uint32_t, uint32_t>, std::pair<uint32_t, uint32_t>> best;
        for (uint32_t u : F) {
            ch.level[u] = r;
            for (const auto& [x, wx] : g.out[u]) ch.up[u].push_back({x, wx});
            for (const auto& [x, wx] : g.in[u]) ch.down[u].push_back({x, wx});
            for (const auto& [v1, w1] : g.in[u])
                for (const auto& [v2, w2] : g.out[u]) {
                    if (v1 == v2) continue;
                    ++st[ST_CANDIDATES];
                    uint32_t via = sat_add(w1, w2);
                    auto it = dist.find(pair_key(v1, v2));
                    uint32_t dh = it == dist.end() ? INF : it->second;
                    if (!keep(via, dh)) continue;
                    ++st[ST_KEPT];
                    auto key = std::make_pair(v1, v2);
                    auto cand = std::make_pair(via, u);
                    auto b = best.find(key);
                    if (b == best.end() || cand < b->second) best[key] = cand;
                }
        }
        st[ST_MERGED] = best.size();

        // Next affected set: neighbours of V_F in this round's overlay.
        std::vector<uint32_t> nextA;
        for (uint32_t u : F) {
            for (const auto& [x, wx] : g.out[u]) nextA.push_back(x);
            for (const auto& [x, wx] : g.in[u]) nextA.push_back(x);
        }
        std::sort(nextA.begin(), nextA.end());
        nextA.erase(std::unique(nextA.begin(), nextA.end()), nextA.end());

        // Insert merged shortcuts that are new or strictly better.
        for (const auto& [key, val] : best) {
            auto [v1, v2] = key;
            auto [ws, via] = val;
            auto it = g.out[v1].find(v2);
            if (it == g.out[v1].end()) {
                ++live_edges;
            } else if (!(ws < it->second)) {
                continue;
            }
            g.out[v1][v2] = ws;
            g.in[v2][v1] = ws;
            ch.shortcuts.push_back({r, v1, v2, ws, via});
            ++st[ST_INSERTED];
        }

        // Remove V_F and its incident edges; neighbours inherit depth and
        // count the removed edges.
        for (uint32_t u : F) {
            ch.label[u] = ch.ed_last[u] + ch.depth[u];
            for (const auto& [x, wx] : g.out[u]) {
                ++ch.cn[x];
                ch.depth[x] = std::max(ch.depth[x], ch.depth[u] + 1);
            }
            for (const auto& [x, wx] : g.in[u]) {
                ++ch.cn[x];
                ch.depth[x] = std::max(ch.depth[x], ch.depth[u] + 1);
            }
        }
        for (uint32_t u : F) {
            for (const auto& [x, wx] : g.out[u]) g.in[x].erase(u);
            for (const auto& [x, wx] : g.in[u]) g.out[x].erase(u);
            live_edges -= g.out[u].size() + g.in[u].size();
            g.out[u].clear();
            g.in[u].clear();
            g.alive[u] = 0;
            inF[u] = 0;
        }
        live -= F.size();
        st[ST_VO_AFTER] = live;
        st[ST_EO_AFTER] = live_edges;
        ch.stats.push_back(st);
        // Memoised distances are cleared lazily: only at the end of a round
        // that leaves more than memo_limit of them (the paper clears its
        // table once a constant fraction of it is full).
        if (wit.memo && dist.size() > memo_limit) dist.clear();
        A.swap(nextA);
    }

    // Postprocess: rank by (level, score, id).
    std::vector<uint32_t> order(n);
    for (uint32_t u = 0; u < n; ++u) order[u] = u;
    std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        return std::make_tuple(ch.level[a], ch.P[a], a) <
               std::make_tuple(ch.level[b], ch.P[b], b);
    });
    ch.rank.assign(n, 0);
    for (uint32_t i = 0; i < n; ++i) ch.rank[order[i]] = i;
}

// Textbook Dijkstra with a binary heap over an adjacency given as a function.
template <class Nbrs>
void dijkstra(uint32_t n, uint32_t s, Nbrs nbrs, std::vector<uint32_t>& d,
              uint64_t* settled) {
    d.assign(n, INF);
    std::vector<char> done(n, 0);
    using QE = std::pair<uint32_t, uint32_t>;
    std::priority_queue<QE, std::vector<QE>, std::greater<QE>> pq;
    d[s] = 0;
    pq.push({0, s});
    uint64_t cnt = 0;
    while (!pq.empty()) {
        auto [du, u] = pq.top();
        pq.pop();
        if (done[u]) continue;
        done[u] = 1;
        ++cnt;
        nbrs(u, [&](uint32_t v, uint32_t wv) {
            uint32_t nd = sat_add(du, wv);
            if (nd < d[v]) {
                d[v] = nd;
                pq.push({nd, v});
            }
        });
    }
    if (settled) *settled = cnt;
}

// Dijkstra whose labels live in a hash map, so that its cost follows the
// search space rather than n (used by the CH query).
template <class Nbrs>
void dijkstra_sparse(uint32_t s, Nbrs nbrs, std::unordered_map<uint32_t, uint32_t>& d) {
    d.clear();
    std::unordered_map<uint32_t, char> done;
    using QE = std::pair<uint32_t, uint32_t>;
    std::priority_queue<QE, std::vector<QE>, std::greater<QE>> pq;
    d[s] = 0;
    pq.push({0, s});
    while (!pq.empty()) {
        auto [du, u] = pq.top();
        pq.pop();
        if (done.count(u)) continue;
        done[u] = 1;
        nbrs(u, [&](uint32_t v, uint32_t wv) {
            uint32_t nd = sat_add(du, wv);
            if (nd == INF) return;  // not reachable within the uint32 range
            auto it = d.find(v);
            if (it == d.end() || nd < it->second) {
                d[v] = nd;
                pq.push({nd, v});
            }
        });
    }
}

// Sec. 5: forward upward search from s, backward upward search from t, both
// run to exhaustion; the answer is the least d_s(v) + d_t(v) over the
// vertices both reach. `settled` receives the two search-space sizes summed
// (vertices reached at a distance below INF, counted once per direction).
uint32_t query(const CH& ch, uint32_t s, uint32_t t, uint64_t* settled) {
    std::unordered_map<uint32_t, uint32_t> ds, dt;
    dijkstra_sparse(s, [&](uint32_t u, auto f) {
        for (const auto& [x, wx] : ch.up[u]) f(x, wx);
    }, ds);
    dijkstra_sparse(t, [&](uint32_t u, auto f) {
        for (const auto& [x, wx] : ch.down[u]) f(x, wx);
    }, dt);
    uint32_t mu = INF;
    for (const auto& [v, dv] : ds) {
        auto it = dt.find(v);
        if (it != dt.end()) mu = std::min(mu, sat_add(dv, it->second));
    }
    if (settled) *settled = ds.size() + dt.size();
    return mu;
}

// One-to-all distances from s (the PHAST scheme the paper cites for SSSP on
// a CH, Sec. 5): an upward search from s over E_up, then one sweep over all
// vertices in descending rank, d(u) = min(d(u), d(x) + w) for every downward
// edge (x, u). Such an edge comes from a vertex contracted in a later round
// (u's in-neighbours at its contraction are outside V_F and outlive it), so
// x has the higher rank and its value is final when u is reached. Core
// vertices need no sweep: their E_up holds the core's edges, so the upward
// search is already a full search inside the core; the sweep over their
// core-core downward edges only re-offers walks and changes nothing.
void one_to_all(const CH& ch, uint32_t s, uint32_t* d) {
    std::unordered_map<uint32_t, uint32_t> ds;
    dijkstra_sparse(s, [&](uint32_t u, auto f) {
        for (const auto& [x, wx] : ch.up[u]) f(x, wx);
    }, ds);
    for (uint32_t v = 0; v < ch.n; ++v) d[v] = INF;
    for (const auto& [v, dv] : ds) d[v] = dv;
    std::vector<uint32_t> by_rank(ch.n);
    for (uint32_t u = 0; u < ch.n; ++u) by_rank[ch.rank[u]] = u;
    for (uint32_t i = ch.n; i-- > 0;) {
        const uint32_t u = by_rank[i];
        for (const auto& [x, wx] : ch.down[u]) d[u] = std::min(d[u], sat_add(d[x], wx));
    }
}

}  // namespace

extern "C" {

int orc_build(uint32_t n, uint64_t m, const uint64_t* off, const uint32_t* tgt,
              const uint32_t* w, uint32_t H, uint32_t tie_mode, uint32_t tie_seed,
              orc_ch** out) {
    if (!out || !validate(n, m, off, tgt, w) || tie_mode > 1) return ORC_EINVAL;
    orc_ch* h = new orc_ch();
    build(h->ch, n, off, tgt, w, H, tie_mode, tie_seed);
    *out = h;
    return ORC_OK;
}

// Build with the learned-priority bookkeeping: `want_trace` records the
// features of every rescoring; a non-empty replay (round, vertex, priority)
// list replaces the edge difference by the given priorities (it must cover
// every rescoring the run makes, else ORC_EINVAL).
int orc_build2(uint32_t n, uint64_t m, const uint64_t* off, const uint32_t* tgt,
               const uint32_t* w, uint32_t H, uint32_t tie_mode, uint32_t tie_seed,
               int want_trace, uint64_t nreplay, const uint32_t* rp_round, const uint32_t* rp_u,
               const int32_t* rp_p, uint64_t cmax, uint64_t ball, uint64_t theta, int prune,
               uint64_t memo_limit, uint64_t level_work, int composite, orc_ch** out) {
    // the settled-vertex cap replaces the hop-limited search, ball bound included
    if (!out || !validate(n, m, off, tgt, w) || tie_mode > 1 || (theta && ball != ~uint64_t(0)))
        return ORC_EINVAL;
    Replay rp;
    for (uint64_t i = 0; i < nreplay; ++i) rp[{rp_round[i], rp_u[i]}] = rp_p[i];
    orc_ch* h = new orc_ch();
    try {
        build(h->ch, n, off, tgt, w, H, tie_mode, tie_seed, want_trace != 0,
              nreplay ? &rp : nullptr, cmax, ball, theta, prune != 0, memo_limit, level_work,
              composite != 0);
    } catch (const std::exception&) {
        delete h;
        return ORC_EINVAL;
    }
    *out = h;
    return ORC_OK;
}

uint64_t orc_num_pruned(const orc_ch* h) { return h->ch.pruned.size(); }
uint64_t orc_searches(const orc_ch* h) { return h->ch.searches; }
uint64_t orc_witness_work(const orc_ch* h) { return h->ch.witness_work; }
void orc_get_pruned(const orc_ch* h, uint32_t* out4) {
    size_t i = 0;
    for (const auto& row : h->ch.pruned)
        for (int k = 0; k < 4; ++k) out4[i++] = row[k];
}

// One-to-all distances for k sources, row i of out (n entries) for src[i].
int orc_one_to_all(const orc_ch* h, uint64_t k, const uint32_t* src, uint32_t* out) {
    for (uint64_t i = 0; i < k; ++i)
        if (src[i] >= h->ch.n) return ORC_EINVAL;
    for (uint64_t i = 0; i < k; ++i) one_to_all(h->ch, src[i], out + i * uint64_t(h->ch.n));
    return ORC_OK;
}

uint64_t orc_num_trace(const orc_ch* h) { return h->ch.trace.size(); }
void orc_get_trace(const orc_ch* h, int64_t* out14) {
    size_t i = 0;
    for (const auto& row : h->ch.trace)
        for (int k = 0; k < 14; ++k) out14[i++] = row[k];
}
void orc_get_labels(const orc_ch* h, int32_t* out) {
    std::memcpy(out, h->ch.label.data(), sizeof(int32_t) * h->ch.n);
}

void orc_free(orc_ch* h) { delete h; }

uint32_t orc_rounds(const orc_ch* h) { return uint32_t(h->ch.stats.size()); }
uint32_t orc_nstat(void) { return NSTAT; }

void orc_get_stats(const orc_ch* h, uint64_t* out) {
    for (size_t r = 0; r < h->ch.stats.size(); ++r)
        for (int f = 0; f < NSTAT; ++f) out[r * NSTAT + f] = h->ch.stats[r][f];
}

void orc_get_level(const orc_ch* h, uint32_t* out) {
    std::memcpy(out, h->ch.level.data(), sizeof(uint32_t) * h->ch.n);
}
void orc_get_priority(const orc_ch* h, int32_t* out) {
    std::memcpy(out, h->ch.P.data(), sizeof(int32_t) * h->ch.n);
}
void orc_get_rank(const orc_ch* h, uint32_t* out) {
    std::memcpy(out, h->ch.rank.data(), sizeof(uint32_t) * h->ch.n);
}

uint64_t orc_num_shortcuts(const orc_ch* h) { return h->ch.shortcuts.size(); }
void orc_get_shortcuts(const orc_ch* h, uint32_t* out5) {
    size_t i = 0;
    for (const auto& s : h->ch.shortcuts) {
        out5[i++] = s.round;
        out5[i++] = s.v1;
        out5[i++] = s.v2;
        out5[i++] = s.w;
        out5[i++] = s.via;
    }
}

// Upward edges (u, x, w) and downward edges (x, u, w), each as triples.
uint64_t orc_num_up(const orc_ch* h) {
    uint64_t c = 0;
    for (const auto& l : h->ch.up) c += l.size();
    return c;
}
uint64_t orc_num_down(const orc_ch* h) {
    uint64_t c = 0;
    for (const auto& l : h->ch.down) c += l.size();
    return c;
}
void orc_get_up(const orc_ch* h, uint32_t* out3) {
    size_t i = 0;
    for (uint32_t u = 0; u < h->ch.n; ++u)
        for (const auto& [x, wx] : h->ch.up[u]) {
            out3[i++] = u;
            out3[i++] = x;
            out3[i++] = wx;
        }
}
void orc_get_down(const orc_ch* h, uint32_t* out3) {
    size_t i = 0;
    for (uint32_t u = 0; u < h->ch.n; ++u)
        for (const auto& [x, wx] : h->ch.down[u]) {
            out3[i++] = x;
            out3[i++] = u;
            out3[i++] = wx;
        }
}

void orc_query_batch(const orc_ch* h, uint64_t k, const uint32_t* s, const uint32_t* t,
                     uint32_t* out, uint64_t* settled) {
#ifdef ORACLE_THREADS
    // Threaded build: pairs are split over host threads; each answer depends
    // on its pair alone, so the output is the sequential one.
    const uint64_t nt = std::max(1u, std::thread::hardware_concurrency());
    std::vector<std::thread> pool;
    for (uint64_t th = 0; th < nt; ++th)
        pool.emplace_back([&, th] {
            for (uint64_t i = th; i < k; i += nt)
                out[i] = query(h->ch, s[i], t[i], settled ? settled + i : nullptr);
        });
    for (auto& x : pool) x.join();
#else
    for (uint64_t i = 0; i < k; ++i)
        out[i] = query(h->ch, s[i], t[i], settled ? settled + i : nullptr);
#endif
}

// Scores of every vertex of the input graph as round 0 computes them.
int orc_round0_scores(uint32_t n, uint64_t m, const uint64_t* off, const uint32_t* tgt,
                      const uint32_t* w, uint32_t H, uint64_t ball, int32_t* P) {
    if (!validate(n, m, off, tgt, w)) return ORC_EINVAL;
    Overlay g;
    load(g, n, off, tgt, w);
    std::vector<uint32_t> A(n);
    std::vector<char> inA(n, 1);
    for (uint32_t u = 0; u < n; ++u) A[u] = u;
    Searcher hs(n);
    Witness wit;
    wit.H = H;
    wit.ball = ball;
    std::unordered_map<uint64_t, uint32_t> dist;
    local_search(g, inA, A, wit, hs, dist);
    for (uint32_t u = 0; u < n; ++u) P[u] = score_one(g, u, dist);
    return ORC_OK;
}

// Normalised input (self-loops dropped, parallel edges merged by min) as an
// out-CSR sorted by head. Call with off_out == NULL to get the edge count.
int orc_normalize(uint32_t n, uint64_t m, const uint64_t* off, const uint32_t* tgt,
                  const uint32_t* w, uint64_t* m_out, uint64_t* off_out,
                  uint32_t* tgt_out, uint32_t* w_out) {
    if (!validate(n, m, off, tgt, w)) return ORC_EINVAL;
    Overlay g;
    load(g, n, off, tgt, w);
    uint64_t c = 0;
    for (uint32_t u = 0; u < n; ++u) c += g.out[u].size();
    *m_out = c;
    if (!off_out) return ORC_OK;
    uint64_t e = 0;
    for (uint32_t u = 0; u < n; ++u) {
        off_out[u] = e;
        for (const auto& [v, wv] : g.out[u]) {
            tgt_out[e] = v;
            w_out[e] = wv;
            ++e;
        }
    }
    off_out[n] = e;
    return ORC_OK;
}

// d_H from `src` on the normalised input graph, for every vertex.
int orc_hop_limited(uint32_t n, uint64_t m, const uint64_t* off, const uint32_t* tgt,
                    const uint32_t* w, uint32_t H, uint32_t src, uint32_t* dist) {
    if (!validate(n, m, off, tgt, w) || src >= n) return ORC_EINVAL;
    Overlay g;
    load(g, n, off, tgt, w);
    HopSearch hs(n);
    hs.run(g.out, src, H);
    for (uint32_t v = 0; v < n; ++v) dist[v] = hs.dist(v);
    return ORC_OK;
}

// Exact single-source distances on the normalised input graph (Dijkstra).
int orc_dijkstra(uint32_t n, uint64_t m, const uint64_t* off, const uint32_t* tgt,
                 const uint32_t* w, uint32_t src, uint32_t* dist) {
    if (!validate(n, m, off, tgt, w) || src >= n) return ORC_EINVAL;
    Overlay g;
    load(g, n, off, tgt, w);
    std::vector<uint32_t> d;
    dijkstra(n, src, [&](uint32_t u, auto f) {
        for (const auto& [x, wx] : g.out[u]) f(x, wx);
    }, d, nullptr);
    std::memcpy(dist, d.data(), sizeof(uint32_t) * n);
    return ORC_OK;
}

// Exact s-t distances for a batch of pairs on the input graph (one Dijkstra
// per distinct source, pairs grouped by source).
int orc_dijkstra_pairs(uint32_t n, uint64_t m, const uint64_t* off, const uint32_t* tgt,
                       const uint32_t* w, uint64_t k, const uint32_t* s,
                       const uint32_t* t, uint32_t* out) {
    if (!validate(n, m, off, tgt, w)) return ORC_EINVAL;
    Overlay g;
    load(g, n, off, tgt, w);
    std::vector<uint64_t> idx(k);
    for (uint64_t i = 0; i < k; ++i) {
        if (s[i] >= n || t[i] >= n) return ORC_EINVAL;
        idx[i] = i;
    }
    std::sort(idx.begin(), idx.end(), [&](uint64_t a, uint64_t b) { return s[a] < s[b]; });
    std::vector<uint32_t> d;
    uint32_t cur = INF;
    for (uint64_t i : idx) {
        if (s[i] != cur) {
            cur = s[i];
            dijkstra(n, cur, [&](uint32_t u, auto f) {
                for (const auto& [x, wx] : g.out[u]) f(x, wx);
            }, d, nullptr);
        }
        out[i] = d[t[i]];
    }
    return ORC_OK;
}

}  // extern "C"
