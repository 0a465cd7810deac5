"""Every trace row of every round, recomputed from definitions (no GPU).

Each round's overlay is rebuilt from the exported hierarchy alone: the
normalised input, with the logged shortcuts of earlier rounds applied (a
logged shortcut is an insertion or a strictly lighter replacement), minus the
vertices contracted in earlier rounds. The 12 features of each rescoring
then follow from their definitions on that overlay: the score uses the
plain hop-limited distance (oracle.hop_limited, pinned in test_oracle.py),
the contracted-neighbour count and depth use the CH edges recorded at
earlier contractions. This pins the round loop's bookkeeping, its overlay
updates and its scores in every round, independently of the loop itself."""
from collections import defaultdict

import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I
from tests.graphs import INF, small_families


def _graph_from_pairs(n, pairs):
    if pairs:
        src, dst, w = (np.array(x, dtype=np.int64) for x in zip(*[(a, b, c) for (a, b), c in pairs.items()]))
    else:
        src = dst = w = np.zeros(0, np.int64)
    return I.csr_from_edges(n, src, dst, w)


def _check(g, H, cmax=O.CMAX_ALL):
    och = O.build_ch(g, H, trace=True, cmax=cmax)
    n = g.n
    off, tgt, w = O.normalize(g)
    base = {}
    for a in range(n):
        for e in range(int(off[a]), int(off[a + 1])):
            base[(a, int(tgt[e]))] = int(w[e])
    orig_deg = np.zeros(n, np.int64)
    for (a, b) in base:
        orig_deg[a] += 1
        orig_deg[b] += 1
    level = och.level.astype(np.int64)
    by_round = defaultdict(list)
    for r, v1, v2, ws, via in och.shortcuts.tolist():
        by_round[r].append((v1, v2, ws))
    # CH edges recorded at each contraction: (contracted u, neighbour x)
    ch_nb = defaultdict(list)  # u -> neighbours x (one entry per edge)
    for u, x, _ in och.up.tolist():
        ch_nb[u].append(x)
    for x, u, _ in och.down.tolist():
        ch_nb[u].append(x)
    # depth: 1 + the deepest CH neighbour contracted earlier (0 if none)
    nb_before = defaultdict(list)  # x -> contracted neighbours u (one per CH edge)
    for u, xs in ch_nb.items():
        for x in xs:
            nb_before[x].append(u)

    def depth_of(x, r):
        ds = [depth_at_c(u) + 1 for u in nb_before[x] if level[u] < r]
        return max(ds, default=0)

    memo = {}

    def depth_at_c(u):
        if u not in memo:
            memo[u] = depth_of(u, level[u])
        return memo[u]

    edges = dict(base)
    rows = och.trace.tolist()
    seen = defaultdict(int)
    ri = 0
    for r in range(och.rounds):
        # overlay of round r: shortcuts of rounds < r applied, dead vertices removed
        for v1, v2, ws in by_round.get(r - 1, []):
            edges[(v1, v2)] = ws
        live = {k: v for k, v in edges.items() if level[k[0]] >= r and level[k[1]] >= r}
        gr = _graph_from_pairs(n, live)
        out, inn = defaultdict(dict), defaultdict(dict)
        for (a, b), c in live.items():
            out[a][b] = c
            inn[b][a] = c
        dh = {}
        while ri < len(rows) and rows[ri][0] == r:
            _, x, *f = rows[ri]
            ri += 1
            i, o = len(inn[x]), len(out[x])
            S = 0
            for v1, w1 in inn[x].items():
                if v1 not in dh:
                    dh[v1] = O.hop_limited(gr, H, v1)
                for v2, w2 in out[x].items():
                    if v1 != v2 and w1 + w2 < INF and w1 + w2 <= dh[v1][v2]:
                        S += 1
            ed = S - i - o
            wsum = sum(inn[x].values()) + sum(out[x].values())
            cn = sum(1 for u in nb_before[x] if level[u] < r)
            want = [S, i, o, len(set(inn[x]) | set(out[x])), ed, cn, depth_of(x, r), r, i * o,
                    int(orig_deg[x]), seen[x], wsum // (i + o) if i + o else 0]
            assert f == want, (r, x, f, want)
            seen[x] += 1
    assert ri == len(rows)
    # the score at contraction is the last rescoring's edge difference
    last_ed = {}
    for r, x, *f in rows:
        last_ed[x] = f[4]
    contracted = level < och.rounds
    for x in np.flatnonzero(contracted).tolist():
        assert och.priority[x] == last_ed[x]
        assert och.labels[x] == last_ed[x] + depth_at_c(x)


@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph0", "digraph4", "sparse3", "grid8", "geo150",
                                             "rmat8", "chain30", "star9")],
                         ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("H", [2, 5])
def test_trace_rows_recomputed_for_every_round(name, g, H):
    _check(g, H)


def test_trace_rows_recomputed_with_a_core():
    _check(I.random_digraph(70, 300, 1, 20, seed=41), 5, cmax=9)


# ---------------------------------------------------------------------------
# Every round re-derived: affected set, eligibility, selection, candidates,
# witness decisions, merge, insertion and the round's counters
# ---------------------------------------------------------------------------

P_INELIGIBLE = 2**31 - 2


def _fmix32(h):
    # MurmurHash3 32-bit finaliser (Appleby), as published
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    h ^= h >> 16
    return h


def _settled_distances(gr, s, theta):
    """Distances from s that a Dijkstra capped at theta settled vertices
    reports: the true distance for the first theta vertices in (distance,
    id) order, INF for the rest (scipy's Dijkstra, then a sort)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import dijkstra

    src, dst, w = gr.edges()
    mat = sp.csr_matrix((w.astype(np.float64), (src, dst)), shape=(gr.n, gr.n))
    dist = dijkstra(mat, directed=True, indices=s)
    reach = np.flatnonzero(np.isfinite(dist))
    order = reach[np.lexsort((reach, dist[reach]))]
    out = np.full(gr.n, INF, np.uint64)
    first = order[:theta]
    out[first] = dist[first].astype(np.uint64)
    return out


def _ball_labels(gr, s, H, bound, ball, level_work=None):
    """Labels below `bound` of a hop-synchronous search from s: those of
    level H, or with a ball bound those of the first level at which more than
    `ball` vertices hold one, or with a level-work bound those of the last
    level before one whose frontier (the vertices whose label dropped in the
    level before) has more than `level_work` out-edges; INF elsewhere."""
    return _ball_search(gr, s, H, bound, ball, level_work)[0]


def _ball_search(gr, s, H, bound, ball, level_work=None):
    """(_ball_labels's labels, the frontier out-edges of the levels run)."""
    outdeg = np.diff(gr.offsets.astype(np.int64))
    lab = np.where(np.arange(gr.n) == s, 0, INF).astype(np.int64)
    front = np.array([s])
    work = 0
    for h in range(1, H + 1):
        wk = int(outdeg[front].sum())
        if level_work is not None and h >= 2 and wk > level_work:
            break
        work += wk
        dist_h = O.hop_limited(gr, h, s).astype(np.int64)
        new = np.where(dist_h < bound, dist_h, INF)
        front = np.flatnonzero(new < lab)
        lab = new
        if ball is not None and int((lab != INF).sum()) > ball:
            break
    return lab, work


def _rederive(g, H, tie, seed=0, cmax=O.CMAX_ALL, ball=None, theta=0, prune=False, memo=0,
              level_work=None):
    och = O.build_ch(g, H, tie, tie_seed=seed, cmax=cmax, ball=O.CMAX_ALL if ball is None else ball,
                     theta=theta, prune=prune, memo=memo,
                     level_work=O.CMAX_ALL if level_work is None else level_work)
    memo_d = {}
    searches = [0]
    work = [0]
    n = g.n
    off, tgt, w = O.normalize(g)
    edges = {}
    for a in range(n):
        for e in range(int(off[a]), int(off[a + 1])):
            edges[(a, int(tgt[e]))] = int(w[e])
    log = defaultdict(set)
    for r, v1, v2, ws, via in och.shortcuts.tolist():
        log[r].add((v1, v2, ws, via))
    level = och.level.astype(np.int64)
    alive = np.ones(n, bool)
    P = np.zeros(n, np.int64)
    eligible = np.ones(n, bool)
    A = set(range(n))
    pruned = []

    def key(u):
        lo = u if tie == O.TIE_ID else _fmix32(u ^ seed)
        return ((int(P[u]) & 0xFFFFFFFF) ^ 0x80000000) << 32 | lo

    def overlay():
        live = {k: v for k, v in edges.items() if alive[k[0]] and alive[k[1]]}
        out, inn = defaultdict(dict), defaultdict(dict)
        for (a, b), c in live.items():
            out[a][b] = c
            inn[b][a] = c
        return live, out, inn, _graph_from_pairs(n, live), {}

    r = 0
    while alive.any():
        live, out, inn, gr, dh = overlay()

        def d(v1, v2, middles):
            # witness distance of the phase whose contracted middles are
            # `middles`: d_H; or with a ball bound the distances of the first
            # level at which more than `ball` vertices hold a label below the
            # source's heaviest candidate weight; or with a settled-vertex
            # cap the capped Dijkstra's
            if theta:
                if v1 not in dh:
                    dh[v1] = _settled_distances(gr, v1, theta)
                return int(dh[v1][v2])
            if ball is None and level_work is None:
                if v1 not in dh:
                    dh[v1] = O.hop_limited(gr, H, v1)
                return int(dh[v1][v2])
            cands = [(c1 + c2, x) for u, c1 in out[v1].items() if u in middles
                     for x, c2 in out[u].items() if x != v1]
            bound = max([c for c, _ in cands], default=0)
            if prune and ball is None:
                bound = max([bound] + [live[(v1, x)] for _, x in cands if (v1, x) in live])
            keyd = (v1, bound)
            if keyd not in dh:
                dh[keyd] = _ball_labels(gr, v1, H, bound, ball, level_work)
            return int(dh[keyd][v2])

        def fill(middles):
            # the searches of one phase: a source with a candidate target
            # searches once; with memoisation only for targets whose pair has
            # no recorded distance, and the value recorded is the label its
            # search held (labels at or above the heaviest weight the search
            # must decide are dropped), INF if none
            for s in sorted(set().union(*(set(inn[u]) for u in middles))):
                cands = [(c1 + c2, v) for u, c1 in out[s].items() if u in middles
                         for v, c2 in out[u].items() if v != s and not (memo and (s, v) in memo_d)]
                if not cands:
                    continue
                searches[0] += 1
                new = {v for _, v in cands}
                if theta:
                    lab = _settled_distances(gr, s, theta)
                else:
                    bound = max(c for c, _ in cands)
                    if prune and ball is None:
                        bound = max([bound] + [live[(s, v)] for v in new if (s, v) in live])
                    lab, wk = _ball_search(gr, s, H, bound, ball, level_work)
                    work[0] += wk
                if memo:
                    for v in new:
                        memo_d[(s, v)] = int(lab[v])

        def dm(v1, v2, middles):
            return memo_d[(v1, v2)] if memo else d(v1, v2, middles)

        # rescoring of the affected set (Alg. 3, 4) under the candidate bound:
        # every witness distance of the step on the overlay of the round start
        for u in A:
            eligible[u] = len(inn[u]) * len(out[u]) <= cmax
        middles = {u for u in A if eligible[u]}
        score_sources = set().union(*(set(inn[u]) for u in middles))
        fill(middles)
        score_d = {(v1, v2): dm(v1, v2, middles) for u in middles
                   for v1 in inn[u] for v2 in out[u] if v1 != v2}
        if prune:
            # Alg. 3's pruning: overlay edges heavier than their pair's
            # witness distance leave before Score
            for (s, v), dv in sorted(score_d.items()):
                if (s, v) in live and live[(s, v)] > dv:
                    pruned.append((r, s, v, live[(s, v)]))
                    del edges[(s, v)]
            live, out, inn, gr, dh = overlay()
        for u in A:
            if not eligible[u]:
                P[u] = P_INELIGIBLE
                continue
            S = sum(1 for v1 in inn[u] for v2 in out[u]
                    if v1 != v2 and inn[u][v1] + out[u][v2] < INF
                    and inn[u][v1] + out[u][v2] <= score_d[(v1, v2)])
            P[u] = S - len(inn[u]) - len(out[u])
        # selection (Alg. 5): strict local minima of the key over N(u)
        F = [u for u in np.flatnonzero(alive).tolist() if eligible[u]
             and all(key(u) < key(v) for v in set(inn[u]) | set(out[u]))]
        if not F:
            core = np.flatnonzero(alive)
            assert (level[core] == r).all() and och.rounds == r
            break
        assert sorted(F) == np.flatnonzero(level == r).tolist(), r
        # Alg. 5's invariants: V_F is independent, and the live eligible
        # vertex of least key is always in it (so every round makes progress)
        assert not any(v in set(F) for u in F for v in set(inn[u]) | set(out[u]))
        assert min((u for u in np.flatnonzero(alive).tolist() if eligible[u]), key=key) in F
        # contraction (Alg. 6): candidates, witness test on the overlay as it
        # stands now, merge, insertion
        middles = set(F)
        fill(middles)
        best, cand, keep_n = {}, 0, 0
        for u in F:
            for v1 in inn[u]:
                for v2 in out[u]:
                    if v1 == v2:
                        continue
                    cand += 1
                    via = inn[u][v1] + out[u][v2]
                    if via < INF and via <= dm(v1, v2, middles):
                        keep_n += 1
                        best[(v1, v2)] = min(best.get((v1, v2), (INF + 1, n)), (via, u))
        inserted = {(v1, v2, wv, via) for (v1, v2), (wv, via) in best.items()
                    if (v1, v2) not in live or wv < live[(v1, v2)]}
        assert inserted == log[r], r
        contract_sources = set().union(*(set(inn[u]) for u in F))
        nextA = set().union(*(set(inn[u]) | set(out[u]) for u in F))
        for v1, v2, wv, _ in inserted:
            edges[(v1, v2)] = wv
        for u in F:
            alive[u] = False
        live_after = sum(1 for (a, b) in edges if alive[a] and alive[b])
        row = [len(A), len(score_sources), len(F), len(contract_sources), cand, keep_n, len(best),
               len(inserted), int(alive.sum()), live_after]
        assert och.stats[r].tolist() == row, (r, och.stats[r].tolist(), row)
        A = {x for x in nextA if alive[x]}
        if memo and len(memo_d) > memo:
            memo_d.clear()
        r += 1
    assert och.rounds == r
    assert och.pruned.tolist() == [list(p) for p in pruned]
    assert och.searches == searches[0]
    assert och.witness_work == work[0]
    return och


@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph1", "digraph5", "sparse0", "sparse4", "grid8",
                                             "geo150", "rmat8", "chain30d", "star9", "complete6")],
                         ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("H,tie", [(5, O.TIE_HASHED), (2, O.TIE_ID), (0, O.TIE_HASHED)])
def test_every_round_rederived(name, g, H, tie):
    _rederive(g, H, tie, seed=23)


@pytest.mark.parametrize("seed", range(3))
def test_every_round_rederived_with_a_core(seed):
    _rederive(I.random_digraph(70, 300, 1, 20, seed=50 + seed), 5, O.TIE_HASHED, cmax=9)


@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph2", "sparse1", "grid8", "geo150", "rmat8")],
                         ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("ball", [1, 3, 8])
def test_every_round_rederived_with_a_ball_bound(name, g, ball):
    _rederive(g, 4, O.TIE_HASHED, seed=5, ball=ball)


@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph0", "digraph4", "sparse2", "grid8", "grid10u",
                                             "geo150", "rmat8", "chain30", "star9", "complete6")],
                         ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("theta", [1, 2, 5, 20, 10**6])
def test_every_round_rederived_with_a_settled_cap(name, g, theta):
    # Alg. 3's capped Dijkstra, pinned through scipy's Dijkstra and a sort
    _rederive(g, 5, O.TIE_HASHED, seed=7, theta=theta)


@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph1", "digraph3", "sparse3", "grid8", "grid10u",
                                             "geo150", "geo120s", "rmat8", "chain30d")],
                         ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("H,theta,ball", [(1, 0, None), (2, 0, None), (5, 0, None), (4, 0, 3),
                                          (5, 4, None), (5, 30, None)])
def test_every_round_rederived_with_pruning(name, g, H, theta, ball):
    och = _rederive(g, H, O.TIE_HASHED, seed=9, ball=ball, theta=theta, prune=True)
    if name.startswith("geo") and H >= 2 and not theta:
        # hop-limited witnesses leave heavier edges behind that later rounds
        # find shorter walks for
        assert och.pruned.shape[0] > 0


def test_every_round_rederived_with_pruning_and_a_core():
    for seed in range(3):
        _rederive(I.random_digraph(70, 300, 1, 20, seed=60 + seed), 2, O.TIE_HASHED, cmax=9,
                  prune=True)
        _rederive(I.random_digraph(70, 300, 1, 20, seed=63 + seed), 5, O.TIE_ID, cmax=9, theta=6,
                  prune=True)


@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph0", "digraph5", "sparse1", "sparse4", "grid8",
                                             "grid10u", "geo150", "geo120s", "rmat8", "chain30",
                                             "star9", "complete6")],
                         ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("H,theta,ball,prune,memo", [
    (5, 0, None, False, 1 << 40), (2, 0, None, False, 1 << 40), (5, 0, None, True, 1 << 40),
    (5, 0, None, False, 40), (3, 0, 3, False, 1 << 40), (3, 0, 3, True, 25),
    (5, 3, None, False, 1 << 40), (5, 6, None, True, 30), (0, 0, None, True, 1 << 40)])
def test_every_round_rederived_with_memoisation(name, g, H, theta, ball, prune, memo):
    _rederive(g, H, O.TIE_HASHED, seed=11, ball=ball, theta=theta, prune=prune, memo=memo)


def test_every_round_rederived_with_memoisation_and_a_core():
    for seed in range(3):
        _rederive(I.random_digraph(70, 300, 1, 20, seed=70 + seed), 5, O.TIE_HASHED, cmax=9,
                  prune=True, memo=1 << 40)
        _rederive(I.random_digraph(70, 300, 1, 20, seed=73 + seed), 3, O.TIE_ID, cmax=9, memo=50)


@pytest.mark.parametrize("name,g", [(n, g) for n, g in small_families()
                                    if n in ("digraph0", "digraph2", "sparse3", "grid8", "geo150",
                                             "rmat8", "star9", "complete6")],
                         ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("H,lw,ball,prune,memo", [
    (3, 0, None, False, 0), (3, 4, None, False, 0), (5, 12, None, False, 0), (5, 40, None, True, 0),
    (4, 12, 5, False, 0), (4, 8, None, False, 1 << 40), (5, 20, 6, True, 40)])
def test_every_round_rederived_with_a_level_work_bound(name, g, H, lw, ball, prune, memo):
    _rederive(g, H, O.TIE_HASHED, seed=13, ball=ball, prune=prune, memo=memo, level_work=lw)
