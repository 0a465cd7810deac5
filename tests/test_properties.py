"""Property tests over random small digraphs (no GPU): for any hop limit,
tie-break, candidate bound, witness ball bound, level-work bound, settled-
vertex cap, pruning and memoisation setting, every CH query and every
one-to-all row equals the true distance, and every round re-derives from the
definitions."""
import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I
from tests.graphs import all_pairs_truth
from tests.test_trace_pins import _rederive

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")


@st.composite
def _case(draw):
    n = draw(st.integers(1, 40))
    m = draw(st.integers(0, 4 * n))
    seed = draw(st.integers(0, 2**31 - 1))
    wmax = draw(st.sampled_from([1, 3, 30, 1000]))
    H = draw(st.integers(0, 5))
    tie = draw(st.sampled_from([O.TIE_HASHED, O.TIE_ID]))
    cmax = draw(st.sampled_from([O.CMAX_ALL, 0, 1, 4, 16]))
    ball = draw(st.sampled_from([None, 1, 2, 5]))
    theta = 0 if ball is not None else draw(st.sampled_from([0, 0, 1, 2, 4, 9]))
    prune = draw(st.booleans())
    memo = draw(st.sampled_from([0, 0, 5, 1 << 40]))
    level_work = None if theta else draw(st.sampled_from([None, None, 0, 3, 12]))
    return (I.random_digraph(n, m, 1, wmax, seed=seed), H, tie, seed & 0xFFFF, cmax, ball, theta,
            prune, memo, level_work)


@hyp.settings(max_examples=400, deadline=None, derandomize=True)
@hyp.given(_case())
def test_random_digraphs(case):
    g, H, tie, seed, cmax, ball, theta, prune, memo, level_work = case
    och = _rederive(g, H, tie, seed=seed, cmax=cmax, ball=ball, theta=theta, prune=prune,
                    memo=memo, level_work=level_work)
    s, t = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    d = och.query(s.ravel().astype(np.uint32), t.ravel().astype(np.uint32))
    truth = all_pairs_truth(g)
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), truth)
    assert np.array_equal(och.one_to_all(np.arange(g.n)).astype(np.uint64), truth)
