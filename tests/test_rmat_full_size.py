"""The RMAT stress configuration at its full size (2^21 vertices, 2^25 edge
samples) against the threaded oracle at the same settings: the whole
hierarchy element by element, and sampled answers against Dijkstra on the
input graph (Sec. 3's partial hierarchy under a candidate bound; Sec. 5's
queries through the core).

The oracle needs about four minutes on 16 host cores, so the test runs only
when CH_FULL_SIZE=1 is set.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I
from tests.test_gpu_parity import assert_same_hierarchy

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(os.environ.get("CH_FULL_SIZE") != "1",
                       reason="full-size oracle run (minutes); set CH_FULL_SIZE=1"),
]

torch = pytest.importorskip("torch")

SCALE = 21
SETTINGS = dict(hop_limit=2, cmax=256, ball=256, level_work=1024, memo=1_000_000_000)


def test_rmat_2_21_equals_the_oracle():
    from paper_2412_18008_gb300 import ch
    g = I.rmat_graph(scale=SCALE, nsamples=16 << SCALE, wmax=1000, seed=8)
    gch = ch.CH.build(g, hop_limit=SETTINGS["hop_limit"], max_candidates_per_vertex=SETTINGS["cmax"],
                      witness_ball_limit=SETTINGS["ball"], witness_level_work=SETTINGS["level_work"],
                      witness_memo_limit=SETTINGS["memo"])
    och = O.build_ch(g, SETTINGS["hop_limit"], cmax=SETTINGS["cmax"], ball=SETTINGS["ball"],
                     level_work=SETTINGS["level_work"], memo=SETTINGS["memo"], threads=True)
    assert int((och.level == och.rounds).sum()) > 0, "expected a core under the candidate bound"
    assert_same_hierarchy(gch, och)
    s, t = I.random_pairs(g.n, 40, seed=9)
    assert np.array_equal(gch.query(s, t), O.dijkstra_pairs(g, s, t))
