"""Failure detection by host-side injection (no GPU fault): a chosen device
allocation of the library fails as if the device were out of memory. The
call in progress must return CH_ENOMEM and release what it had allocated,
and the library must keep working: the next build equals the oracle's."""
import numpy as np
import pytest

import oracle as O
from paper_2412_18008_gb300 import inputs as I


def _ch():
    from paper_2412_18008_gb300 import ch
    return ch


def test_setting_and_reset_make_no_cuda_call():
    ch = _ch()
    assert ch.debug_fail_alloc(-1) == -1
    assert ch.debug_fail_alloc(7) == -1
    assert ch.debug_fail_alloc(2) == 7
    assert ch.debug_fail_alloc(-9) == 2  # any negative value turns it off
    assert ch.debug_fail_alloc(-1) == -1


@pytest.mark.gpu
def test_every_build_allocation_can_fail_cleanly():
    import torch
    from tests.test_gpu_parity import assert_same_hierarchy
    ch = _ch()
    g = I.geometric_knn_graph(5000, seed=141)
    och = O.build_ch(g, 5)
    ch.CH.build(g, hop_limit=5).close()  # first-call state (static scratch) in place
    ch.trim_memory()  # cached blocks back to CUDA: what is left is held by someone
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    k = 0
    while True:
        ch.debug_fail_alloc(k)
        try:
            h = ch.CH.build(g, hop_limit=5)
        except ch.CHError as e:
            assert e.code == ch.CH_ENOMEM and "injected" in str(e), (k, e)
            failed += 1
        else:
            left = ch.debug_fail_alloc(-1)
            assert left >= 0  # the build needed fewer than k + 1 allocations
            assert_same_hierarchy(h, och)
            h.close()
            break
        ch.debug_fail_alloc(-1)
        assert_same_hierarchy(ch.CH.build(g, hop_limit=5), och)
        k += 1
        assert k < 10_000
    assert failed == k and failed > 10
    ch.trim_memory()
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)  # nothing leaked


@pytest.mark.gpu
def test_query_allocation_failure_leaves_the_handle_usable():
    ch = _ch()
    g = I.grid_graph(20, 20, 0.1, 1, 20, seed=142)
    h = ch.CH.build(g, hop_limit=5)
    s, t = I.random_pairs(g.n, 5000, seed=143)
    want = O.dijkstra_pairs(g, s, t)
    for k in range(0, 6):
        ch.debug_fail_alloc(k)
        try:
            got = h.query(s, t)
        except ch.CHError as e:
            assert e.code == ch.CH_ENOMEM
        else:
            assert np.array_equal(got, want)
        ch.debug_fail_alloc(-1)
        assert np.array_equal(h.query(s, t), want)


def test_settled_cap_with_a_ball_bound_is_rejected_before_any_cuda_call():
    # ch_build checks its parameters first; the settled-vertex cap replaces
    # the hop-limited search, so a ball bound beside it is an error
    ch = _ch()
    g = I.grid_graph(8, 8, 0.1, 1, 20, seed=3)
    with pytest.raises(ch.CHError) as ei:
        ch.CH.build(g, hop_limit=5, witness_settle_cap=4, witness_ball_limit=3)
    assert ei.value.code == ch.CH_EINVAL
    assert "settled-vertex cap" in str(ei.value)
