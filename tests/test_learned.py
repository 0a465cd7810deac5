"""Learned priority: features, MLP inference and training, and the
hierarchy built with it.

The paper has no learned priority; any priority yields exact distances, so
the learned path is checked as follows: integer features and labels bit for
bit against the oracle; MLP outputs and gradients against a float64 CPU
reference with the same BF16 roundings, within stated tolerances; the
hierarchy of a learned build bit for bit against an oracle replay fed the
int32 priorities the GPU computed; distances against Dijkstra.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_2412_18008_gb300 import inputs as I
from tests.graphs import all_pairs_truth

# ---------------------------------------------------------------------------
# CPU pins of the reference MLP
# ---------------------------------------------------------------------------


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(0, 30, 50_000).astype(np.float32)
    x[:5] = [0.0, -0.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, 65504.0]
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), ref)


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    w = M.init_weights(7).astype(np.float64)
    X = rng.normal(0, 3, (40, M.NIN))
    lab = rng.normal(0, 5, 40)
    _, g = M.loss_and_grad(w, X, lab, quantise=False)
    eps = 1e-6
    for i in rng.choice(M.NPARAM, 60, replace=False):
        e = np.zeros(M.NPARAM)
        e[i] = eps
        fd = (M.loss_and_grad(w + e, X, lab, False)[0] - M.loss_and_grad(w - e, X, lab, False)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-5 + 1e-3 * abs(g[i]), (i, fd, g[i])


U_BF16 = 2.0 ** -7   # one BF16 unit, relative to the value (8 significant bits)
U_F32 = 2.0 ** -24


def _gamma(k):
    """Relative error bound of a k-term float32 sum (or dot product)."""
    return k * U_F32 / (1.0 - k * U_F32)


def grad_error_bound(w, X, labels):
    """Per-element bound on |g - g_ref| between a float32 implementation of
    the MLP's loss gradient that rounds as the inference does (inputs, W1, W2
    and the first hidden layer to BF16) and the float64 reference
    M.loss_and_grad. First-order propagation of (a) float32 rounding of every
    sum and (b) one BF16 unit of every first-hidden-layer value (its
    pre-activation may round to the other neighbour), through the forward
    pass and back; a ReLU whose input lies within its error of 0 may switch,
    which adds the whole upstream term."""
    W1, b1, W2, b2, W3, b3 = M.split(w)
    q = M.bf16
    x, W1q, W2q = q(X), q(W1), q(W2)
    n = X.shape[0]
    labels = np.asarray(labels, np.float64)
    z1 = x @ W1q + b1
    e_z1 = _gamma(M.NIN + 1) * (np.abs(x) @ np.abs(W1q) + np.abs(b1))
    a1 = np.maximum(z1, 0.0)
    h1 = q(a1)
    d_h1 = np.where(z1 + e_z1 > 0, e_z1 + U_BF16 * (a1 + e_z1), 0.0)
    m1, u1 = h1 > 0, np.abs(z1) <= e_z1
    z2 = h1 @ W2q + b2
    e_z2 = _gamma(M.NH + 1) * (np.abs(h1) @ np.abs(W2q) + np.abs(b2)) + d_h1 @ np.abs(W2q)
    h2 = np.maximum(z2, 0.0)
    d_h2 = np.where(z2 + e_z2 > 0, e_z2, 0.0)
    m2, u2 = h2 > 0, np.abs(z2) <= e_z2
    y = h2 @ W3 + b3
    e_y = _gamma(M.NH + 1) * (np.abs(h2) @ np.abs(W3) + abs(b3)) + d_h2 @ np.abs(W3)
    dy = 2.0 * (y - labels) / n
    d_dy = 2.0 * (e_y + 2 * U_F32 * (np.abs(y) + np.abs(labels))) / n + 2 * U_F32 * np.abs(dy)
    G = _gamma(n)
    ady = np.abs(dy)
    b_gW3 = d_h2.T @ ady + np.abs(h2).T @ d_dy + d_h2.T @ d_dy + G * (np.abs(h2).T @ ady)
    b_gb3 = d_dy.sum() + G * ady.sum()
    ag2 = np.abs(np.outer(dy, W3))
    g2 = ag2 * m2
    d_g2 = np.outer(d_dy, np.abs(W3)) * (m2 | u2) + u2 * ag2 + U_F32 * ag2
    b_gW2 = d_h1.T @ g2 + np.abs(h1).T @ d_g2 + d_h1.T @ d_g2 + G * (np.abs(h1).T @ g2)
    b_gb2 = d_g2.sum(0) + G * g2.sum(0)
    pre1 = np.abs(np.outer(dy, W3) * m2) @ np.abs(W2q).T
    e_pre1 = d_g2 @ np.abs(W2q).T + _gamma(M.NH) * pre1
    d_g1 = e_pre1 * (m1 | u1) + u1 * pre1
    ag1 = pre1 * m1
    b_gW1 = np.abs(x).T @ d_g1 + G * (np.abs(x).T @ ag1)
    b_gb1 = d_g1.sum(0) + G * ag1.sum(0)
    return M.join(b_gW1, b_gb1, b_gW2, b_gb2, b_gW3, b_gb3)


def _float32_grad(w, X, labels, mistake=None):
    """The gradient computed in float32 with the inference's BF16 roundings
    (a CPU stand-in for the GPU's arithmetic); `mistake` plants one error."""
    f = np.float32
    W1, b1, W2, b2, W3, b3 = (np.asarray(a, f) for a in M.split(w))
    q = lambda a: M.bf16(a).astype(f)
    x = q(X)
    h1 = q(np.maximum(x @ q(W1) + b1, f(0)))
    h2 = np.maximum(h1 @ q(W2) + b2, f(0))
    y = h2 @ W3 + f(b3)
    n = X.shape[0]
    dy = (f(2) * (y - np.asarray(labels, f)) / f(n)).astype(f)
    gW3, gb3 = h2.T @ dy, dy.sum(dtype=f)
    g2 = np.outer(dy, W3) * (h2 > 0)
    gW2, gb2 = h1.T @ g2, g2.sum(0)
    g1 = (g2 @ q(W2).T) * (h1 > 0)
    if mistake == "transposed W2":
        g1 = (g2 @ q(W2)) * (h1 > 0)
    gW1, gb1 = x.T @ g1, g1.sum(0)
    if mistake == "b3 sign":
        gb3 = -gb3
    if mistake == "W3 from h1":
        gW3 = h1.T @ dy
    if mistake == "b2 dropped mask":
        gb2 = np.outer(dy, W3).sum(0)
    return M.join(gW1, gb1, gW2, gb2, gW3, gb3)


def _trace_batch(n_rows=3000, seed=52):
    och = O.build_ch(I.geometric_knn_graph(4_000, seed=seed), 5, trace=True)
    rows = och.trace[:n_rows]
    return M.transform(rows[:, 2:]), M.targets(rows).astype(np.float32)


def test_gradient_bound_holds_for_float32_and_catches_mistakes():
    X, lab = _trace_batch()
    w = M.init_weights(3)
    _, g_ref = M.loss_and_grad(w, X, lab.astype(np.float64))
    bound = grad_error_bound(w, X, lab)
    g32 = _float32_grad(w, X, lab).astype(np.float64)
    assert (np.abs(g32 - g_ref) <= bound).all()
    # the bound is tight enough to matter: below a tenth of |g| for most
    assert np.median(bound / np.maximum(np.abs(g_ref), 1e-30)) < 0.1
    for mistake in ("transposed W2", "b3 sign", "W3 from h1", "b2 dropped mask"):
        bad = _float32_grad(w, X, lab, mistake).astype(np.float64)
        assert (np.abs(bad - g_ref) > bound).any(), mistake


def test_training_target_closed_forms():
    # rows (round, vertex, S, |N_in|, |N_out|, |N|, ED, cn, depth, ...):
    # the target is sign(x) * log2(1 + |x|) of x = ED + 2 * depth
    rows = np.zeros((5, 14), np.int64)
    rows[:, 2 + 4] = [0, 3, -7, 1, -2]   # edge difference
    rows[:, 2 + 6] = [0, 2, 0, 7, 1]     # hierarchy depth
    # x = 0, 7, -7, 15, 0
    assert M.targets(rows).tolist() == [0.0, 3.0, -3.0, 4.0, 0.0]


def test_round0_trace_features_recomputed():
    g = I.random_digraph(60, 200, 1, 20, seed=9)
    och = O.build_ch(g, 5, trace=True)
    rows = och.trace[och.trace[:, 0] == 0]
    assert rows.shape[0] == g.n and (rows[:, 1] == np.arange(g.n)).all()
    ed = O.round0_scores(g, 5)
    off, tgt, w = O.normalize(g)
    outs = [set(tgt[off[u]:off[u + 1]].tolist()) for u in range(g.n)]
    ins = [set() for _ in range(g.n)]
    wsum = np.zeros(g.n, np.int64)
    for u in range(g.n):
        for e in range(off[u], off[u + 1]):
            ins[tgt[e]].add(u)
            wsum[u] += w[e]
            wsum[tgt[e]] += w[e]
    for u in range(g.n):
        i, o = len(ins[u]), len(outs[u])
        want = [ed[u] + i + o, i, o, len(ins[u] | outs[u]), ed[u], 0, 0, 0, i * o, i + o, 0,
                wsum[u] // (i + o) if i + o else 0]
        assert rows[u, 2:].tolist() == want, u


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

gpu = pytest.mark.gpu


def _ch():
    from paper_2412_18008_gb300 import ch
    return ch


def _torch():
    return pytest.importorskip("torch")


@gpu
@pytest.mark.parametrize("which", ["grid", "geo"])
def test_trace_matches_oracle(which):
    g = I.workload("grid64")[0] if which == "grid" else I.geometric_knn_graph(20_000, seed=51)
    gch = _ch().CH.build(g, hop_limit=5, trace=True)
    tr = gch.export_trace()
    och = O.build_ch(g, 5, trace=True)
    assert np.array_equal(tr["rows"], och.trace)
    assert np.array_equal(tr["prio"], och.trace[:, 6].astype(np.int32))  # heuristic = edge difference
    assert np.array_equal(tr["labels"], och.labels)


def _train_data(graphs):
    """Trace rows of plain (edge-difference) builds and their labels."""
    rows, labels = [], []
    for g in graphs:
        tr = _ch().CH.build(g, hop_limit=5, trace=True).export_trace()
        rows.append(tr["rows"])
        labels.append(_ch().training_labels(tr["rows"]))
    return np.concatenate(rows), np.concatenate(labels)


@gpu
def test_training_targets_match_oracle():
    torch = _torch()
    och = O.build_ch(I.geometric_knn_graph(5_000, seed=50), 5, trace=True)
    rows = och.trace
    got = _ch().training_labels(rows)
    want = M.targets(rows).astype(np.float32)
    # both round log2 of the same integer to float32; allow one float32 unit
    assert np.allclose(got, want, rtol=2.0 ** -23, atol=0)
    # device input gives a device result, asynchronous on the stream
    d = _ch().training_labels(torch.from_numpy(rows).cuda())
    assert np.array_equal(d.cpu().numpy(), got)


@gpu
def test_mlp_forward_and_gradient_match_cpu_reference():
    torch = _torch()
    ch = _ch()
    rows, labels = _train_data([I.geometric_knn_graph(8_000, seed=52)])
    rows, labels = rows[:6000], labels[:6000]
    w = M.init_weights(3)
    drows = torch.from_numpy(rows).cuda()
    y = ch.mlp_forward(w, drows).cpu().numpy().astype(np.float64)
    X = M.transform(rows[:, 2:])
    y_ref, _ = M.forward(w, X)
    # FP32 accumulation on the GPU vs float64 here: only BF16 rounding flips
    # of the first hidden layer can differ, one BF16 unit (2^-8) each.
    assert np.allclose(y, y_ref, rtol=2e-2, atol=2e-2), np.max(np.abs(y - y_ref))
    dl = torch.from_numpy(labels).cuda()
    dw = torch.from_numpy(w.copy()).cuda()
    grad, loss = ch.mlp_train(drows, dl, dw, epochs=0, batch=rows.shape[0])
    L_ref, g_ref = M.loss_and_grad(w, X, labels.astype(np.float64))
    g = grad.cpu().numpy().astype(np.float64)
    # element by element, within the bound BF16 and float32 rounding allow
    bound = grad_error_bound(w, X, labels)
    bad = np.nonzero(np.abs(g - g_ref) > bound)[0]
    assert bad.size == 0, (bad[:10], g[bad[:10]], g_ref[bad[:10]], bound[bad[:10]])
    assert abs(loss[0] - L_ref) <= 1e-3 * L_ref


@gpu
def test_training_lowers_loss_and_is_deterministic():
    torch = _torch()
    ch = _ch()
    rows, labels = _train_data([I.geometric_knn_graph(20_000, seed=s) for s in (53, 54)])
    drows, dl = torch.from_numpy(rows).cuda(), torch.from_numpy(labels).cuda()
    w0 = M.init_weights(4)
    wa = torch.from_numpy(w0.copy()).cuda()
    wb = torch.from_numpy(w0.copy()).cuda()
    la = ch.mlp_train(drows, dl, wa, epochs=4, batch=4096)
    lb = ch.mlp_train(drows, dl, wb, epochs=4, batch=4096)
    assert la[-1] < 0.5 * la[0] and all(np.diff(la) < 0)
    assert np.array_equal(la, lb) and torch.equal(wa, wb)


def _trained_weights(graphs, epochs=8):
    torch = _torch()
    rows, labels = _train_data(graphs)
    w = torch.from_numpy(M.init_weights(11)).cuda()
    loss = _ch().mlp_train(torch.from_numpy(rows).cuda(), torch.from_numpy(labels).cuda(), w,
                           epochs=epochs, batch=4096)
    print("training loss per epoch", np.round(loss, 4).tolist())
    return w.cpu().numpy()


@gpu
def test_learned_build_matches_oracle_replay_and_keeps_distances():
    w = _trained_weights([I.geometric_knn_graph(20_000, seed=55)], epochs=3)
    for g in (I.geometric_knn_graph(15_000, seed=56), I.random_digraph(400, 1500, 1, 30, seed=57)):
        gch = _ch().CH.build(g, hop_limit=5, mlp_weights=w, trace=True)
        tr = gch.export_trace()
        och = O.build_ch(g, 5, replay=(tr["rows"][:, 0], tr["rows"][:, 1], tr["prio"]))
        from tests.test_gpu_parity import assert_same_hierarchy
        assert_same_hierarchy(gch, och)
        s, t = I.random_pairs(g.n, 3000, seed=58)
        d = gch.query(s, t)
        assert np.array_equal(d, O.dijkstra_pairs(g, s, t))
    g = I.random_digraph(150, 600, 1, 30, seed=59)
    gch = _ch().CH.build(g, hop_limit=5, mlp_weights=w)
    ss, tt = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    d = gch.query(ss.ravel().astype(np.uint32), tt.ravel().astype(np.uint32))
    assert np.array_equal(d.astype(np.uint64).reshape(g.n, g.n), all_pairs_truth(g))


@gpu
def test_learned_priority_gain_over_edge_difference():
    """Trained on traces of the plain method, the learned priority gives a
    hierarchy with a smaller mean search space on a held-out graph of the
    family (its target score adds twice the hierarchy depth to the edge
    difference, which keeps the hierarchy shallow)."""
    w = _trained_weights([I.geometric_knn_graph(40_000, seed=s) for s in (60, 61, 62, 63)])
    g = I.geometric_knn_graph(60_000, seed=64)
    s, t = I.random_pairs(g.n, 20_000, seed=65)
    heur = _ch().CH.build(g, hop_limit=5)
    lrn = _ch().CH.build(g, hop_limit=5, mlp_weights=w)
    dh, sh = heur.query(s, t, want_settled=True)
    dl, sl = lrn.query(s, t, want_settled=True)
    assert np.array_equal(dh, dl)
    print(f"edge difference: {heur.stats()['shortcuts']} shortcuts, mean search space {sh.mean():.1f}; "
          f"learned: {lrn.stats()['shortcuts']} shortcuts, mean search space {sl.mean():.1f}")
    assert sl.mean() < sh.mean()
