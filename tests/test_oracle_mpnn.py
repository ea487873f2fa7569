"""Pins of the learned initial partitioner's oracle (oracle/mpnn.py): the
network's structure against dense-matrix restatements, its analytic gradient
against central finite differences, the bf16 rounding against torch's
conversion, the features against hand-computed values and the C oracle's
greedy order, and the balanced decode against hand cases and invariants."""
import math

import numpy as np
import pytest
import torch

import graphgen
import oracle
from helpers import graph_from_triples
from oracle import mpnn


def _dense_mean(g):
    """Row-normalised 0/1 adjacency (rows of isolated vertices are zero)."""
    M = np.zeros((g.n, g.n))
    for v in range(g.n):
        nb = g.adjncy[g.xadj[v]:g.xadj[v + 1]]
        for u in nb:
            M[v, u] += 1.0 / len(nb)
    return M


def _small_graph(seed=3):
    g = graphgen.with_weights(graphgen.gnp(30, 0.12, seed=seed),
                              vwgt=np.random.default_rng(seed).integers(1, 5, 30).astype(np.int32))
    return g


def _theta(k, seed, scale=0.3):
    r = np.random.default_rng(seed)
    return r.normal(0, scale, mpnn.num_params(k))


def test_bf16_rounding_matches_torch():
    r = np.random.default_rng(0)
    x = np.concatenate([r.normal(0, 3, 4000), r.normal(0, 1e-30, 100), [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9,
                                                                        -(1 + 2 ** -8), 65504.0, 3e38]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mpnn.bf16(x), ref)
    # ties to even, by hand
    assert mpnn.bf16(np.float32(1 + 2 ** -8)) == 1.0
    assert mpnn.bf16(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


@pytest.mark.parametrize("g,k", [(graphgen.grid2d(9, 7), 4), (graphgen.rmat(9, seed=2, vw=(1, 4)), 8),
                                 (graphgen.disjoint_union(graphgen.grid2d(4, 4), graphgen.gnp(20, 0.05, seed=1)), 3)],
                         ids=["grid", "rmat_w", "union"])
def test_greedy_order_matches_initial_partition(g, k):
    _, _, S, W = mpnn.greedy_order(g)
    assert np.array_equal((k * S) // W, oracle.initial_partition(g, k))


def test_features_hand_computed():
    # path 0-1-2 (edge weights 5 and 7) and isolated vertex 3; weights 1..4
    g = graph_from_triples(4, [[0, 1, 5], [1, 2, 7]])
    g = graphgen.with_weights(g, vwgt=np.array([1, 2, 3, 4], np.int32))
    X = mpnn.features(g).astype(np.float64)
    s = np.array([0, 1, 3, 6]) / 10
    want = np.zeros((4, 16))
    want[:, 0] = 1
    want[:, 1] = [0.5, 1, 0.5, 0]
    want[:, 2] = [0.25, 0.5, 0.75, 1]
    want[:, 3] = s
    want[:, 4] = [0, 0.5, 1, 0]
    want[:, 5] = np.array([5, 12, 7, 0]) / 12
    for j in range(5):
        for t, off in ((6, 0.0), (11, 0.25)):
            y = s * 2 ** j + off
            want[:, t + j] = np.abs(2 * (y - np.floor(y)) - 1)
    assert np.allclose(X, want, atol=1e-6)


def test_features_unit_graph_and_ranges():
    g = graphgen.rmat(10, seed=4)
    X = mpnn.features(g)
    assert X.dtype == np.float32 and X.shape == (g.n, 16)
    assert (X >= 0).all() and (X <= 1).all() and (X[:, 0] == 1).all()
    assert np.array_equal(X[:, 5], X[:, 1])          # unit edge weights: weighted degree = degree


def test_mean_aggregation_is_row_normalised_adjacency():
    g = _small_graph()
    H = np.random.default_rng(1).normal(size=(g.n, 7))
    assert np.allclose(mpnn.mean_agg(g, H), _dense_mean(g) @ H, atol=1e-12)
    G = np.random.default_rng(2).normal(size=(g.n, 7))
    assert np.allclose(mpnn.mean_agg_t(g, G), _dense_mean(g).T @ G, atol=1e-12)


def test_zero_network_gives_uniform_softmax():
    g = _small_graph()
    k = 6
    y = np.random.default_rng(5).integers(0, k, g.n)
    loss, grad = mpnn.loss_and_grad(g, mpnn.features(g), np.zeros(mpnn.num_params(k)), k, y)
    assert abs(loss - math.log(k)) < 1e-12
    P = mpnn.unflatten(grad, k)
    want_bo = 1.0 / k - np.bincount(y, minlength=k) / g.n
    assert np.allclose(P[-1], want_bo, atol=1e-15)
    assert all(np.abs(p).max() == 0 for p in P[:-1])   # every path to the loss passes a zero weight


def _structured_theta(k, take):
    """Weights that copy one half of [H, A] through every layer: take = 0
    passes H (the vertex's own state), take = 1 passes A (the mean of its
    neighbours').  Output logits = the first k columns."""
    P = [np.zeros(s) for s in mpnn.param_shapes(k)]
    d = mpnn.FEATURES
    for l in range(mpnn.LAYERS):
        W = P[2 * l]
        for i in range(d):
            W[take * d + i, i] = 1.0
        d = mpnn.HIDDEN
    for i in range(k):
        P[-2][i, i] = 1.0
    return mpnn.flatten(P)


def test_self_half_passes_features_through():
    g = _small_graph()
    k = 5
    X = mpnn.features(g)
    logits, _, _ = mpnn.forward(g, X, _structured_theta(k, 0), k)
    assert np.array_equal(logits, X[:, :k].astype(np.float64))


def test_neighbour_half_is_three_mean_hops():
    g = _small_graph()
    k = 5
    X = mpnn.features(g).astype(np.float64)
    logits, _, _ = mpnn.forward(g, X, _structured_theta(k, 1), k)
    M = _dense_mean(g)
    assert np.allclose(logits, M @ M @ M @ X[:, :k], atol=1e-12)


def test_gradient_matches_central_differences():
    g = _small_graph(7)
    k = 5
    X = mpnn.features(g)
    rng = np.random.default_rng(11)
    theta = _theta(k, 12)
    y = rng.integers(0, k, g.n)
    _, grad = mpnn.loss_and_grad(g, X, theta, k, y)
    # a sample of every parameter block, plus the largest gradients
    offs = np.cumsum([0] + [int(np.prod(s)) for s in mpnn.param_shapes(k)])
    idx = np.concatenate([rng.choice(np.arange(offs[i], offs[i + 1]), min(25, offs[i + 1] - offs[i]), replace=False)
                          for i in range(len(offs) - 1)] + [np.argsort(-np.abs(grad))[:20]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mpnn.loss_and_grad(g, X, tp, k, y)[0] - mpnn.loss_and_grad(g, X, tm, k, y)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 + 1e-5 * abs(grad[i]), (i, fd, grad[i])


def test_bf16_emulation_stays_within_bf16_error():
    g = _small_graph(9)
    k = 8
    X = mpnn.features(g)
    y = np.random.default_rng(3).integers(0, k, g.n)
    theta = _theta(k, 4)
    l64, g64 = mpnn.loss_and_grad(g, X, theta, k, y)
    l16, g16 = mpnn.loss_and_grad(g, X, theta, k, y, emulate_bf16=True)
    assert abs(l16 - l64) < 0.02 * abs(l64)
    assert np.linalg.norm(g16 - g64) < 0.05 * np.linalg.norm(g64)


def test_canonical_relabelling():
    # mean positions: part 3 -> 0.5, parts 0 and 1 -> 3 (tie: lower id first), part 2 -> 5
    part = np.array([3, 3, 1, 0, 1, 2])
    assert list(mpnn.canonical(part)) == [0, 0, 2, 1, 2, 3]
    # reversed visit order: part 2 -> 0, parts 0 and 1 -> 2, part 3 -> 4.5
    assert list(mpnn.canonical(part, order=[5, 4, 3, 2, 1, 0])) == [3, 3, 2, 1, 2, 0]
    # a partition into consecutive pieces of the order keeps its numbering
    r = np.random.default_rng(1)
    order = r.permutation(40)
    seq = np.repeat(np.arange(8), 5)
    p = np.empty(40, np.int64)
    p[order] = r.permutation(8)[seq]
    assert np.array_equal(mpnn.canonical(p, order)[order], seq)


def test_decode_keeps_argmax_when_every_part_has_room():
    r = np.random.default_rng(2)
    L = r.normal(size=(50, 7)).astype(np.float32)
    assert np.array_equal(mpnn.decode(L, None, 7, 50), np.argmax(L, axis=1))


def test_decode_overflow_goes_to_lightest_part_by_margin():
    # all three vertices prefer part 0; margins 3, 2, 1; cap 2: the vertex
    # with the smallest margin (id 2) goes to the lightest part, part 1
    L = np.array([[4, 1, 0], [3, 1, 0], [2, 1, 0]], np.float32)
    assert list(mpnn.decode(L, None, 3, 2)) == [0, 0, 1]
    # equal margins: ids break the tie, the highest id moves
    L = np.array([[1, 0], [1, 0], [1, 0]], np.float32)
    assert list(mpnn.decode(L, None, 2, 2)) == [0, 0, 1]


def test_decode_respects_cap_with_unit_weights():
    r = np.random.default_rng(8)
    n, k = 400, 16
    L = (r.normal(size=(n, k)) + np.linspace(0, 3, k)).astype(np.float32)   # skewed preferences
    Lim, opt = oracle.limit(n, k, 0.03)
    part = mpnn.decode(L, None, k, Lim)
    assert np.bincount(part, minlength=k).max() <= Lim
