"""Plain statement of the learned initial partitioner's network (the learned
form of the coarsest-level partition; the paper's initial partition is Metis,
Sec. 3, and the learned form is an extension of this build).

TEST INFRASTRUCTURE ONLY: the tests call it to check the library's kernels;
the library never imports it.  Everything here is numpy, written out step by
step: the input features (float32, operation by operation, so that they are
bit-identical to the library's), a 3-layer mean-aggregation message-passing
network with hidden width 64 and a softmax over k parts, its cross-entropy
loss and its analytic backward pass (float64), an optional emulation of the
bf16 rounding that the library applies to the operands of its dense layers,
and the canonical relabelling of a partition.

Network (rows are vertices):
    H0 = X                                        (n x 16 features)
    A_l = mean over N(v) of H_{l-1}               (0 for isolated vertices)
    H_l = relu([H_{l-1}, A_l] W_l + b_l)          l = 1, 2, 3 (width 64)
    logits = H3 Wo + bo                           (n x k)
    loss = mean over v of -log softmax(logits_v)[y_v]
Parameter vector order: W1 (32 x 64), b1, W2 (128 x 64), b2, W3 (128 x 64),
b3, Wo (64 x k), bo; matrices row-major (input index first).
"""
from __future__ import annotations

from collections import deque

import numpy as np

FEATURES = 16
HIDDEN = 64
LAYERS = 3


def param_shapes(k: int):
    shapes = []
    din = FEATURES
    for _ in range(LAYERS):
        shapes += [(2 * din, HIDDEN), (HIDDEN,)]
        din = HIDDEN
    shapes += [(HIDDEN, k), (k,)]
    return shapes


def num_params(k: int) -> int:
    return int(sum(np.prod(s) for s in param_shapes(k)))


def unflatten(theta, k: int):
    out, o = [], 0
    for s in param_shapes(k):
        c = int(np.prod(s))
        out.append(np.asarray(theta[o:o + c], dtype=np.float64).reshape(s))
        o += c
    return out


def flatten(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def greedy_order(g):
    """Component root (lowest id), BFS distance from it, and S(v): the weight
    of the vertices before v in (root, distance, id) order (the greedy initial
    partition's order)."""
    n = g.n
    root = -np.ones(n, np.int64)
    dist = np.zeros(n, np.int64)
    for s in range(n):
        if root[s] >= 0:
            continue
        root[s] = s
        q = deque([s])
        while q:
            v = q.popleft()
            for u in g.adjncy[g.xadj[v]:g.xadj[v + 1]]:
                if root[u] < 0:
                    root[u] = s
                    dist[u] = dist[v] + 1
                    q.append(u)
    vw = np.ones(n, np.int64) if g.vwgt is None else np.asarray(g.vwgt, np.int64)
    order = np.lexsort((np.arange(n), dist, root))
    S = np.zeros(n, np.int64)
    S[order] = np.concatenate([[0], np.cumsum(vw[order])[:-1]]) if n else S
    return root, dist, S, int(vw.sum())


def _tri(y):
    y = np.float32(y) if np.isscalar(y) else y.astype(np.float32)
    fr = (y - np.floor(y)).astype(np.float32)
    return np.abs((np.float32(2) * fr).astype(np.float32) - np.float32(1)).astype(np.float32)


def features(g) -> np.ndarray:
    """n x 16 float32: 1, deg/maxdeg, vw/maxvw, S/W, dist/maxdist,
    wdeg/maxwdeg, then triangle waves of 2^j S/W (j = 0..4) and of
    2^j S/W + 1/4 (j = 0..4).  Each ratio is a single float32 division of
    float32-converted integers."""
    n = g.n
    _, dist, S, W = greedy_order(g)
    deg = np.diff(np.asarray(g.xadj, np.int64))
    vw = np.ones(n, np.int64) if g.vwgt is None else np.asarray(g.vwgt, np.int64)
    ew = None if g.adjwgt is None else np.asarray(g.adjwgt, np.int64)
    wdeg = np.zeros(n, np.int64)
    for v in range(n):
        row = slice(int(g.xadj[v]), int(g.xadj[v + 1]))
        wdeg[v] = deg[v] if ew is None else int(ew[row].sum())
    f32 = np.float32

    def ratio(a, b):
        b = max(int(b), 1)
        return (a.astype(np.float32) / f32(b)).astype(np.float32)
    X = np.zeros((n, FEATURES), np.float32)
    X[:, 0] = 1
    X[:, 1] = ratio(deg, deg.max() if n else 1)
    X[:, 2] = ratio(vw, vw.max() if n else 1)
    s = ratio(S, W)
    X[:, 3] = s
    X[:, 4] = ratio(dist, dist.max() if n else 1)
    X[:, 5] = ratio(wdeg, wdeg.max() if n else 1)
    for j in range(5):
        X[:, 6 + j] = _tri((s * f32(2 ** j)).astype(np.float32))
        X[:, 11 + j] = _tri(((s * f32(2 ** j)).astype(np.float32) + f32(0.25)).astype(np.float32))
    return X


def mean_agg(g, H):
    n = g.n
    A = np.zeros_like(H)
    for v in range(n):
        nb = g.adjncy[g.xadj[v]:g.xadj[v + 1]]
        if len(nb):
            A[v] = H[nb].sum(axis=0) / len(nb)
    return A


def mean_agg_t(g, dA):
    """Transpose of mean_agg: dH[u] = sum over v in N(u) of dA[v] / deg(v)."""
    n = g.n
    deg = np.diff(np.asarray(g.xadj, np.int64))
    dH = np.zeros_like(dA)
    for v in range(n):
        nb = g.adjncy[g.xadj[v]:g.xadj[v + 1]]
        if len(nb):
            dH[nb] += dA[v] / len(nb)
    return dH


def forward(g, X, theta, k, emulate_bf16=False):
    rnd = bf16 if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    P = unflatten(theta, k)
    H = np.asarray(X, np.float64)
    cache = []
    for l in range(LAYERS):
        W, b = P[2 * l], P[2 * l + 1]
        A = mean_agg(g, H)
        Z = np.concatenate([H, A], axis=1)
        Y = rnd(Z) @ rnd(W) + b
        cache.append((H, A, Z, Y))
        H = np.maximum(Y, 0)
    Wo, bo = P[-2], P[-1]
    logits = rnd(H) @ rnd(Wo) + bo
    return logits, cache, H


def loss_and_grad(g, X, theta, k, y, emulate_bf16=False):
    """Mean cross-entropy and its gradient with respect to theta (float64)."""
    rnd = bf16 if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    P = unflatten(theta, k)
    n = g.n
    logits, cache, H3 = forward(g, X, theta, k, emulate_bf16)
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    sm = e / e.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(sm[np.arange(n), y])))
    dlog = sm.copy()
    dlog[np.arange(n), y] -= 1
    dlog /= n
    grads = [None] * len(P)
    Wo = P[-2]
    grads[-2] = rnd(H3).T @ rnd(dlog)
    grads[-1] = dlog.sum(axis=0)
    dH = rnd(dlog) @ rnd(Wo).T
    for l in reversed(range(LAYERS)):
        H, A, Z, Y = cache[l]
        W = P[2 * l]
        dY = dH * (Y > 0)
        grads[2 * l] = rnd(Z).T @ rnd(dY)
        grads[2 * l + 1] = dY.sum(axis=0)
        dZ = rnd(dY) @ rnd(W).T
        d = H.shape[1]
        dH = dZ[:, :d] + mean_agg_t(g, dZ[:, d:])
    return loss, flatten(grads)


def canonical(part, order=None) -> np.ndarray:
    """Relabel parts 0, 1, 2, ... by the mean position of their vertices when
    the vertices are visited in `order` (default: id order); equal means by
    part id; parts without vertices take no label.  Means are compared
    exactly (sum_p * count_q against sum_q * count_p)."""
    part = np.asarray(part)
    order = np.arange(len(part)) if order is None else np.asarray(order)
    pos = np.empty(len(part), np.int64)
    pos[order] = np.arange(len(part))
    parts = sorted(set(int(p) for p in part))
    tot = {p: 0 for p in parts}
    cnt = {p: 0 for p in parts}
    for v in range(len(part)):
        tot[int(part[v])] += int(pos[v])
        cnt[int(part[v])] += 1

    def before(q, p):
        a, b = tot[q] * cnt[p], tot[p] * cnt[q]
        return a < b or (a == b and q < p)
    label = {p: sum(before(q, p) for q in parts if q != p) for p in parts}
    return np.array([label[int(p)] for p in part], dtype=part.dtype)


def greedy_sequence(g) -> np.ndarray:
    """Vertices in (component root, BFS distance, id) order."""
    root, dist, _, _ = greedy_order(g)
    return np.lexsort((np.arange(g.n), dist, root))


def decode(logits, vw, k: int, cap: int) -> np.ndarray:
    """Balanced decode of float32 logits (n x >= k; columns past k ignored).
    Each vertex prefers a(v) = argmax of its k logits (lowest part on ties);
    its margin is the float32 difference between the largest and the second
    largest logit (0 when k = 1).  Vertices are visited by margin descending,
    then id ascending; a vertex takes a(v) when that part's weight plus its
    own stays <= cap, else the lightest part (lowest id on ties)."""
    L = np.asarray(logits, np.float32)[:, :k]
    n = L.shape[0]
    vw = np.ones(n, np.int64) if vw is None else np.asarray(vw, np.int64)
    a = np.argmax(L, axis=1) if n else np.zeros(0, np.int64)
    margin = np.zeros(n, np.float32)
    if k > 1 and n:
        top = L[np.arange(n), a]
        rest = L.copy()
        rest[np.arange(n), a] = -np.inf
        margin = (top - rest.max(axis=1)).astype(np.float32)
    order = np.lexsort((np.arange(n), -margin))
    w = np.zeros(k, np.int64)
    part = np.empty(n, np.int32)
    for v in order:
        p = int(a[v])
        if w[p] + vw[v] > cap:
            p = int(np.argmin(w))
        part[v] = p
        w[p] += vw[v]
    return part
