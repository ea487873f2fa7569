"""Small helpers shared by the tests (no method arithmetic)."""
import itertools

import numpy as np

import graphgen


def graph_from_triples(n, triples):
    """CSR from undirected [u, v, w] triples (rows in ascending neighbour id)."""
    rows = [[] for _ in range(n)]
    for u, v, w in triples:
        rows[u].append((v, w)); rows[v].append((u, w))
    xadj = [0]; adj = []; ew = []
    for r in rows:
        for v, w in sorted(r):
            adj.append(v); ew.append(w)
        xadj.append(len(adj))
    return graphgen.Graph(n, np.array(xadj, np.int64), np.array(adj, np.int32),
                          np.ones(n, np.int32), np.array(ew, np.int32), "triples")


def dense_adjacency(g):
    A = np.zeros((g.n, g.n), np.int64)
    for v in range(g.n):
        for j in range(g.xadj[v], g.xadj[v + 1]):
            A[v, g.adjncy[j]] += g.adjwgt[j]
    return A


def brute_force_best(g, k, L):
    """Minimum cut over all k^n assignments with every part weight <= L
    (numpy enumeration; tiny graphs only).  Returns (cut, assignment)."""
    n = g.n
    A = dense_adjacency(g)
    iu = np.triu_indices(n, 1)
    w = A[iu]
    nz = w > 0
    eu, ev, ewt = iu[0][nz], iu[1][nz], w[nz]
    vw = np.asarray(g.vwgt, np.int64)
    best = None
    # enumerate in chunks
    digits = np.array(list(itertools.product(range(k), repeat=n)), dtype=np.int32)
    pw = np.zeros((len(digits), k), np.int64)
    for p in range(k):
        pw[:, p] = ((digits == p) * vw[None, :]).sum(1)
    ok = pw.max(1) <= L
    cuts = ((digits[:, eu] != digits[:, ev]) * ewt[None, :]).sum(1)
    cuts = np.where(ok, cuts, np.iinfo(np.int64).max)
    i = int(np.argmin(cuts))
    best = (int(cuts[i]), digits[i]) if ok.any() else (None, None)
    return best
