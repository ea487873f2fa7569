"""Pins of the oracle's two-hop matching (Sec. 3.1: leaves, twins and
relatives, added after heavy-edge matching when more than 25% of the
vertices are unmatched).  Hand-derived cases plus invariants checked from the
definitions with plain set operations (never through the oracle's hash)."""
import numpy as np
import pytest

import graphgen
import oracle
from helpers import graph_from_triples


def _nbrs(g, v):
    return set(int(u) for u in g.adjncy[g.xadj[v]:g.xadj[v + 1]])


def _deg(g, v):
    return int(g.xadj[v + 1] - g.xadj[v])


def _check_invariants(g, mate0, mate1, added):
    """Every two-hop pair is a leaf pair, a twin pair or a relative pair;
    heavy-edge pairs are untouched; each stage leaves at most one vertex of
    each of its groups unmatched; the 25% trigger holds."""
    n = g.n
    assert ((mate1 < 0) | (mate1[np.maximum(mate1, 0)] == np.arange(n))).all()     # symmetric
    kept = mate0 >= 0
    assert (mate1[kept] == mate0[kept]).all()
    new = [(v, int(mate1[v])) for v in range(n) if mate0[v] < 0 and mate1[v] > v]
    assert 2 * len(new) == sum(added)
    for a, b in new:
        na, nb = _nbrs(g, a), _nbrs(g, b)
        leaf = _deg(g, a) == 1 and _deg(g, b) == 1 and na == nb
        twin = na == nb
        rel = len(na & nb) > 0
        assert leaf or twin or rel, (a, b)
    if 4 * int((mate0 < 0).sum()) <= n:
        assert added == [0, 0, 0]


def test_star_leaves_pair_in_ascending_id():
    # K_{1,5}: the centre matches one leaf x by heavy-edge matching; the other
    # four leaves share the centre and pair up in ascending id
    g = graph_from_triples(6, [[0, i, 1] for i in range(1, 6)])
    m0 = oracle.hem(g, 1, 0, 8)
    x = int(m0[0])
    assert x in range(1, 6) and int((m0 >= 0).sum()) == 2
    m1, added = oracle.two_hop(g, m0)
    rest = [v for v in range(1, 6) if v != x]
    assert added == [4, 0, 0]
    assert m1[rest[0]] == rest[1] and m1[rest[2]] == rest[3]


def test_bipartite_twins():
    # K_{2,4}: right vertices all see {0, 1}; after heavy-edge matching two
    # of them are left, and they are twins
    g = graph_from_triples(6, [[a, b, 1] for a in (0, 1) for b in range(2, 6)])
    m0 = oracle.hem(g, 3, 0, 8)
    un = [v for v in range(6) if m0[v] < 0]
    assert len(un) == 2 and all(v >= 2 for v in un)
    m1, added = oracle.two_hop(g, m0)
    assert added == [0, 2, 0] and m1[un[0]] == un[1]


def test_relatives_through_lowest_matchmaker():
    # heavy edges force 0-1, 5-6, 7-8, 9-10; vertices 2, 3, 4 hang off 0 and
    # one heavy-matched vertex each: no leaves, no twins ({0,5} {0,7} {0,9});
    # their lowest matched neighbour is 0, so 2-3 pair and 4 stays alone
    t = [[0, 1, 10], [5, 6, 10], [7, 8, 10], [9, 10, 10],
         [0, 2, 1], [0, 3, 1], [0, 4, 1], [2, 5, 1], [3, 7, 1], [4, 9, 1]]
    g = graph_from_triples(11, t)
    m0 = oracle.hem(g, 1, 0, 8)
    assert [int(m0[v]) for v in (0, 5, 7, 9)] == [1, 6, 8, 10] and all(m0[v] < 0 for v in (2, 3, 4))
    m1, added = oracle.two_hop(g, m0)
    assert added == [0, 0, 2]
    assert m1[2] == 3 and m1[3] == 2 and m1[4] < 0


def test_high_degree_vertices_are_not_matchmakers():
    # two vertices reachable only through a matched hub of degree > 1024
    # (the hub's other neighbours are leaves matched among themselves first
    # would be leaves, so give them a second hub to keep them out)
    d = oracle.MATCHMAKER_MAX_DEG + 10
    hub, mate_h = 0, 1
    t = [[hub, mate_h, 100]]
    nxt = 2
    for _ in range(d):
        t.append([hub, nxt, 1]); nxt += 1
    # the two candidates a, b: neighbours hub and a private heavy-matched vertex each
    a, b, pa, qa, pb, qb = nxt, nxt + 1, nxt + 2, nxt + 3, nxt + 4, nxt + 5
    t += [[hub, a, 1], [hub, b, 1], [a, pa, 1], [pa, qa, 50], [b, pb, 1], [pb, qb, 50]]
    g = graph_from_triples(qb + 1, t)
    m0 = oracle.hem(g, 1, 0, 8)
    m1, added = oracle.two_hop(g, m0)
    # a's lowest matched neighbour of small degree is pa, b's is pb: different groups
    assert m1[a] < 0 or m1[a] != b


def test_isolated_vertices_are_twins():
    g = graphgen.Graph(7, np.zeros(8, np.int64), np.zeros(0, np.int32), None, None)
    m1, added = oracle.two_hop(g, np.full(7, -1, np.int32))
    assert added == [0, 6, 0]
    assert list(m1[:6]) == [1, 0, 3, 2, 5, 4] and m1[6] == -1


def test_no_two_hop_when_at_most_a_quarter_unmatched():
    g = graphgen.grid2d(20, 20)
    m0 = oracle.hem(g, 1, 0, 8)
    assert 4 * int((m0 < 0).sum()) <= g.n
    m1, added = oracle.two_hop(g, m0)
    assert added == [0, 0, 0] and (m1 == m0).all()


def test_twin_key_is_order_free_and_separates_neighbourhoods():
    # same neighbour set listed in two orders -> same key; different sets differ
    g1 = graphgen.Graph(4, np.array([0, 3, 4, 5, 6], np.int64), np.array([1, 2, 3, 0, 0, 0], np.int32), None, None)
    g2 = graphgen.Graph(4, np.array([0, 3, 4, 5, 6], np.int64), np.array([3, 1, 2, 0, 0, 0], np.int32), None, None)
    assert oracle.twin_key(g1, 0) == oracle.twin_key(g2, 0)
    assert oracle.twin_key(g1, 1) == oracle.twin_key(g1, 2)
    assert oracle.twin_key(g1, 0) != oracle.twin_key(g1, 1)


@pytest.mark.parametrize("g", [graphgen.rmat(12, seed=5), graphgen.rmat(11, seed=7, ew=(1, 5)),
                               graphgen.rgg(3000, seed=2), graphgen.gnp(400, 0.02, seed=3)],
                         ids=["rmat12", "rmat11w", "rgg3000", "gnp400"])
def test_invariants_on_generated_graphs(g):
    m0 = oracle.hem(g, 1, 0, 8)
    m1, added = oracle.two_hop(g, m0)
    _check_invariants(g, m0, m1, added)


def test_relatives_stage_pairs_share_their_matchmaker():
    g = graphgen.rmat(12, seed=9)
    m0 = oracle.hem(g, 1, 0, 8)
    # replay the first two stages, then check each relative pair against the
    # definition: same lowest matched neighbour of degree <= the cap
    m1, added = oracle.two_hop(g, m0)
    assert added[2] > 0
    before = m0.copy()
    # vertices matched by leaves/twins are exactly those pairs with equal neighbourhoods;
    # rebuild the state at the start of the relatives stage from that
    for v in range(g.n):
        if before[v] < 0 and m1[v] >= 0 and _nbrs(g, v) == _nbrs(g, int(m1[v])):
            before[v] = m1[v]
    for v in range(g.n):
        u = int(m1[v])
        if u > v and m0[v] < 0 and before[v] < 0:
            def mm(x):
                c = [w for w in _nbrs(g, x) if before[w] >= 0 and _deg(g, w) <= oracle.MATCHMAKER_MAX_DEG]
                return min(c) if c else None
            assert mm(v) is not None and mm(v) == mm(u)


def test_coarsening_of_power_law_graph_no_longer_stalls():
    g = graphgen.rmat(12, seed=5)
    with_th = [lv.graph.n for lv in oracle.coarsen(g, 8, 1, oracle.Options(flags=oracle.TWO_HOP))]
    without = [lv.graph.n for lv in oracle.coarsen(g, 8, 1)]
    assert with_th[-1] <= max(8 * 8, 256) < without[-1]
    # two-hop pairs merge vertices only: weight is preserved level by level
    lv = oracle.coarsen(g, 8, 1, oracle.Options(flags=oracle.TWO_HOP))
    assert all(int(l.graph.vwgt.sum()) == g.n for l in lv)
