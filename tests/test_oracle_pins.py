"""Pins for the oracle: each test checks it against something other than
itself — closed forms, hand-derived fixtures (tests/golden), brute force on
tiny graphs, a library routine the definition reduces to, or an invariant the
paper states.  CPU only."""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle
from helpers import brute_force_best, dense_adjacency, graph_from_triples

NONE = oracle.NONE


# --------------------------------------------------------------------------
# counter-based hash: published test vectors of SplitMix64 (seed 0 outputs)
# --------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    gold = 0x9E3779B97F4A7C15
    # SplitMix64 seeded with 0: first outputs
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(gold) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64((2 * gold) & (2**64 - 1)) == 0x06C45D188009454F


# --------------------------------------------------------------------------
# Sec. 2.1: cost and balance
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nx,ny,strips", [(8, 6, 2), (16, 4, 4), (64, 64, 8)])
def test_cut_grid_strips_closed_form(nx, ny, strips):
    # vertical strips of a 5-point grid cut (strips - 1) * ny unit edges
    g = graphgen.grid2d(nx, ny)
    x = np.arange(g.n) % nx
    part = (x * strips // nx).astype(np.int32)
    assert oracle.cut(g, part) == (strips - 1) * ny
    pw = oracle.part_weights(g, part, strips)
    assert pw.sum() == g.n and (pw == nx // strips * ny).all()


def test_cut_special_cases():
    g = graphgen.grid3d(5, 4, 3, vw=(1, 4), ew=(1, 10), seed=7)
    # k = 1: nothing is cut
    assert oracle.cut(g, np.zeros(g.n, np.int32)) == 0
    # every vertex alone: every edge is cut -> half the CSR weight sum
    assert oracle.cut(g, np.arange(g.n, dtype=np.int32)) == int(g.adjwgt.astype(np.int64).sum()) // 2
    # edgeless graph
    e = graphgen.Graph(5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.ones(5, np.int32), np.zeros(0, np.int32))
    assert oracle.cut(e, np.arange(5, dtype=np.int32)) == 0
    # relabelling parts changes nothing
    rng = np.random.default_rng(3)
    part = rng.integers(0, 6, g.n).astype(np.int32)
    perm = rng.permutation(6).astype(np.int32)
    assert oracle.cut(g, part) == oracle.cut(g, perm[part])


def test_cut_matches_dense_quadratic_form():
    # cut = sum_{u<v} A_uv [P(u) != P(v)] computed with a dense matrix product
    g = graphgen.gnp(30, 0.2, seed=5, ew=(1, 9))
    rng = np.random.default_rng(1)
    part = rng.integers(0, 4, g.n).astype(np.int32)
    A = dense_adjacency(g)
    S = np.eye(4, dtype=np.int64)[part]           # n x k indicator
    internal = np.trace(S.T @ A @ S) // 2
    total = A.sum() // 2
    assert oracle.cut(g, part) == total - internal


@pytest.mark.parametrize("W,k,eps,L,opt", [
    (4096, 8, 0.03, 527, 512),      # 64x64 grid, k = 8
    (100, 3, 0.03, 35, 34),         # 34 * 1.03 = 35.02
    (10, 3, 0.03, 4, 4),            # 4 * 1.03 = 4.12
    (1000, 10, 0.0, 100, 100),      # no slack
    (5242880, 64, 0.03, 84377, 81920),  # 81920 * 1.03 = 84377.6
    (7, 7, 0.5, 1, 1),
])
def test_balance_limit_closed_form(W, k, eps, L, opt):
    assert oracle.limit(W, k, eps) == (L, opt)


def test_sigma_dead_zone():
    for opt, L in [(512, 527), (4, 4), (81920, 84377), (10, 11)]:
        s = oracle.sigma(opt, L)
        assert opt <= s <= L
        assert s == opt + (L - opt) // 2
        if L > opt:
            assert s < L  # a non-empty dead zone (sigma, L]


def test_slot_definition_values():
    # slot(x) = 0 (x < 0), 1 (x = 0), 2 + floor(log2 x) (x > 0), Sec. 4.2.1
    cases = {-7: 0, -1: 0, 0: 1, 1: 2, 2: 3, 3: 3, 4: 4, 7: 4, 8: 5, 1023: 11, 1024: 12, 2**31 - 1: 32}
    for x, s in cases.items():
        assert oracle.slot(x) == s, x


# --------------------------------------------------------------------------
# Alg. 4: Jetlp on hand-derived cases
# --------------------------------------------------------------------------

def _load_json(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def test_jetlp_hand_cases(golden_dir):
    data = _load_json(golden_dir, "jetlp_cases.json")
    for case in data["cases"]:
        g = graph_from_triples(case["n"], case["edges"])
        r = oracle.jetlp(g, case["k"], case["part"], case["locked"], c=case["c"])
        assert r["Pd"].tolist() == case["Pd"], case["name"]
        F = [None if f == NONE else int(f) for f in r["F"]]
        assert F == case["F"], case["name"]
        assert np.flatnonzero(r["inX"]).tolist() == case["X"], case["name"]
        for v, f2 in case["F2"].items():
            assert int(r["F2"][int(v)]) == f2, (case["name"], v)
        assert np.flatnonzero(r["inM"]).tolist() == case["M"], case["name"]


def test_jetlp_properties_random():
    # Definition-level properties on random weighted graphs: P_d is adjacent
    # with maximal connectivity, F is the stated difference, X obeys the
    # first filter, M is a subset of X, locked vertices never enter X.
    for seed in range(5):
        g = graphgen.gnp(60, 0.08, seed=seed, ew=(1, 6))
        rng = np.random.default_rng(seed)
        k = 5
        part = rng.integers(0, k, g.n).astype(np.int32)
        locked = (rng.random(g.n) < 0.2).astype(np.uint8)
        r = oracle.jetlp(g, k, part, locked, c=0.25)
        A = dense_adjacency(g)
        S = np.eye(k, dtype=np.int64)[part]
        conn = A @ S  # conn[v, p]
        for v in range(g.n):
            others = [p for p in range(k) if p != part[v] and conn[v, p] > 0]
            if locked[v] or not others:
                assert r["F"][v] == NONE and r["Pd"][v] == part[v] and not r["inX"][v]
                continue
            best = max(conn[v, p] for p in others)
            assert r["Pd"][v] == min(p for p in others if conn[v, p] == best)
            assert r["F"][v] == best - conn[v, part[v]]
            F = int(r["F"][v])
            assert bool(r["inX"][v]) == (F >= 0 or -F < conn[v, part[v]] // 4)
        assert not (r["inM"] & ~r["inX"]).any()


# --------------------------------------------------------------------------
# Alg. 5 / Sec. 4.2.2: rebalancing on hand-derived cases
# --------------------------------------------------------------------------

def test_rebalance_hand_cases(golden_dir):
    data = _load_json(golden_dir, "rebalance_cases.json")
    for case in data["cases"]:
        g = graph_from_triples(case["n"], case["edges"])
        g.vwgt = np.asarray(case["vwgt"], np.int32)
        k, eps = case["k"], case["eps"]
        if case["kind"] == "rw":
            r = oracle.jetrw(g, k, case["part"], eps=eps, seed=1, it=0)
        else:
            r = oracle.jetrs(g, k, case["part"], eps=eps)
        assert (r["L"], r["opt"], r["sigma"]) == (case["L"], case["opt"], case["sigma"]), case["name"]
        for v, lo in case["loss"].items():
            assert int(r["loss"][int(v)]) == lo, (case["name"], v)
        for v, s in case.get("slot", {}).items():
            assert oracle.slot(int(r["loss"][int(v)])) == s
        assert r["dest"].tolist() == case["dest"], case["name"]
        newp = np.where(r["dest"] >= 0, r["dest"], np.asarray(case["part"])).astype(np.int32)
        assert oracle.part_weights(g, newp, k).tolist() == case["part_weights_after"], case["name"]


def _unbalanced_start(g, k, heavy=0.6, seed=0):
    rng = np.random.default_rng(seed)
    part = rng.integers(1, k, g.n).astype(np.int32) if k > 1 else np.zeros(g.n, np.int32)
    part[rng.random(g.n) < heavy] = 0
    return part


def test_jetrw_random_destination_in_B():
    # a vertex with no adjacent part of B goes to some part of B (randomPart(B))
    g = graphgen.grid2d(12, 12)
    k = 4
    part = np.zeros(g.n, np.int32)
    part[-10:] = 1; part[-5:] = 2
    r = oracle.jetrw(g, k, part, eps=0.03, seed=9, it=3)
    B = {p for p in range(k) if r["pw"][p] <= r["sigma"]}
    moved = np.flatnonzero(r["dest"] >= 0)
    assert len(moved) > 0
    assert all(int(r["dest"][v]) in B for v in moved)
    # exclusive-prefix eviction: part 0 drops to at most L (unit weights: exactly L)
    newp = np.where(r["dest"] >= 0, r["dest"], part)
    assert oracle.part_weights(g, newp, k)[0] == r["L"]


def test_theorem1_bucket_prefix_within_factor_two():
    # Theorem 1 (Sec. 4.2.1): k = 2, unit weights, no negative losses:
    # loss(L'_x) <= 2 loss(L_x), L_x the exact smallest-loss prefix of equal size.
    checked = 0
    for seed in range(40):
        g = graphgen.gnp(80, 0.2, seed=seed, ew=(1, 4))
        rng = np.random.default_rng(seed)
        part = (rng.random(g.n) < 0.2).astype(np.int32)  # part 0 (~80%) oversized
        r = oracle.jetrw(g, 2, part, eps=0.03, seed=1, it=0)
        cand = r["loss"] != NONE
        if not cand.any() or r["loss"][cand].min() < 0:
            continue
        taken = r["dest"] >= 0
        nt = int(taken.sum())
        assert nt == r["pw"][0] - r["L"]  # |L'_x| equals the excess
        exact = np.sort(r["loss"][cand])[:nt].sum()
        assert r["loss"][taken].sum() <= 2 * exact
        checked += 1
    assert checked >= 10


def test_jetrw_balances_within_k_iterations_unit_weights():
    # Sec. 4.2.2: at most k Jetrw iterations with uniform vertex weights
    o = oracle.Options(weak_limit=10**6, max_no_improve=10**6, max_iters=200)
    for seed, (g, k) in enumerate([(graphgen.grid2d(30, 30), 8), (graphgen.gnp(200, 0.03, seed=2), 6),
                                   (graphgen.rgg(2000, seed=3), 16)]):
        part = _unbalanced_start(g, k, seed=seed)
        r = oracle.refine(g, k, part, eps=0.03, is_finest=True, seed=5, opts=o, trace_cap=200)
        kinds, maxw = r.trace["kind"], r.trace["maxw"]
        L, _ = oracle.limit(g.n, k, 0.03)
        first_bal = int(np.argmax(maxw <= L))
        assert maxw[first_bal] <= L
        assert (kinds[:first_bal + 1] == oracle.KIND_RW).all()
        assert first_bal + 1 <= k


def test_jetrs_balances_in_one_iteration_unit_weights():
    # Sec. 4.2.2: Jetrs leaves no oversized part after one iteration (unit weights)
    o = oracle.Options(weak_limit=0)
    for seed, (g, k) in enumerate([(graphgen.grid2d(40, 25), 8), (graphgen.gnp(300, 0.02, seed=4), 5),
                                   (graphgen.rmat(10, seed=2), 16)]):
        part = _unbalanced_start(g, k, heavy=0.8, seed=seed)
        r = oracle.refine(g, k, part, eps=0.03, seed=3, opts=o, trace_cap=10)
        L, _ = oracle.limit(g.n, k, 0.03)
        assert r.trace["kind"][0] == oracle.KIND_RS
        assert r.trace["maxw"][0] <= L


# --------------------------------------------------------------------------
# Alg. 3: the driver
# --------------------------------------------------------------------------

def test_driver_composes_passes_and_keeps_locks_through_rebalancing():
    # Rebuild the first iterations of refine() from the single-pass functions:
    # Jetlp moves lock their vertices (R := M); Jetrw/Jetrs neither read nor
    # change locks (Sec. 4.1.3), so the next Jetlp still sees the old R.
    g = graphgen.grid2d(24, 24, ew=(1, 5), seed=3)
    k, eps = 4, 0.03
    o = oracle.Options(max_no_improve=10**6, max_iters=25)
    part0 = oracle.initial_partition(g, k)
    r = oracle.refine(g, k, part0, eps=eps, is_finest=True, seed=11, opts=o, trace_cap=25)
    L, opt = oracle.limit(g.n, k, eps)
    P = part0.copy(); locked = np.zeros(g.n, np.uint8); weak = 0
    for it in range(len(r.trace["kind"])):
        pw = oracle.part_weights(g, P, k)
        if pw.max() <= L:
            s = oracle.jetlp(g, k, P, locked, c=0.25)
            kind, nx = oracle.KIND_LP, int(s["inX"].sum())
            dest = np.where(s["inM"], s["Pd"], -1)
            locked = s["inM"].astype(np.uint8); weak = 0
        elif weak < 2:
            s = oracle.jetrw(g, k, P, eps=eps, seed=11, it=it); weak += 1
            kind, nx, dest = oracle.KIND_RW, s["ncand"], s["dest"]
        else:
            s = oracle.jetrs(g, k, P, eps=eps)
            kind, nx, dest = oracle.KIND_RS, s["ncand"], s["dest"]
        P = np.where(dest >= 0, dest, P).astype(np.int32)
        assert r.trace["kind"][it] == kind
        assert r.trace["nx"][it] == nx
        assert r.trace["nm"][it] == int((dest >= 0).sum())
        assert r.trace["cut"][it] == oracle.cut(g, P)
        assert r.trace["maxw"][it] == oracle.part_weights(g, P, k).max()
    # the trajectory must contain a Jetlp, a rebalancing pass and another
    # Jetlp, so that the carried-over locks were actually exercised
    kinds = r.trace["kind"].tolist()
    assert any(kinds[i] == oracle.KIND_LP and kinds[i + 1] != oracle.KIND_LP and kinds[i + 2] == oracle.KIND_LP
               for i in range(len(kinds) - 2))


def test_driver_returns_best_and_stops_after_12_without_improvement():
    for g, k in [(graphgen.grid2d(32, 32), 4), (graphgen.rgg(3000, seed=8), 8),
                 (graphgen.grid3d(10, 10, 10, vw=(1, 4), ew=(1, 10)), 8)]:
        part0 = oracle.initial_partition(g, k)
        r = oracle.refine(g, k, part0, eps=0.03, seed=2)
        L, _ = oracle.limit(int(g.vwgt.sum()), k, 0.03)
        cuts, maxw = r.trace["cut"], r.trace["maxw"]
        c0 = oracle.cut(g, part0)
        bal0 = oracle.part_weights(g, part0, k).max() <= L
        cand = [c0] if bal0 else []
        cand += [int(c) for c, w in zip(cuts, maxw) if w <= L]
        assert r.status == 0 and cand
        assert r.cut == min(cand)                      # P_best is the best balanced state
        assert r.cut == oracle.cut(g, r.part)
        assert oracle.part_weights(g, r.part, k).max() <= L
        if bal0:
            assert r.cut <= c0                         # never worse than the input
        # stopping rule: the last 12 iterations brought no phi-improvement
        best = c0 if bal0 else None
        last_reset = -1
        for i, (c, w) in enumerate(zip(cuts, maxw)):
            if w <= L and (best is None or c < best):
                if best is None or 1000000 * c < 999000 * best:
                    last_reset = i
                best = c
        assert r.iters == last_reset + 1 + 12


def test_refine_k1_and_edgeless():
    g = graphgen.grid2d(10, 10)
    r = oracle.refine(g, 1, np.zeros(g.n, np.int32), eps=0.03)
    assert r.cut == 0 and r.iters == 12 and r.status == 0
    e = graphgen.Graph(8, np.zeros(9, np.int64), np.zeros(0, np.int32), np.ones(8, np.int32), np.zeros(0, np.int32))
    r = oracle.refine(e, 4, np.zeros(8, np.int32), eps=0.03)
    assert r.cut == 0 and oracle.part_weights(e, r.part, 4).max() <= 2


# --------------------------------------------------------------------------
# Sec. 3.1 / Alg. 2: matching, mapping, contraction, projection
# --------------------------------------------------------------------------

def test_hem_validity_and_maximality():
    for seed, g in enumerate([graphgen.grid2d(20, 20, ew=(1, 10), seed=1), graphgen.rmat(10, seed=4),
                              graphgen.rgg(2000, seed=5, ew=(1, 3))]):
        mate = oracle.hem(g, seed=seed, rounds=64)
        for v in range(g.n):
            u = mate[v]
            if u >= 0:
                assert mate[u] == v and u != v
                assert u in g.adjncy[g.xadj[v]:g.xadj[v + 1]]
        # after convergence no edge joins two unmatched vertices (maximal)
        for v in np.flatnonzero(mate < 0):
            assert (mate[g.adjncy[g.xadj[v]:g.xadj[v + 1]]] >= 0).all()


def test_hem_heavy_edges_on_weighted_path():
    # path 0-1-2-3-4-5 with weights 1,5,2,6,3: locally heaviest edges 1-2 and
    # 3-4 match in the first round; 0 and 5 then have no unmatched neighbour.
    g = graph_from_triples(6, [[0, 1, 1], [1, 2, 5], [2, 3, 2], [3, 4, 6], [4, 5, 3]])
    assert oracle.hem(g, seed=1).tolist() == [-1, 2, 1, 4, 3, -1]


def _splitmix64_ref(x):
    """SplitMix64 (Steele, Lea, Flood 2014) written out here, independently of
    the oracle's C version; checked against the published seed-0 outputs."""
    M = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_splitmix64_reference_matches_published_vectors():
    assert _splitmix64_ref(0) == 0xE220A8397B1DCDAF
    assert _splitmix64_ref(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_hem_equal_weight_tie_break_by_hash():
    # Vertex 0 has two unmatched neighbours 1 and 2 over edges of equal
    # weight; 1 and 2 only see 0.  Reading 14: the proposal goes to the
    # neighbour with the smaller splitmix64(seed ^ salt(level, round) ^ u),
    # salt = 0xD1B54A32D192ED03 * (64 level + r + 1), then to the smaller id.
    # Seeds are chosen so that the hash picks 2 (against the id order) for
    # some and 1 for others: a dropped hash or a reversed comparison fails.
    g = graph_from_triples(3, [[0, 1, 4], [0, 2, 4]])
    M = (1 << 64) - 1
    seen = set()
    for seed in range(1, 40):
        for level in (0, 3):
            salt = (0xD1B54A32D192ED03 * (64 * level + 0 + 1)) & M
            h1 = _splitmix64_ref(seed ^ salt ^ 1)
            h2 = _splitmix64_ref(seed ^ salt ^ 2)
            want = 1 if h1 < h2 else 2
            other = 3 - want
            seen.add(want)
            exp = [-1, -1, -1]
            exp[0], exp[want] = want, 0
            assert oracle.hem(g, seed=seed, level=level).tolist() == exp
            # a heavier edge overrides the hash
            gh = graph_from_triples(3, [[0, want, 4], [0, other, 5]])
            mate = oracle.hem(gh, seed=seed, level=level)
            assert mate[0] == other and mate[other] == 0 and mate[want] == -1
    assert seen == {1, 2}


def test_coarse_map_numbering_by_smaller_id():
    # Reading (mapping): a pair is represented by its smaller id, singletons by
    # themselves; coarse ids are the ranks of the representatives in id order.
    # pairs {0,3}, {2,4}; singletons 1, 5 -> representatives 0, 1, 2, 5
    cmap, nc = oracle.coarse_map(np.array([3, -1, 4, 0, 2, -1], np.int32))
    assert nc == 4 and cmap.tolist() == [0, 1, 2, 0, 2, 3]
    # pairs {1,5}, {0,2}, {3,4}: representatives 0, 1, 3
    cmap, nc = oracle.coarse_map(np.array([2, 5, 0, 4, 3, 1], np.int32))
    assert nc == 3 and cmap.tolist() == [0, 1, 0, 2, 2, 1]


def test_contraction_hand_case():
    # 4-cycle 0-1-2-3-0 with weights 1,2,3,4 plus chord 0-2 (5); vwgt 1..4.
    # Matching {0,1}, {2,3}: coarse 0 = {0,1}, coarse 1 = {2,3}; the edges
    # 1-2 (2) and 3-0 (4) and the chord 0-2 (5) join them: weight 11; the
    # internal edges 0-1 and 2-3 disappear (no self-loops).
    g = graph_from_triples(4, [[0, 1, 1], [1, 2, 2], [2, 3, 3], [3, 0, 4], [0, 2, 5]])
    g.vwgt = np.array([1, 2, 3, 4], np.int32)
    cmap, nc = oracle.coarse_map(np.array([1, 0, 3, 2], np.int32))
    assert nc == 2 and cmap.tolist() == [0, 0, 1, 1]
    cg = oracle.contract(g, cmap, nc)
    assert cg.xadj.tolist() == [0, 1, 2]
    assert cg.adjncy.tolist() == [1, 0] and cg.adjwgt.tolist() == [11, 11]
    assert cg.vwgt.tolist() == [3, 7]


def test_contraction_equals_dense_triple_product():
    # coarse adjacency = C^T A C without its diagonal (Alg. 2), rows sorted
    for seed, g in enumerate([graphgen.grid2d(9, 7, ew=(1, 10), seed=2), graphgen.gnp(40, 0.15, seed=3, ew=(1, 5)),
                              graphgen.rmat(8, seed=1)]):
        mate = oracle.hem(g, seed=seed)
        cmap, nc = oracle.coarse_map(mate)
        assert nc == g.n - int((mate >= 0).sum()) // 2
        cg = oracle.contract(g, cmap, nc)
        Cm = np.zeros((g.n, nc), np.int64); Cm[np.arange(g.n), cmap] = 1
        Ac = Cm.T @ dense_adjacency(g) @ Cm
        np.fill_diagonal(Ac, 0)
        assert (dense_adjacency(cg) == Ac).all()
        for c in range(nc):
            row = cg.adjncy[cg.xadj[c]:cg.xadj[c + 1]]
            assert (np.diff(row) > 0).all()
        assert (cg.vwgt == Cm.T @ g.vwgt.astype(np.int64)).all()


def test_projection_preserves_cut_and_weights():
    g = graphgen.grid3d(8, 8, 8, vw=(1, 4), ew=(1, 10), seed=3)
    levels = oracle.coarsen(g, 4, seed=2, opts=oracle.Options(coarsen_target=20))
    assert len(levels) >= 3
    rng = np.random.default_rng(0)
    for i in range(len(levels) - 1):
        fine, coarse, cmap = levels[i].graph, levels[i + 1].graph, levels[i].cmap
        pc = rng.integers(0, 5, coarse.n).astype(np.int32)
        pf = pc[cmap]
        assert oracle.cut(fine, pf) == oracle.cut(coarse, pc)
        assert (oracle.part_weights(fine, pf, 5) == oracle.part_weights(coarse, pc, 5)).all()
    assert levels[-1].graph.n <= 20 or 100 * levels[-1].graph.n > 95 * levels[-2].graph.n


def test_coarsening_stops_at_target():
    g = graphgen.grid2d(64, 64)
    lv = oracle.coarsen(g, 8, seed=1)
    T = oracle.coarsen_target(8)
    assert T == 256
    assert lv[-1].graph.n <= T < lv[-2].graph.n
    assert all(l.graph.vwgt.sum() == g.n for l in lv)


# --------------------------------------------------------------------------
# Initial partition (greedy graph growing)
# --------------------------------------------------------------------------

def test_initial_partition_path_closed_form():
    n, k = 37, 5
    g = graph_from_triples(n, [[i, i + 1, 1] for i in range(n - 1)])
    part = oracle.initial_partition(g, k)
    assert part.tolist() == [(k * i) // n for i in range(n)]


def test_initial_partition_hand_case():
    # 3x3 grid from vertex 0: levels {0}, {1,3}, {2,4,6}, {5,7}, {8};
    # order 0,1,3,2,4,6,5,7,8 and P = floor(2 S / 9) for k = 2
    g = graphgen.grid2d(3, 3)
    part = oracle.initial_partition(g, 2)
    order = [0, 1, 3, 2, 4, 6, 5, 7, 8]
    exp = np.zeros(9, np.int32)
    for s, v in enumerate(order):
        exp[v] = (2 * s) // 9
    assert part.tolist() == exp.tolist()
    # two components: the one holding the lowest id comes first
    u = graphgen.disjoint_union(graphgen.grid2d(2, 2), graphgen.grid2d(2, 2))
    assert oracle.initial_partition(u, 2).tolist() == [0, 0, 0, 0, 1, 1, 1, 1]


# --------------------------------------------------------------------------
# Alg. 1: whole pipeline against brute force
# --------------------------------------------------------------------------

def test_partition_vs_brute_force_tiny():
    rng = np.random.default_rng(7)
    checked = 0
    for seed in range(12):
        n = int(rng.integers(6, 10))
        g = graphgen.gnp(n, 0.4, seed=seed, ew=(1, 4))
        for k in (2, 3):
            L, _ = oracle.limit(g.n, k, 0.03)
            best, _ = brute_force_best(g, k, L)
            r = oracle.partition(g, k, 0.03, seed=seed)
            pw = oracle.part_weights(g, r.part, k)
            if best is None:
                continue
            assert r.status == 0 and pw.max() <= L
            cut_np = sum(int(g.adjwgt[j]) for v in range(g.n) for j in range(g.xadj[v], g.xadj[v + 1])
                         if r.part[g.adjncy[j]] != r.part[v]) // 2
            assert r.cut == cut_np >= best
            checked += 1
    assert checked >= 15


def test_partition_easy_instances_reach_optimum():
    # two K8 joined by one edge, k = 2: optimum 1 (brute force confirms)
    tri = []
    for base in (0, 8):
        tri += [[base + i, base + j, 1] for i in range(8) for j in range(i + 1, 8)]
    tri.append([0, 8, 1])
    g = graph_from_triples(16, tri)
    L, _ = oracle.limit(16, 2, 0.03)
    assert brute_force_best(g, 2, L)[0] == 1
    assert oracle.partition(g, 2, 0.03, seed=1).cut == 1
    # four disjoint 4-cycles, k = 4: optimum 0
    c4 = graph_from_triples(4, [[0, 1, 1], [1, 2, 1], [2, 3, 1], [3, 0, 1]])
    u = graphgen.disjoint_union(c4, c4, c4, c4)
    r = oracle.partition(u, 4, 0.0, seed=1)
    assert r.cut == 0 and (oracle.part_weights(u, r.part, 4) == 4).all()


def test_partition_grid_g1_balanced_and_deterministic():
    g = graphgen.grid2d(64, 64)
    a = oracle.partition(g, 8, 0.03, seed=1)
    b = oracle.partition(g, 8, 0.03, seed=1)
    assert (a.part == b.part).all() and a.cut == b.cut
    L, _ = oracle.limit(g.n, 8, 0.03)
    assert a.status == 0 and oracle.part_weights(g, a.part, 8).max() <= L
    assert a.cut == oracle.cut(g, a.part)
    # a 64x64 grid cut into 8 parts needs at least 4 * 64 - ... ; sanity bounds
    assert 200 <= a.cut <= 64 * 7
