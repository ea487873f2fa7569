"""GPU parity: every step of the CUDA path, called through the C ABI, against
the oracle on the same seeded inputs — bit-exact (all results are integers).
Sizes span several thread blocks, warp-path rows (> 16 entries) and ragged
tails; the full-size workloads are at the end."""
import json
import os

import numpy as np
import pytest
import torch

import graphgen
import oracle
from helpers import graph_from_triples

pytestmark = pytest.mark.gpu

jet = pytest.importorskip("paper_2304_13194_gb300")
NONE32 = -(2 ** 31)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = jet.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_hostloop():
    c = jet.Context(0, flags=jet.FLAG_HOSTLOOP)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_cluster():
    """Every level on the one-cluster loop."""
    c = jet.Context(0, cluster_max_n=1 << 30)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_graph():
    """Every level on the CUDA-graph loop (no thread-block-cluster loop)."""
    c = jet.Context(0, cluster_max_n=0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_grid():
    """Every level on the persistent loop (one cooperative launch per level)."""
    c = jet.Context(0, flags=jet.FLAG_GRID_LOOP, cluster_max_n=0)
    yield c
    c.close()


def _np(t):
    return t.cpu().numpy()


def _oracle_ablation(flags):
    """The oracle's switches for the library's Jetlp ablation flags."""
    return sum(o for f, o in [(jet.FLAG_NO_LOCKS, oracle.ABL_NO_LOCKS), (jet.FLAG_NO_AFTERBURN, oracle.ABL_NO_AFTERBURN),
                              (jet.FLAG_WEAK_AFTERBURN, oracle.ABL_WEAK_AFTERBURN),
                              (jet.FLAG_BASELINE_LP, oracle.ABL_BASELINE_LP),
                              (jet.FLAG_STRICT_GAIN, oracle.ABL_STRICT_GAIN)] if flags & f)


def _vw(g, unit):
    return None if unit else g.vwgt


def _ew(g, unit):
    return None if unit else g.adjwgt


def graphs_small():
    """Inputs shaped like the paper's workloads, small enough for the oracle."""
    star = graph_from_triples(301, [[0, i, 1 + i % 7] for i in range(1, 301)] +
                              [[i, i + 1, 2] for i in range(1, 300, 2)])
    return [
        ("grid2d_40x33", graphgen.grid2d(40, 33), True),
        ("grid3d_17x13x11_w", graphgen.grid3d(17, 13, 11, vw=(1, 4), ew=(1, 10), seed=3), False),
        ("rmat_s12", graphgen.rmat(12, seed=5), True),
        ("rmat_s11_w", graphgen.rmat(11, seed=7, vw=(1, 3), ew=(1, 5)), False),
        ("rgg_5000", graphgen.rgg(5000, seed=2), True),
        ("gnp_700_dense", graphgen.gnp(700, 0.06, seed=4, ew=(1, 9)), False),   # rows of ~42: warp path
        ("star_300", star, False),
    ]


# --------------------------------------------------------------------------
# single passes
# --------------------------------------------------------------------------

def test_lp_pass_hand_cases(ctx, golden_dir):
    data = json.load(open(os.path.join(golden_dir, "jetlp_cases.json")))
    for case in data["cases"]:
        g = graph_from_triples(case["n"], case["edges"])
        r = ctx.lp_pass(g.xadj, g.adjncy, g.vwgt, g.adjwgt, case["k"], np.array(case["part"], np.int32),
                        np.array(case["locked"], np.uint8), c=case["c"])
        assert _np(r["Pd"]).tolist() == case["Pd"], case["name"]
        F = [None if f == NONE32 else int(f) for f in _np(r["F"])]
        assert F == case["F"], case["name"]
        assert np.flatnonzero(_np(r["inX"])).tolist() == case["X"], case["name"]
        for v, f2 in case["F2"].items():
            assert int(_np(r["F2"])[int(v)]) == f2
        assert np.flatnonzero(_np(r["inM"])).tolist() == case["M"], case["name"]


@pytest.mark.parametrize("name,g,unit", graphs_small(), ids=[x[0] for x in graphs_small()])
@pytest.mark.parametrize("k,c,abl", [(8, 0.25, 0), (64, 0.75, 0), (5, 0.25, jet.FLAG_NO_AFTERBURN),
                                     (16, 0.25, jet.FLAG_WEAK_AFTERBURN), (16, 0.25, jet.FLAG_BASELINE_LP),
                                     (16, 0.75, jet.FLAG_STRICT_GAIN | jet.FLAG_NO_AFTERBURN)])
def test_lp_pass_random(ctx, name, g, unit, k, c, abl):
    rng = np.random.default_rng(k + abl)
    part = oracle.initial_partition(g, k)
    noise = rng.random(g.n) < 0.1
    part[noise] = rng.integers(0, k, int(noise.sum()))
    locked = (rng.random(g.n) < 0.15).astype(np.uint8)
    vw, ew = _vw(g, unit), _ew(g, unit)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, ew)
    oabl = _oracle_ablation(abl)
    ref = oracle.jetlp(og, k, part, locked, c=c, ablation=oabl)
    r = ctx.lp_pass(g.xadj, g.adjncy, vw, ew, k, part, locked, c=c, flags=abl)
    F = _np(r["F"]).astype(np.int64)
    refF = np.where(ref["F"] == oracle.NONE, NONE32, ref["F"])
    assert (F == refF).all()
    assert (_np(r["Pd"]) == ref["Pd"]).all()
    assert (_np(r["inX"]) == ref["inX"]).all()
    inX = ref["inX"]
    if not abl & (jet.FLAG_NO_AFTERBURN | jet.FLAG_BASELINE_LP):
        assert (_np(r["F2"])[inX] == ref["F2"][inX]).all()
    assert (_np(r["inM"]) == ref["inM"]).all()


def test_rebalance_hand_cases(ctx, golden_dir):
    data = json.load(open(os.path.join(golden_dir, "rebalance_cases.json")))
    for case in data["cases"]:
        g = graph_from_triples(case["n"], case["edges"])
        vw = np.array(case["vwgt"], np.int32)
        r = ctx.rebalance_pass(g.xadj, g.adjncy, vw, g.adjwgt, case["k"], np.array(case["part"], np.int32),
                               eps=case["eps"], strong=case["kind"] == "rs", seed=1, it=0)
        assert _np(r["dest"]).tolist() == case["dest"], case["name"]
        for v, lo in case["loss"].items():
            assert int(_np(r["loss"])[int(v)]) == lo, (case["name"], v)


@pytest.mark.parametrize("name,g,unit", graphs_small(), ids=[x[0] for x in graphs_small()])
@pytest.mark.parametrize("strong", [False, True])
def test_rebalance_pass_many_oversized_parts(ctx, name, g, unit, strong):
    """40 of 64 parts over the limit: more (part, slot) buckets than a block
    keeps in shared memory, so the slot weights are summed per warp and key
    (the warp-aggregated path), element by element against the oracle."""
    k = 64
    rng = np.random.default_rng(40)
    part = rng.integers(0, 40, g.n).astype(np.int32)
    vw, ew = _vw(g, unit), _ew(g, unit)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, ew)
    if strong:
        ref = oracle.jetrs(og, k, part, eps=0.03)
    else:
        ref = oracle.jetrw(og, k, part, eps=0.03, seed=17, it=5)
    r = ctx.rebalance_pass(g.xadj, g.adjncy, vw, ew, k, part, eps=0.03, strong=strong, seed=17, it=5)
    assert r["ncand"] == ref["ncand"]
    loss = _np(r["loss"]).astype(np.int64)
    refl = np.where(ref["loss"] == oracle.NONE, NONE32, ref["loss"])
    assert (loss == refl).all()
    assert (_np(r["dest"]) == ref["dest"]).all()
    assert r["nmoves"] == ref["nmoves"]


@pytest.mark.parametrize("name,g,unit", graphs_small(), ids=[x[0] for x in graphs_small()])
@pytest.mark.parametrize("k", [2, 7, 64])
@pytest.mark.parametrize("strong", [False, True])
def test_rebalance_pass_random(ctx, name, g, unit, k, strong):
    rng = np.random.default_rng(k)
    part = rng.integers(0, k, g.n).astype(np.int32)
    part[rng.random(g.n) < 0.3] = 0          # part 0 (and maybe others) oversized
    vw, ew = _vw(g, unit), _ew(g, unit)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, ew)
    if strong:
        ref = oracle.jetrs(og, k, part, eps=0.03)
    else:
        ref = oracle.jetrw(og, k, part, eps=0.03, seed=17, it=5)
    r = ctx.rebalance_pass(g.xadj, g.adjncy, vw, ew, k, part, eps=0.03, strong=strong, seed=17, it=5)
    assert r["ncand"] == ref["ncand"]
    loss = _np(r["loss"]).astype(np.int64)
    refl = np.where(ref["loss"] == oracle.NONE, NONE32, ref["loss"])
    assert (loss == refl).all()
    assert (_np(r["dest"]) == ref["dest"]).all()
    assert r["nmoves"] == ref["nmoves"]


@pytest.mark.parametrize("name,g,unit", graphs_small(), ids=[x[0] for x in graphs_small()])
def test_cut_and_weights(ctx, name, g, unit):
    k = 13
    part = np.random.default_rng(1).integers(0, k, g.n).astype(np.int32)
    vw, ew = _vw(g, unit), _ew(g, unit)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, ew)
    cut, pw = ctx.cut(g.xadj, g.adjncy, vw, ew, k, part)
    assert cut == oracle.cut(og, part)
    assert (_np(pw) == oracle.part_weights(og, part, k)).all()


@pytest.mark.parametrize("name,g,unit", graphs_small(), ids=[x[0] for x in graphs_small()])
def test_hem_matches_oracle(ctx, name, g, unit):
    ew = _ew(g, unit)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, None, ew)
    for level, rounds in [(0, 8), (3, 2), (1, 64)]:
        ref = oracle.hem(og, seed=9, level=level, rounds=rounds)
        got = _np(ctx.hem(g.xadj, g.adjncy, ew, seed=9, level=level, rounds=rounds))
        assert (got == ref).all()


@pytest.mark.parametrize("name,g,unit", graphs_small(), ids=[x[0] for x in graphs_small()])
def test_initial_partition_matches_oracle(ctx, name, g, unit):
    vw = _vw(g, unit)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, None)
    for k in (2, 8, 64):
        assert (_np(ctx.initial_partition(g.xadj, g.adjncy, vw, k)) == oracle.initial_partition(og, k)).all()


def _initpart_mix():
    """Many components of every kind: isolated vertices, a long path (more
    breadth-first levels than one batch of launches), a grid, an R-MAT graph
    with its own isolated vertices; ids interleaved by a permutation so that
    components are not contiguous; > 2 sort tiles and > 2 radix passes."""
    path = graphgen.from_edges(3000, [(i, i + 1) for i in range(2999)], vw=(1, 3), seed=2)
    iso = graphgen.Graph(500, np.zeros(501, np.int64), np.zeros(0, np.int32), np.full(500, 2, np.int32),
                         np.zeros(0, np.int32))
    u = graphgen.disjoint_union(path, iso, graphgen.grid2d(50, 40, vw=(1, 4)), graphgen.rmat(13, seed=3, vw=(1, 2)))
    perm = np.random.default_rng(7).permutation(u.n).astype(np.int64)
    src = np.repeat(np.arange(u.n, dtype=np.int64), np.diff(u.xadj))
    edges = np.stack([perm[src], perm[u.adjncy.astype(np.int64)]], 1)
    edges = edges[edges[:, 0] < edges[:, 1]]
    g = graphgen.from_edges(u.n, edges, seed=4)
    vw = np.empty(u.n, np.int32)
    vw[perm] = u.vwgt
    return graphgen.Graph(g.n, g.xadj, g.adjncy, vw, g.adjwgt, "initpart_mix")


def test_initial_partition_many_components_and_levels(ctx):
    g = _initpart_mix()
    for k in (3, 64, 1000):
        ref = oracle.initial_partition(g, k)
        assert (_np(ctx.initial_partition(g.xadj, g.adjncy, g.vwgt, k)) == ref).all()
    ref = oracle.initial_partition(graphgen.Graph(g.n, g.xadj, g.adjncy, None, None), 16)
    assert (_np(ctx.initial_partition(g.xadj, g.adjncy, None, 16)) == ref).all()


def _two_hop_graphs():
    iso = graphgen.Graph(301, np.zeros(302, np.int64), np.zeros(0, np.int32), np.ones(301, np.int32),
                         np.zeros(0, np.int32))
    star = graph_from_triples(200, [[0, i, 1] for i in range(1, 200)])
    return graphs_small() + [
        ("rmat_s14", graphgen.rmat(14, seed=11), True),
        ("isolated_301", iso, True),
        ("star_199", star, True),
        ("rmat_s12_plus_isolated", graphgen.disjoint_union(graphgen.rmat(12, seed=2), iso), True),
    ]


@pytest.mark.parametrize("name,g,unit", _two_hop_graphs(), ids=[x[0] for x in _two_hop_graphs()])
def test_two_hop_matches_oracle(ctx, name, g, unit):
    ew = _ew(g, unit)
    mate0 = _np(ctx.hem(g.xadj, g.adjncy, ew, seed=3, level=1))
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, None, ew)
    assert (mate0 == oracle.hem(og, 3, 1, 8)).all()
    ref, ref_added = oracle.two_hop(og, mate0)
    got, added = ctx.two_hop(g.xadj, g.adjncy, mate0)
    assert added == ref_added
    assert (_np(got) == ref).all()


@pytest.fixture(scope="module")
def ctx_two_hop():
    """Coarsening with two-hop matches (Sec. 3.1)."""
    c = jet.Context(0, flags=jet.FLAG_TWO_HOP)
    yield c
    c.close()


def test_coarsen_with_two_hop_matches_oracle(ctx_two_hop):
    g = graphgen.rmat(13, seed=4)
    h = ctx_two_hop.coarsen(g.xadj, g.adjncy, None, None, k=8, seed=2)
    ref = oracle.coarsen(graphgen.Graph(g.n, g.xadj, g.adjncy, None, None), 8, 2, oracle.Options(flags=oracle.TWO_HOP))
    try:
        lv, ns, ms = h.info()
        assert lv == len(ref) and list(ns) == [r.graph.n for r in ref]
        for i in range(lv - 1):
            assert (_np(h.level(i)["cmap"]) == ref[i].cmap).all()
    finally:
        h.close()


@pytest.mark.parametrize("name,g,unit,k", [
    ("rmat_s14", graphgen.rmat(14, seed=11), True, 64),
    ("rmat_s12_w", graphgen.rmat(12, seed=6, vw=(1, 3), ew=(1, 5)), False, 8),
    ("grid3d_24_w", graphgen.grid3d(24, 24, 24, vw=(1, 4), ew=(1, 10), seed=1), False, 64),
])
def test_partition_with_two_hop_matches_oracle(ctx_two_hop, name, g, unit, k):
    vw, ew = _vw(g, unit), _ew(g, unit)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, ew)
    ref = oracle.partition(og, k, 0.03, 2, oracle.Options(flags=oracle.TWO_HOP))
    part, cut, st = ctx_two_hop.partition(g.xadj, g.adjncy, vw, ew, k=k, eps=0.03, seed=2, return_stats=True)
    assert st.n == ref.stats["n"] and st.cut_level == ref.stats["cut_level"]
    assert cut == ref.cut and (_np(part) == ref.part).all()


@pytest.mark.parametrize("name,g,unit", graphs_small() + [("rmat_s16_hub_rows", graphgen.rmat(16, seed=5), True)],
                         ids=[x[0] for x in graphs_small()] + ["rmat_s16_hub_rows"])
def test_coarsen_hierarchy_matches_oracle(ctx, name, g, unit):
    """Every level's CSR, weights and map bit-exact with the oracle.  The
    R-MAT case merges rows of more than 4,096 entries (17 on its first level),
    which take the radix-sort path of the contraction."""
    vw, ew = _vw(g, unit), _ew(g, unit)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, ew)
    k = 8
    ref = oracle.coarsen(og, k, seed=3)
    h = ctx.coarsen(g.xadj, g.adjncy, vw, ew, k=k, seed=3)
    try:
        lv, ns, ms = h.info()
        assert lv == len(ref)
        for i in range(lv):
            L = h.level(i)
            R = ref[i].graph
            assert L["n"] == R.n
            assert (_np(L["xadj"]) == R.xadj).all()
            assert (_np(L["adjncy"]) == R.adjncy).all()
            assert (_np(L["vwgt"]) == R.vwgt).all()
            if i > 0 or ew is not None:
                assert (_np(L["adjwgt"]) == R.adjwgt).all()
            if i + 1 < lv:
                assert (_np(L["cmap"]) == ref[i].cmap).all()
    finally:
        h.close()


# --------------------------------------------------------------------------
# one level of refinement (Alg. 3): result and the whole trajectory
# --------------------------------------------------------------------------

def _check_refine(ctx, g, unit, k, part0, is_finest, seed, eps=0.03):
    vw, ew = _vw(g, unit), _ew(g, unit)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, ew)
    ref = oracle.refine(og, k, part0, eps=eps, is_finest=is_finest, seed=seed)
    p, cut = ctx.refine(g.xadj, g.adjncy, vw, ew, k, part0, eps=eps, is_finest=is_finest, seed=seed)
    tr = ctx.last_trace()
    assert tr["iters"] == ref.iters
    n = min(len(tr["kind"]), len(ref.trace["kind"]))
    for key in ("kind", "nx", "nm", "cut", "maxw"):
        assert (tr[key][:n] == ref.trace[key][:n]).all(), key
    assert cut == ref.cut
    assert (_np(p) == ref.part).all()


@pytest.mark.parametrize("name,g,unit", graphs_small(), ids=[x[0] for x in graphs_small()])
@pytest.mark.parametrize("k", [4, 64])
def test_refine_matches_oracle(ctx, name, g, unit, k):
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, _vw(g, unit), None)
    part0 = oracle.initial_partition(og, k)
    _check_refine(ctx, g, unit, k, part0, True, seed=5)
    _check_refine(ctx, g, unit, k, part0, False, seed=6)


def test_refine_hostloop_equals_graph_loop(ctx, ctx_hostloop):
    g = graphgen.grid3d(20, 20, 20, vw=(1, 4), ew=(1, 10), seed=9)
    part0 = oracle.initial_partition(g, 16)
    a = ctx.refine(g.xadj, g.adjncy, g.vwgt, g.adjwgt, 16, part0, seed=2)
    ta = ctx.last_trace()
    b = ctx_hostloop.refine(g.xadj, g.adjncy, g.vwgt, g.adjwgt, 16, part0, seed=2)
    tb = ctx_hostloop.last_trace()
    assert a[1] == b[1] and (_np(a[0]) == _np(b[0])).all()
    assert all((ta[key] == tb[key]).all() for key in ("kind", "nx", "nm", "cut", "maxw"))


@pytest.mark.parametrize("name,g,unit,k", [
    ("grid3d_20_w", graphgen.grid3d(20, 20, 20, vw=(1, 4), ew=(1, 10), seed=9), False, 16),
    ("rmat_s12", graphgen.rmat(12, seed=5), True, 64),                  # long rows: warp paths
    ("gnp_700_dense", graphgen.gnp(700, 0.06, seed=4, ew=(1, 9)), False, 8),
    ("rgg_30000", graphgen.rgg(30000, seed=3), True, 128),              # many 1024-vertex tiles
    ("rmat_s12_k256", graphgen.rmat(12, seed=5), True, 256),            # one block meets > 2048 X members
])
def test_refine_cluster_loop_equals_graph_loop(ctx_cluster, ctx_graph, name, g, unit, k):
    vw, ew = _vw(g, unit), _ew(g, unit)
    part0 = oracle.initial_partition(graphgen.Graph(g.n, g.xadj, g.adjncy, vw, None), k)
    for is_finest in (True, False):
        a = ctx_cluster.refine(g.xadj, g.adjncy, vw, ew, k, part0, seed=2, is_finest=is_finest)
        ta = ctx_cluster.last_trace()
        b = ctx_graph.refine(g.xadj, g.adjncy, vw, ew, k, part0, seed=2, is_finest=is_finest)
        tb = ctx_graph.last_trace()
        assert a[1] == b[1] and (_np(a[0]) == _np(b[0])).all()
        assert ta["iters"] == tb["iters"]
        assert all((ta[key] == tb[key]).all() for key in ("kind", "nx", "nm", "cut", "maxw"))


@pytest.mark.parametrize("name,g,unit,k", [
    ("grid3d_20_w", graphgen.grid3d(20, 20, 20, vw=(1, 4), ew=(1, 10), seed=9), False, 16),
    ("rmat_s12", graphgen.rmat(12, seed=5), True, 64),                  # long rows: warp paths
    ("gnp_700_dense", graphgen.gnp(700, 0.06, seed=4, ew=(1, 9)), False, 8),
    ("rgg_30000", graphgen.rgg(30000, seed=3), True, 128),              # many tiles per block
    ("rmat_s12_k256", graphgen.rmat(12, seed=5), True, 256),
    ("rmat_s14_hubs", graphgen.rmat(14, seed=2), True, 32),             # rows past 1024 entries: block rows
])
def test_refine_grid_loop_matches_oracle(ctx_grid, name, g, unit, k):
    """The persistent loop (grid barriers instead of kernel boundaries, the
    serial tails in the last block to arrive) follows the oracle's whole
    trajectory on finest and coarse settings."""
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, _vw(g, unit), None)
    part0 = oracle.initial_partition(og, k)
    _check_refine(ctx_grid, g, unit, k, part0, True, seed=5)
    _check_refine(ctx_grid, g, unit, k, part0, False, seed=6)


@pytest.mark.parametrize("name,g,unit", graphs_small()[1:4], ids=[x[0] for x in graphs_small()[1:4]])
def test_partition_grid_loop_matches_oracle(ctx_grid, name, g, unit):
    _check_partition(ctx_grid, g, unit, 64, seed=3)


def test_partition_grid_loop_mesh_k64(ctx_grid):
    """A 48^3 mesh at k = 64 on the persistent loop: Jetlp, Jetrw and Jetrs
    iterations on every level, bit-exact with the oracle."""
    g = graphgen.grid3d(48, 48, 48, vw=(1, 4), ew=(1, 10), seed=4)
    _check_partition(ctx_grid, g, False, 64, seed=2)


@pytest.mark.parametrize("blocks", [2, 4])
def test_small_clusters_equal_graph_loop(ctx_graph, blocks):
    """cluster_blocks caps the cluster (execution choice): fewer blocks take
    more 1024-vertex tiles each, with the same result."""
    with jet.Context(0, cluster_max_n=1 << 30, cluster_blocks=blocks) as c:
        for g, unit, k in ((graphgen.rgg(30000, seed=3), True, 128),
                           (graphgen.grid3d(20, 20, 20, vw=(1, 4), ew=(1, 10), seed=9), False, 16)):
            vw, ew = _vw(g, unit), _ew(g, unit)
            part0 = oracle.initial_partition(graphgen.Graph(g.n, g.xadj, g.adjncy, vw, None), k)
            a = c.refine(g.xadj, g.adjncy, vw, ew, k, part0, seed=2)
            b = ctx_graph.refine(g.xadj, g.adjncy, vw, ew, k, part0, seed=2)
            assert a[1] == b[1] and (_np(a[0]) == _np(b[0])).all()
        g = graphgen.grid3d(24, 24, 24, vw=(1, 4), ew=(1, 10), seed=1)
        _, cut, st = c.partition(g.xadj, g.adjncy, g.vwgt, g.adjwgt, k=64, seed=1, return_stats=True)
        assert all(b == blocks for b in st.cluster_blocks)
        assert cut == oracle.partition(g, 64, 0.03, 1).cut


def test_cluster_loop_is_used_on_small_levels(ctx, ctx_cluster, ctx_graph):
    g = graphgen.grid3d(24, 24, 24, vw=(1, 4), ew=(1, 10), seed=1)
    _, c1, st = ctx_cluster.partition(g.xadj, g.adjncy, g.vwgt, g.adjwgt, k=64, seed=1, return_stats=True)
    assert all(b >= 2 for b in st.cluster_blocks)
    _, c2, st2 = ctx_graph.partition(g.xadj, g.adjncy, g.vwgt, g.adjwgt, k=64, seed=1, return_stats=True)
    assert all(b == 0 for b in st2.cluster_blocks)
    assert st.kernel_launches < st2.kernel_launches and c1 == c2
    # default threshold: only the small levels take the cluster loop
    _, c3, st3 = ctx.partition(g.xadj, g.adjncy, g.vwgt, g.adjwgt, k=64, seed=1, return_stats=True)
    limit = ctx.options.cluster_max_n
    assert all((b > 0) == (nv <= limit) for b, nv in zip(st3.cluster_blocks, st3.n)) and c3 == c1


# --------------------------------------------------------------------------
# the whole pipeline (Alg. 1)
# --------------------------------------------------------------------------

def _check_partition(ctx, g, unit, k, eps=0.03, seed=1):
    vw, ew = _vw(g, unit), _ew(g, unit)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, ew)
    ref = oracle.partition(og, k, eps, seed)
    part, cut, st = ctx.partition(g.xadj, g.adjncy, vw, ew, k=k, eps=eps, seed=seed, return_stats=True)
    assert st.levels == ref.stats["levels"]
    assert st.n == ref.stats["n"] and st.m == ref.stats["m"]
    assert st.iters_lp == ref.stats["it_lp"] and st.iters_rw == ref.stats["it_rw"] and st.iters_rs == ref.stats["it_rs"]
    assert st.cut_level == ref.stats["cut_level"]
    assert st.edge_iters == ref.stats["edge_iters"]
    assert cut == ref.cut == st.cut
    assert (_np(part) == ref.part).all()
    return part, cut, st


def test_partition_grid_64x64_k8(ctx):
    g = graphgen.grid2d(64, 64)
    _check_partition(ctx, g, True, 8)


@pytest.mark.parametrize("name,g,unit", graphs_small(), ids=[x[0] for x in graphs_small()])
@pytest.mark.parametrize("k", [2, 8, 64])
def test_partition_matches_oracle(ctx, name, g, unit, k):
    _check_partition(ctx, g, unit, k, seed=k)


# the Jetlp versions of Table 2 (Sec. 6.1.4): whole partitions, bit-exact
LP_VERSIONS = [("baseline", jet.FLAG_BASELINE_LP), ("baseline+locks", jet.FLAG_STRICT_GAIN | jet.FLAG_NO_AFTERBURN),
               ("baseline+weak_afterburner", jet.FLAG_WEAK_AFTERBURN | jet.FLAG_NO_LOCKS),
               ("baseline+full_afterburner", jet.FLAG_NO_LOCKS), ("full_jetlp", 0)]


@pytest.mark.parametrize("version,flags", LP_VERSIONS, ids=[v[0] for v in LP_VERSIONS])
def test_partition_lp_versions_match_oracle(version, flags):
    g = graphgen.grid3d(20, 20, 20, vw=(1, 4), ew=(1, 10), seed=3)
    c = jet.Context(0, flags=flags)
    try:
        ref = oracle.partition(g, 32, 0.03, 1, oracle.Options(flags=_oracle_ablation(flags)))
        part, cut, st = c.partition(g.xadj, g.adjncy, g.vwgt, g.adjwgt, k=32, eps=0.03, seed=1, return_stats=True)
        assert st.cut_level == ref.stats["cut_level"]
        assert cut == ref.cut and (_np(part) == ref.part).all()
    finally:
        c.close()


def test_partition_hostloop(ctx_hostloop):
    g = graphgen.grid3d(24, 24, 24, vw=(1, 4), ew=(1, 10), seed=1)
    _check_partition(ctx_hostloop, g, False, 64)


@pytest.mark.parametrize("name,g,unit", graphs_small()[1:4], ids=[x[0] for x in graphs_small()[1:4]])
def test_partition_graph_loop_matches_oracle(ctx_graph, name, g, unit):
    _check_partition(ctx_graph, g, unit, 64, seed=3)


def test_partition_batch_matches_oracle(ctx):
    """The batched form: graphs of uneven size (RGGs as in the batched
    workload, a mesh, an R-MAT graph), each with its own k and seed, on
    4 workers; every graph bit-exact with the oracle."""
    rng = np.random.default_rng(3)
    gs = [graphgen.rgg(int(n), seed=i + 1) for i, n in enumerate(np.exp(rng.uniform(np.log(1000), np.log(60000), 10)))]
    gs += [graphgen.grid3d(16, 16, 16, vw=(1, 4), ew=(1, 10), seed=2), graphgen.rmat(12, seed=4)]
    ks = [int(x) for x in rng.choice(np.arange(2, 65, 2), len(gs))]
    items = [dict(xadj=g.xadj, adjncy=g.adjncy, vwgt=g.vwgt, adjwgt=g.adjwgt, k=k, eps=0.03, seed=i + 7)
             for i, (g, k) in enumerate(zip(gs, ks))]
    out = ctx.partition_batch(items, workers=4)
    for (part, cut, status, ms), g, k, it in zip(out, gs, ks, items):
        ref = oracle.partition(g, k, 0.03, it["seed"])
        assert status == ref.status and cut == ref.cut and (_np(part) == ref.part).all()


def _batch_graphs():
    """Uneven sizes and kinds: small RGGs (every level within the cluster
    threshold), weighted meshes, a weighted R-MAT graph, larger RGGs."""
    rng = np.random.default_rng(11)
    gs = [graphgen.rgg(int(n), seed=i + 20) for i, n in enumerate(rng.integers(300, 4000, 14))]
    gs += [graphgen.grid3d(12, 10, 9, vw=(1, 4), ew=(1, 10), seed=3), graphgen.grid2d(70, 50, ew=(1, 5), seed=2),
           graphgen.rmat(11, seed=8, vw=(1, 3), ew=(1, 5)), graphgen.rgg(20000, seed=5), graphgen.rgg(45000, seed=6)]
    ks = [int(x) for x in rng.choice([2, 4, 8, 16, 32, 64, 128], len(gs))]
    return gs, ks


@pytest.mark.parametrize("opts", [{}, {"cluster_blocks": 2}, {"cluster_blocks": 8}, {"cluster_max_n": 0},
                                  {"cluster_max_n": 64}, {"cluster_max_n": 1 << 20}],
                         ids=["default", "clusters2", "clusters8", "no_small_levels", "threshold64", "all_small"])
def test_partition_batch_small_levels_in_one_launch(opts):
    """The batched form refines every graph's levels up to cluster_max_n in
    one persistent cluster launch over a queue of graphs (the rest level by
    level); each graph bit-exact with the oracle, under every threshold and
    cluster size."""
    gs, ks = _batch_graphs()
    items = [dict(xadj=g.xadj, adjncy=g.adjncy, vwgt=g.vwgt if i >= 14 else None,
                  adjwgt=g.adjwgt if i >= 14 else None, k=k, eps=0.03, seed=i + 3) for i, (g, k) in enumerate(zip(gs, ks))]
    with jet.Context(0, **opts) as c:
        out = c.partition_batch(items, workers=3)
    for i, ((part, cut, status, ms), g, k, it) in enumerate(zip(out, gs, ks, items)):
        og = graphgen.Graph(g.n, g.xadj, g.adjncy, it["vwgt"], it["adjwgt"])
        ref = oracle.partition(og, k, 0.03, it["seed"])
        assert status == ref.status and cut == ref.cut, i
        assert (_np(part) == ref.part).all(), i


@pytest.mark.parametrize("g,k", [(graphgen.grid3d(24, 24, 24, vw=(1, 4), ew=(1, 10), seed=9), 64),
                                 (graphgen.rmat(12, seed=5), 16)], ids=["grid24w_k64", "rmat12_k16"])
def test_coarsest_refined_matches_oracle(ctx, g, k):
    """jet_coarsest_refined (the learned form's training labels): the greedy
    initial partition of the coarsest level refined by Alg. 3 with that
    level's seed and c_coarse, bit for bit."""
    seed = 3
    h = ctx.coarsen(g.xadj, g.adjncy, g.vwgt, g.adjwgt, k=k, seed=seed)
    part, cut = ctx.coarsest_refined(h, k=k, eps=0.03, seed=seed)
    h.close()
    lv = oracle.coarsen(g, k, seed)
    gc = lv[-1].graph
    ref = oracle.refine(gc, k, oracle.initial_partition(gc, k), 0.03, is_finest=len(lv) == 1,
                        seed=oracle.level_seed(seed, len(lv) - 1))
    assert cut == ref.cut and (_np(part) == ref.part).all()
    assert cut == oracle.partition(g, k, 0.03, seed).stats["cut_level"][len(lv) - 1]


def test_partition_without_pdl_is_identical(ctx):
    """Programmatic dependent launch is an execution choice: the same
    partition with JET_FLAG_NO_PDL, on the CUDA-graph and the host loop."""
    g = graphgen.grid3d(40, 40, 40, vw=(1, 4), ew=(1, 10), seed=6)
    ref = ctx.partition(g.xadj, g.adjncy, g.vwgt, g.adjwgt, k=32, seed=2)
    for flags in (jet.FLAG_NO_PDL, jet.FLAG_NO_PDL | jet.FLAG_HOSTLOOP, jet.FLAG_HOSTLOOP, jet.FLAG_GRID_LOOP):
        with jet.Context(0, flags=flags, cluster_max_n=0) as c:
            part, cut = c.partition(g.xadj, g.adjncy, g.vwgt, g.adjwgt, k=32, seed=2)
        assert cut == ref[1] and torch.equal(part, ref[0])


def test_autotune_picks_fastest_and_keeps_results():
    """jet_autotune: every candidate timed, the fastest cluster threshold
    kept in the context, and every graph still bit-exact with the oracle
    (execution choices never change results)."""
    rng = np.random.default_rng(5)
    gs = [graphgen.rgg(int(n), seed=i + 3) for i, n in enumerate(np.exp(rng.uniform(np.log(1000), np.log(20000), 6)))]
    ks = [int(x) for x in rng.choice(np.arange(2, 33, 2), len(gs))]
    items = [dict(xadj=g.xadj, adjncy=g.adjncy, k=k, eps=0.03, seed=i + 1) for i, (g, k) in enumerate(zip(gs, ks))]
    c = jet.Context(0)
    rep = c.autotune(items, reps=1)
    cands = rep["candidates"]
    sizes = {"cluster_blocks": 4, "cluster_max_n": 6, "workers": 5, "list_blocks_per_sm": 3, "apply_blocks_per_sm": 3,
             "list_items_per_block": 3, "scan_blocks_per_sm": 3, "hub_degree": 3}
    assert [x["stage"] for x in cands] == [st for st, m in sizes.items() for _ in range(m)]
    for st in sizes:
        assert rep[st] == min((x for x in cands if x["stage"] == st), key=lambda x: x["ms"])["value"], st
        if st != "workers":
            assert getattr(c.options, st) == rep[st], st
    for (part, cut), g, k, it in zip(rep["parts"], gs, ks, items):
        ref = oracle.partition(g, k, 0.03, it["seed"])
        assert cut == ref.cut and (_np(part) == ref.part).all()
    part, cut = c.partition(gs[0].xadj, gs[0].adjncy, None, None, k=ks[0], seed=1)
    assert cut == oracle.partition(gs[0], ks[0], 0.03, 1).cut
    c.close()


def test_partition_host_entry_point(ctx):
    g = graphgen.grid3d(16, 16, 16, vw=(1, 4), ew=(1, 10), seed=4)
    ref = oracle.partition(g, 32, 0.03, 3)
    part, cut = ctx.partition_host(g.xadj, g.adjncy, g.vwgt, g.adjwgt, k=32, eps=0.03, seed=3)
    assert cut == ref.cut and (part == ref.part).all()


def test_partition_deterministic_and_seed_sensitive(ctx):
    g = graphgen.rgg(20000, seed=11)
    a = ctx.partition(g.xadj, g.adjncy, None, None, k=16, seed=4)
    b = ctx.partition(g.xadj, g.adjncy, None, None, k=16, seed=4)
    c = ctx.partition(g.xadj, g.adjncy, None, None, k=16, seed=5)
    assert a[1] == b[1] and (_np(a[0]) == _np(b[0])).all()
    assert not (_np(a[0]) == _np(c[0])).all()


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

def test_edge_cases(ctx):
    # empty graph
    e = graphgen.Graph(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    part, cut = ctx.partition(e.xadj, e.adjncy, None, None, k=4)
    assert part.numel() == 0 and cut == 0
    # edgeless graph, k = 3
    iso = graphgen.Graph(10, np.zeros(11, np.int64), np.zeros(0, np.int32), np.ones(10, np.int32), np.zeros(0, np.int32))
    _check_partition(ctx, iso, True, 3)
    # k = 1 and k > n
    g = graphgen.grid2d(7, 5)
    _check_partition(ctx, g, True, 1)
    _check_partition(ctx, g, True, 50)
    # the largest supported k
    g = graphgen.rgg(30000, seed=3)
    _check_partition(ctx, g, True, jet.JET_MAX_K)
    # a vertex heavier than the balance limit: cannot be balanced
    g = graphgen.grid2d(10, 10)
    vw = np.ones(g.n, np.int32); vw[0] = 60
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, None)
    ref = oracle.partition(og, 4, 0.03, 1)
    part, cut = ctx.partition(g.xadj, g.adjncy, vw, None, k=4)
    assert ref.status == 1 and ctx.last_status == 1   # JET_WUNBALANCED
    assert cut == ref.cut and (_np(part) == ref.part).all()


def test_partition_star_hub_matches_oracle(ctx):
    """One hub adjacent to 12,000 leaves that form a ring (ring edges heavier):
    the hub row is one long row in every refinement phase, and its merged
    coarse row (each coarse leaf twice) goes through the radix-sort path of
    the contraction; eps = 0 as well (the tightest balance)."""
    n = 12001
    tri = [[0, v, 1] for v in range(1, n)]
    tri += [[v, v % (n - 1) + 1, 2] for v in range(1, n)]
    g = graph_from_triples(n, tri)
    assert np.diff(g.xadj).max() == n - 1
    _check_partition(ctx, g, False, 16, seed=4)
    _check_partition(ctx, g, False, 8, seed=5, eps=0.0)


def test_errors(ctx):
    g = graphgen.grid2d(6, 6)
    with pytest.raises(jet.JetError) as ei:
        ctx.partition(g.xadj, g.adjncy, None, None, k=0)
    assert ei.value.status == -1
    with pytest.raises(jet.JetError):
        ctx.partition(g.xadj, g.adjncy, None, None, k=jet.JET_MAX_K + 1)
    with pytest.raises(jet.JetError):
        ctx.partition(g.xadj, g.adjncy, None, None, k=4, eps=-0.1)
    # overflowing weight sums
    big = np.full(g.nnz, 2 ** 30, np.int32)
    with pytest.raises(jet.JetError) as ei:
        ctx.partition(g.xadj, g.adjncy, None, big, k=4)
    assert ei.value.status == -6
    # invalid graphs are caught with JET_FLAG_VALIDATE
    with jet.Context(0, flags=jet.FLAG_VALIDATE) as vctx:
        ok = vctx.partition(g.xadj, g.adjncy, None, None, k=4)
        assert ok[1] >= 0
        bad = g.adjncy.copy(); bad[0] = 0            # self-loop at vertex 0
        with pytest.raises(jet.JetError) as ei:
            vctx.partition(g.xadj, bad, None, None, k=4)
        assert ei.value.status == -2
        asym = g.adjwgt.copy(); asym[0] = 5           # asymmetric weight
        with pytest.raises(jet.JetError) as ei:
            vctx.partition(g.xadj, g.adjncy, None, asym, k=4)
        assert ei.value.status == -2
    # out-of-range partition passed to refine
    with pytest.raises(jet.JetError):
        ctx.refine(g.xadj, g.adjncy, None, None, 4, np.full(g.n, 7, np.int32))


# --------------------------------------------------------------------------
# full-size workloads (the benchmark's launch configuration)
# --------------------------------------------------------------------------

def test_partition_grid_128cube_k64_full_size(ctx):
    """128^3 mesh, vwgt U[1,4], adjwgt U[1,10], k = 64, eps = 0.03, seed 1:
    the benchmark workload; the oracle runs it end to end."""
    g = graphgen.grid3d(128, 128, 128, vw=(1, 4), ew=(1, 10), seed=1)
    part, cut, st = _check_partition(ctx, g, False, 64, seed=1)
    L, _ = oracle.limit(int(g.vwgt.sum()), 64, 0.03)
    assert st.max_part_w <= L


def test_initial_partition_rmat_s22_full_size(ctx):
    """R-MAT scale 22 (the power-law workload, 4.2M vertices with its isolated
    vertices kept): the greedy initial partition of the whole graph, as it runs
    when coarsening stalls at the first level."""
    g = graphgen.rmat(22, seed=1)
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, None, None)
    for k in (2, 256):
        assert (_np(ctx.initial_partition(g.xadj, g.adjncy, None, k)) == oracle.initial_partition(og, k)).all()


def test_partition_rmat_s16_k64(ctx):
    g = graphgen.rmat(16, seed=1)
    _check_partition(ctx, g, True, 64)
