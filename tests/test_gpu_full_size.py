"""Whole-partition parity at full size: every plain configuration of the
scope table, run end to end through the C ABI in the benchmark's launch
configuration, against the oracle on the same seeded graph — partition vector
element by element, cut, maximum part weight and every per-level statistic
(vertices, edges, Jetlp / Jetrw / Jetrs iterations, cut after each level,
refinement edge passes).

  * power-law graph: R-MAT scale 22 (4,194,304 vertices with the isolated ones
    kept, edge factor 16, a=.57 b=c=.19 d=.05, symmetrised, unit weights) at
    k = 2, 8, 64, 256 — heavy-edge matching stalls at its first level, so the
    whole 64M-edge graph is refined, hub rows of up to 162,560 entries
    included;
  * the weighted 128^3 mesh (vwgt U[1,4], adjwgt U[1,10]) at seeds 2-5 (seed 1
    is in test_gpu_parity.py);
  * the paper's own synthetic meshes (Sec. 5): the 2000 x 4000 grid and the
    200^3 cube, unit weights, k = 64.

The oracle partitions (tens of seconds each on one core) start together on
worker threads when the module's fixture is first used; the C oracle runs
without the interpreter lock, so they overlap each other and the GPU work.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu

jet = pytest.importorskip("paper_2304_13194_gb300")

EPS = 0.03
RMAT_KS = (2, 8, 64, 256)
MESH_SEEDS = (2, 3, 4, 5)


def _cases():
    """(id, graph factory, unit weights, k, partition seed)."""
    out = [(f"rmat22_k{k}", "rmat22", True, k, 1) for k in RMAT_KS]
    out += [(f"grid3d_128_w_seed{s}", f"grid3d_128_seed{s}", False, 64, s) for s in MESH_SEEDS]
    out += [("grid2d_2000x4000_k64", "grid2d_2000x4000", True, 64, 1),
            ("grid3d_200_k64", "grid3d_200", True, 64, 1)]
    return out


def _make(name):
    if name == "rmat22":
        return graphgen.rmat(22, seed=1)
    if name.startswith("grid3d_128_seed"):
        return graphgen.grid3d(128, 128, 128, vw=(1, 4), ew=(1, 10), seed=int(name[len("grid3d_128_seed"):]))
    if name == "grid2d_2000x4000":
        return graphgen.grid2d(2000, 4000)
    if name == "grid3d_200":
        return graphgen.grid3d(200, 200, 200)
    raise KeyError(name)


class _Runs:
    """Graphs (generated once) and the oracle's partitions, computed on a
    thread pool in the order the tests need them."""

    def __init__(self):
        self.graphs = {}
        workers = max(2, min(10, (os.cpu_count() or 4)))
        self.pool = ThreadPoolExecutor(max_workers=workers)
        self.futs = {}
        for cid, gname, unit, k, seed in _cases():
            g = self.graph(gname)
            og = graphgen.Graph(g.n, g.xadj, g.adjncy, None if unit else g.vwgt, None if unit else g.adjwgt)
            self.futs[cid] = self.pool.submit(oracle.partition, og, k, EPS, seed)

    def graph(self, gname):
        if gname not in self.graphs:
            self.graphs[gname] = _make(gname)
        return self.graphs[gname]

    def close(self):
        self.pool.shutdown(wait=True, cancel_futures=True)


@pytest.fixture(scope="module")
def runs():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    r = _Runs()
    yield r
    r.close()


@pytest.fixture(scope="module")
def ctx():
    c = jet.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("cid,gname,unit,k,seed", _cases(), ids=[c[0] for c in _cases()])
def test_full_size_partition_matches_oracle(runs, ctx, cid, gname, unit, k, seed):
    g = runs.graph(gname)
    dev = torch.device("cuda", 0)
    xadj = torch.from_numpy(g.xadj).to(dev)
    adj = torch.from_numpy(g.adjncy).to(dev)
    vw = None if unit else torch.from_numpy(g.vwgt).to(dev)
    ew = None if unit else torch.from_numpy(g.adjwgt).to(dev)
    part, cut, st = ctx.partition(xadj, adj, vw, ew, k=k, eps=EPS, seed=seed, return_stats=True)
    status = ctx.last_status
    got = part.cpu().numpy()
    del xadj, adj, vw, ew, part
    ref = runs.futs[cid].result()
    rs = ref.stats
    assert status == ref.status
    assert st.levels == rs["levels"]
    assert st.n == rs["n"] and st.m == rs["m"]
    assert st.iters_lp == rs["it_lp"] and st.iters_rw == rs["it_rw"] and st.iters_rs == rs["it_rs"]
    assert st.cut_level == rs["cut_level"]
    assert st.edge_iters == rs["edge_iters"]
    assert cut == ref.cut == st.cut
    assert st.max_part_w == rs["maxw"]
    assert np.array_equal(got, ref.part)
    # the balance bound of the result (every configuration here can be balanced)
    W = g.n if unit else int(g.vwgt.astype(np.int64).sum())
    L, _ = oracle.limit(W, k, EPS)
    assert st.max_part_w <= L
