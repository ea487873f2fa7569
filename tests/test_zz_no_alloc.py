"""jet_lp_pass_noalloc — the Jetlp pass for callers that cannot let the
library allocate device memory (a process whose memory is reserved by its own
pool, a latency-bound loop where cudaMalloc/cudaFree would synchronise the
device).  Its scratch is a fixed array inside the library, shared by all
calls; this file checks, through the C ABI, that two calls in a row give
exactly what jet_lp_pass gives and what the oracle's Jetlp pass (Alg. 4)
computes, that the calls make no device allocation, and that oversized
inputs are refused.

Named so that pytest collects it last."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu

jet = pytest.importorskip("paper_2304_13194_gb300")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = jet.Context(0)
    yield c
    c.close()


def _inputs(g, k, seed):
    rng = np.random.default_rng(seed)
    part = oracle.initial_partition(g, k)
    noise = rng.random(g.n) < 0.1
    part[noise] = rng.integers(0, k, int(noise.sum()))
    locked = (rng.random(g.n) < 0.1).astype(np.uint8)
    return part, locked


def _same(a, b):
    for key in ("Pd", "F", "inX", "F2", "inM"):
        assert torch.equal(a[key], b[key]), key


def _matches_oracle(got, g, vw, ew, k, part, locked, c):
    og = graphgen.Graph(g.n, g.xadj, g.adjncy, vw, ew)
    ref = oracle.jetlp(og, k, part, locked, c=c)
    F = got["F"].cpu().numpy().astype(np.int64)
    assert (F == np.where(ref["F"] == oracle.NONE, jet.NONE_GAIN, ref["F"])).all()
    assert (got["Pd"].cpu().numpy() == ref["Pd"]).all()
    inX = ref["inX"]
    assert (got["inX"].cpu().numpy().astype(bool) == inX).all()
    assert (got["F2"].cpu().numpy()[inX] == ref["F2"][inX]).all()
    assert (got["inM"].cpu().numpy().astype(bool) == ref["inM"]).all()


def test_noalloc_equals_lp_pass_on_two_calls_in_a_row(ctx):
    # call 1: weighted 3D mesh; call 2: R-MAT with rows > 16 (warp path) and
    # unit weights, a different size, so stale scratch from call 1 would show
    g1 = graphgen.grid3d(40, 30, 25, vw=(1, 4), ew=(1, 10), seed=2)
    g2 = graphgen.rmat(14, seed=3)
    for g, unit, k, c, seed in [(g1, False, 64, 0.25, 1), (g2, True, 16, 0.75, 2)]:
        part, locked = _inputs(g, k, seed)
        ew = None if unit else g.adjwgt
        vw = None if unit else g.vwgt
        ref = ctx.lp_pass(g.xadj, g.adjncy, vw, ew, k, part, locked, c=c)
        got = ctx.lp_pass_noalloc(g.xadj, g.adjncy, vw, ew, k, part, locked, c=c)
        _same(got, ref)
        _matches_oracle(got, g, vw, ew, k, part, locked, c)
        assert int(got["inX"].sum()) > 0 and int(got["inM"].sum()) > 0


def test_noalloc_makes_no_device_allocation(ctx):
    g = graphgen.grid3d(30, 30, 20, vw=(1, 4), ew=(1, 10), seed=6)
    part, locked = _inputs(g, 32, 7)
    dev = torch.device("cuda", 0)
    t = [torch.from_numpy(a).to(dev) for a in (g.xadj, g.adjncy, g.vwgt, g.adjwgt, part, locked)]
    out = {"Pd": torch.empty(g.n, dtype=torch.int32, device=dev), "F": torch.empty(g.n, dtype=torch.int32, device=dev),
           "inX": torch.empty(g.n, dtype=torch.uint8, device=dev), "F2": torch.empty(g.n, dtype=torch.int32, device=dev),
           "inM": torch.empty(g.n, dtype=torch.uint8, device=dev)}
    ctx.lp_pass_noalloc(*t[:4], 32, t[4], t[5], c=0.25, out=out)          # first call: address look-up
    before = jet.binding.alloc_count()
    for _ in range(2):
        ctx.lp_pass_noalloc(*t[:4], 32, t[4], t[5], c=0.25, out=out)
    assert jet.binding.alloc_count() == before
    # the counter does move for the allocating entry point
    ctx.lp_pass(*t[:4], 32, t[4], t[5], c=0.25)
    assert jet.binding.alloc_count() > before
    _matches_oracle(out, g, g.vwgt, g.adjwgt, 32, part, locked, 0.25)


def test_noalloc_repeated_call_same_result(ctx):
    g = graphgen.grid2d(300, 200, ew=(1, 5), seed=4)
    part, locked = _inputs(g, 8, 5)
    a = ctx.lp_pass_noalloc(g.xadj, g.adjncy, None, g.adjwgt, 8, part, locked, c=0.25)
    a = {k: v.clone() for k, v in a.items()}
    b = ctx.lp_pass_noalloc(g.xadj, g.adjncy, None, g.adjwgt, 8, part, locked, c=0.25)
    _same(a, b)
    _same(a, ctx.lp_pass(g.xadj, g.adjncy, None, g.adjwgt, 8, part, locked, c=0.25))


def test_noalloc_refuses_oversized_graph(ctx):
    n = jet.binding.JET_NOALLOC_MAX_N + 1
    xadj = np.zeros(n + 1, np.int64)           # edgeless: refused on size before any device work
    with pytest.raises(jet.JetError) as ei:
        ctx.lp_pass_noalloc(xadj, np.zeros(0, np.int32), None, None, 4, np.zeros(n, np.int32))
    assert ei.value.status == -1 and "JET_NOALLOC_MAX_N" in str(ei.value)
