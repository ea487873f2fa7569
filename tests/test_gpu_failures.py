"""Failure detection without a GPU fault.

  * Device allocation failure: jet_debug_fail_alloc makes the nth allocation
    the library attempts fail on the host, before it reaches CUDA.  Every
    allocation point of a partition is hit in turn; each call must return
    JET_ENOMEM, release what it holds, and leave the context able to produce
    the oracle's partition on the next call.
  * A bounded device wait that runs out: the persistent level loop's grid
    barriers give up after `barrier_polls` polls; with a limit of one poll a
    block that arrives before the others gives up at once, every block
    leaves the launch, and the call returns JET_ETIMEOUT — the kernel ends,
    nothing hangs, and the context and device keep working.
"""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu

jet = pytest.importorskip("paper_2304_13194_gb300")

ENOMEM, ETIMEOUT = -3, -5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.device("cuda", 0)


def _dev_graph(g, dev):
    return [torch.from_numpy(a).to(dev) if a is not None else None for a in (g.xadj, g.adjncy, g.vwgt, g.adjwgt)]


def test_every_allocation_failure_returns_enomem_and_context_recovers(dev):
    g = graphgen.grid3d(18, 16, 14, vw=(1, 4), ew=(1, 10), seed=5)
    ref = oracle.partition(g, 16, 0.03, 3)
    t = _dev_graph(g, dev)
    with jet.Context(0, cluster_max_n=0) as ctx:
        ctx.partition(*t, k=16, seed=3)                       # warm (pools, attributes)
        a0 = jet.binding.alloc_count()
        part, cut = ctx.partition(*t, k=16, seed=3)
        n_alloc = jet.binding.alloc_count() - a0
        assert n_alloc > 5 and cut == ref.cut
        for nth in range(1, n_alloc + 1):
            jet.binding.debug_fail_alloc(nth)
            with pytest.raises(jet.JetError) as ei:
                ctx.partition(*t, k=16, seed=3)
            assert ei.value.status == ENOMEM, nth
            assert "injected" in str(ei.value)
            # the context still partitions correctly
            part, cut = ctx.partition(*t, k=16, seed=3)
            assert cut == ref.cut and (part.cpu().numpy() == ref.part).all(), nth
    jet.binding.debug_fail_alloc(0)
    torch.cuda.synchronize()


def test_allocation_failure_in_one_batch_item(dev):
    gs = [graphgen.rgg(3000 + 500 * i, seed=i + 1) for i in range(4)]
    items = [dict(xadj=torch.from_numpy(g.xadj).to(dev), adjncy=torch.from_numpy(g.adjncy).to(dev), k=8, eps=0.03,
                  seed=i + 1) for i, g in enumerate(gs)]
    refs = [oracle.partition(g, 8, 0.03, i + 1) for i, g in enumerate(gs)]
    with jet.Context(0) as ctx:
        jet.binding.debug_fail_alloc(3)
        with pytest.raises(jet.JetError) as ei:
            ctx.partition_batch(items, workers=2)
        assert ei.value.status == ENOMEM
        out = ctx.partition_batch(items, workers=2)
        for (part, cut, status, ms), r in zip(out, refs):
            assert status == r.status and cut == r.cut and (part.cpu().numpy() == r.part).all()
    jet.binding.debug_fail_alloc(0)


def test_grid_barrier_wait_runs_out_and_returns_etimeout(dev):
    g = graphgen.grid3d(40, 40, 40, vw=(1, 4), ew=(1, 10), seed=2)
    t = _dev_graph(g, dev)
    with jet.Context(0, flags=jet.FLAG_GRID_LOOP, cluster_max_n=0, barrier_polls=1) as ctx:
        with pytest.raises(jet.JetError) as ei:
            ctx.partition(*t, k=32, seed=2)
        assert ei.value.status == ETIMEOUT
        assert "grid barrier" in str(ei.value)
        # the same context still runs work that has no grid barrier
        p0 = oracle.initial_partition(g, 32)
        cut, pw = ctx.cut(*t, 32, p0)
        assert cut == oracle.cut(g, p0) and (pw.cpu().numpy() == oracle.part_weights(g, p0, 32)).all()
    torch.cuda.synchronize()
    # and the device is fine: the persistent loop with the default limit
    ref = oracle.partition(g, 32, 0.03, 2)
    with jet.Context(0, flags=jet.FLAG_GRID_LOOP, cluster_max_n=0) as ctx:
        part, cut = ctx.partition(*t, k=32, seed=2)
    assert cut == ref.cut and (part.cpu().numpy() == ref.part).all()
