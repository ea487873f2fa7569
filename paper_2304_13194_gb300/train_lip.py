"""Training and evaluation of the learned initial partition (jet_lip_*).

Data: (coarsest graph, plain-pipeline partition) pairs.  For each seeded
input graph and coarsening seed, jet_coarsen builds the hierarchy and
jet_coarsest_refined gives the plain pipeline's refined partition of its
coarsest level; jet_lip_features and jet_lip_labels (canonical part numbers)
turn the pair into a training example.  Pairs whose coarsest level has more
than ``max_n`` vertices are skipped.  Minibatches are block-diagonal unions
of several coarsest graphs (every vertex aggregates only its own graph's
neighbours), so one forward/backward/Adam launch sequence trains on many
graphs at once.  All arithmetic runs in the library's kernels; this module
only generates inputs, concatenates arrays and loops.

Default recipe (``python -m paper_2304_13194_gb300.train_lip``): 20,000
pairs from seeded R-MAT graphs of scale 16-20 (edge factor 16, unit weights)
and 3D grids 32^3-96^3 (vertex weights 1-4, edge weights 1-10), k = 64,
eps = 0.03, coarsening with two-hop matches (Sec. 3.1) so that the power-law
graphs reach coarsest levels of a few hundred vertices; evaluation on graphs
from seeds that training never saw, through the same context options.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import binding as _b


def init_params(k: int, seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases (parameter order of jet.h)."""
    r = np.random.default_rng(seed)
    parts = []
    din = _b.LIP_FEATURES
    for _ in range(3):
        fan_in, fan_out = 2 * din, _b.LIP_HIDDEN
        a = math.sqrt(6.0 / (fan_in + fan_out))
        parts += [r.uniform(-a, a, fan_in * fan_out), np.zeros(fan_out)]
        din = _b.LIP_HIDDEN
    a = math.sqrt(6.0 / (_b.LIP_HIDDEN + k))
    parts += [r.uniform(-a, a, _b.LIP_HIDDEN * k), np.zeros(k)]
    return np.concatenate(parts).astype(np.float32)


def _dev(ctx, a, dtype):
    import torch
    return None if a is None else torch.as_tensor(np.asarray(a)).to(device=torch.device("cuda", ctx.device),
                                                                     dtype=dtype)


def make_pairs(ctx, g, k: int, eps: float, seeds, max_n: int = 16384):
    """Training examples from graph g (graphgen.Graph), one per coarsening
    seed: dicts (n, xadj, adjncy, x, y) of the coarsest level; seeds whose
    coarsest level has more than max_n vertices give none."""
    import torch
    args = (_dev(ctx, g.xadj, torch.int64), _dev(ctx, g.adjncy, torch.int32), _dev(ctx, g.vwgt, torch.int32),
            _dev(ctx, g.adjwgt, torch.int32))
    out = []
    for seed in seeds:
        hier = ctx.coarsen(*args, k=k, seed=seed)
        try:
            levels, ns, _ = hier.info()
            if ns[-1] > max_n:
                continue
            lv = hier.level(levels - 1)
            part, _ = ctx.coarsest_refined(hier, k=k, eps=eps, seed=seed)
        finally:
            hier.close()
        x = ctx.lip_features(lv["xadj"], lv["adjncy"], lv["vwgt"], lv["adjwgt"])
        y = ctx.lip_labels(lv["xadj"], lv["adjncy"], k, part)
        out.append(dict(n=lv["n"], xadj=lv["xadj"], adjncy=lv["adjncy"], x=x, y=y))
    return out


def collate(pairs):
    """Block-diagonal union of several examples (concatenation with the
    row-pointer and neighbour-id offsets shifted)."""
    import torch
    xs, adjs, ptrs, ys = [], [], [], []
    voff, eoff = 0, 0
    for p in pairs:
        ptrs.append(p["xadj"][:-1] + eoff)
        adjs.append(p["adjncy"] + voff)
        xs.append(p["x"])
        ys.append(p["y"])
        voff += p["n"]
        eoff += int(p["xadj"][-1].item())
    dev = pairs[0]["x"].device
    ptrs.append(torch.tensor([eoff], dtype=torch.int64, device=dev))
    return dict(n=voff, xadj=torch.cat(ptrs), adjncy=torch.cat(adjs).to(torch.int32), x=torch.cat(xs),
                y=torch.cat(ys))


def batches(pairs, batch_graphs: int, rng):
    order = rng.permutation(len(pairs))
    return [collate([pairs[i] for i in order[s:s + batch_graphs]]) for s in range(0, len(order), batch_graphs)]


def train(model, pairs, epochs: int = 20, batch_graphs: int = 32, lr: float = 3e-3, seed: int = 0, log=None):
    """Adam over shuffled block-diagonal minibatches; returns the mean loss of
    each epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        tot, cnt = 0.0, 0
        step_lr = lr * 0.5 * (1 + math.cos(math.pi * ep / max(epochs, 1)))   # cosine schedule
        for b in batches(pairs, batch_graphs, rng):
            loss = model.train_step(b["xadj"], b["adjncy"], b["x"], b["y"], lr=step_lr)
            tot += loss * b["n"]
            cnt += b["n"]
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep} loss {hist[-1]:.4f}")
    return hist


def accuracy(model, pairs) -> float:
    """Fraction of vertices whose argmax equals their label."""
    hit, tot = 0, 0
    for p in pairs:
        lg = model.forward(p["xadj"], p["adjncy"], p["x"])
        hit += int((lg.argmax(dim=1).to(p["y"].dtype) == p["y"]).sum().item())
        tot += p["n"]
    return hit / max(tot, 1)


def evaluate(ctx, model, graphs, eps: float = 0.03, seed: int = 1):
    """jet_partition_learned on each (name, graph): plain and learned final
    cuts, which was kept, and the phase times."""
    import torch
    out = []
    for name, g in graphs:
        args = (_dev(ctx, g.xadj, torch.int64), _dev(ctx, g.adjncy, torch.int32), _dev(ctx, g.vwgt, torch.int32),
                _dev(ctx, g.adjwgt, torch.int32))
        _, cut, info = model.partition(*args, eps=eps, seed=seed)
        out.append(dict(graph=name, n=g.n, cut=cut, **info))
    return out


def recipe(scales=(16, 17, 18, 19, 20), grid_sides=(32, 48, 64, 80, 96), graph_seeds=(1, 2), pairs=20000):
    """(graph factory list, coarsening seeds per graph) of the default data set."""
    import graphgen
    facts = []
    for s in scales:
        for gs in graph_seeds:
            facts.append((f"rmat{s}_s{gs}", lambda s=s, gs=gs: graphgen.rmat(s, seed=gs)))
    for d in grid_sides:
        for gs in graph_seeds:
            facts.append((f"grid{d}^3_s{gs}", lambda d=d, gs=gs: graphgen.grid3d(d, d, d, vw=(1, 4), ew=(1, 10),
                                                                                   seed=gs)))
    per = max(1, -(-pairs // len(facts)))
    return facts, per


def step_benchmark(ctx, k: int = 64, graphs: int = 64, side: int = 24, steps: int = 50, seed: int = 0):
    """Times training steps (forward, backward, Adam) with CUDA events on a
    block-diagonal batch of `graphs` coarsest levels of seeded weighted
    meshes side^3; returns dict(vertices, ms_per_step, vertices_per_s)."""
    import torch
    import graphgen
    pairs = []
    s = 0
    while len(pairs) < graphs:
        g = graphgen.grid3d(side, side, side, vw=(1, 4), ew=(1, 10), seed=1 + s)
        pairs += make_pairs(ctx, g, k, 0.03, seeds=range(1000, 1000 + min(8, graphs - len(pairs))))
        s += 1
    b = collate(pairs[:graphs])
    model = _b.LearnedPartitioner(ctx, k, init_params(k, seed))
    for _ in range(3):
        model.train_step(b["xadj"], b["adjncy"], b["x"], b["y"], lr=1e-3)
    stream = torch.cuda.current_stream(ctx.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        model.train_step(b["xadj"], b["adjncy"], b["x"], b["y"], lr=1e-3)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    model.close()
    return dict(vertices=b["n"], graphs=graphs, ms_per_step=ms, vertices_per_s=b["n"] / ms * 1e3)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--eps", type=float, default=0.03)
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--scales", default="16,17,18,19,20")
    ap.add_argument("--grids", default="32,48,64,80,96")
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch-graphs", type=int, default=32)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--eval-seeds", default="101,102")
    ap.add_argument("--save", default="")
    ap.add_argument("--no-two-hop", action="store_true")
    ap.add_argument("--step-benchmark", action="store_true",
                    help="only time training steps on a batch of 64 coarsest mesh levels")
    a = ap.parse_args(argv)
    ctx = _b.Context(0, flags=0 if a.no_two_hop else _b.FLAG_TWO_HOP)
    if a.step_benchmark:
        print(json.dumps(step_benchmark(ctx, a.k)))
        return
    facts, _ = recipe(tuple(int(x) for x in a.scales.split(",") if x),
                      tuple(int(x) for x in a.grids.split(",") if x), pairs=a.pairs)
    t0 = time.time()
    data = []
    # graphs whose coarsest level stays above 16,384 vertices for the first
    # three seeds give no pairs; the others share the requested count
    graphs = []
    for name, f in facts:
        g = f()
        first = make_pairs(ctx, g, a.k, a.eps, seeds=range(1000, 1003))
        if first:
            graphs.append((name, g, first))
        else:
            print(f"{name}: coarsest level above 16,384 vertices, skipped ({time.time() - t0:.1f} s)", flush=True)
    per = max(3, -(-a.pairs // max(len(graphs), 1)))
    for name, g, first in graphs:
        data += first + make_pairs(ctx, g, a.k, a.eps, seeds=range(1003, 1000 + per))
        print(f"{name}: {len(data)} pairs so far ({time.time() - t0:.1f} s)", flush=True)
    model = _b.LearnedPartitioner(ctx, a.k, init_params(a.k, a.seed))
    t1 = time.time()
    hist = train(model, data, a.epochs, a.batch_graphs, a.lr, a.seed, log=lambda m: print(m, flush=True))
    t2 = time.time()
    if a.save:
        np.save(a.save, model.get_params())
    import graphgen
    ev_graphs = []
    for es in (int(x) for x in a.eval_seeds.split(",")):
        ev_graphs.append((f"rmat18_s{es}", graphgen.rmat(18, seed=es)))
        ev_graphs.append((f"grid64^3_s{es}", graphgen.grid3d(64, 64, 64, vw=(1, 4), ew=(1, 10), seed=es)))
    ev = evaluate(ctx, model, ev_graphs, a.eps, seed=7)
    print(json.dumps(dict(pairs=len(data), data_s=t1 - t0, train_s=t2 - t1, loss=hist, eval=ev)))


if __name__ == "__main__":
    main()
