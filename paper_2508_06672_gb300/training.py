"""Training of the proposal network on coarse maps the method itself
computes, and evaluation of the learned search against the full-grid search.

The scenes come from the caller (``scenes(seeds)`` yields dicts with the
captures y1, y2 (K x N x 2), their format, the full search's grid, the
ephemerides, fs, fc and the true emitter position); the repository's
``train_proposal.py`` drives this with the seeded simulator. For every
training scene the library computes the K coarse maps of the footprint
(dg_coarse_maps); windows of ``crop`` x ``crop`` cells around the emitter
(and one elsewhere) with a Gaussian target on the emitter's cell are kept on
the device, and the network is trained on them with the library's forward,
backward and Adam kernels.
"""
from __future__ import annotations

import json
import time

import numpy as np


def make_crops(maps, ci, cj, crop, rng, n_pos=2, n_neg=1):
    """Windows of the maps (device, K x cells x cells) and their targets."""
    from .learned import target_map
    cells = maps.shape[-1]
    xs, ts = [], []
    full_t = target_map(cells, ci, cj)
    for k in range(n_pos + n_neg):
        if k < n_pos:
            i0 = int(np.clip(ci - rng.integers(4, crop - 4), 0, cells - crop))
            j0 = int(np.clip(cj - rng.integers(4, crop - 4), 0, cells - crop))
        else:
            i0, j0 = int(rng.integers(0, cells - crop + 1)), int(rng.integers(0, cells - crop + 1))
        xs.append(maps[:, i0:i0 + crop, j0:j0 + crop].clone())
        ts.append(full_t[i0:i0 + crop, j0:j0 + crop].copy())
    return xs, ts


def train(args, scenes, first):
    """Train a ProposalNet on the scenes of seeds 1000 .. 1000 + args.train - 1."""
    import torch
    from . import learned as L
    from .proposal import ProposalNet

    search = L.LearnedSearch(first["grid"], first["ephem"], first["fs"], first["fc"], None, cells=args.cells)
    K = search.K
    net = ProposalNet([K] + [int(c) for c in args.channels.split(",")] + [1], seed=args.seed,
                      tc=getattr(args, "tc", False))
    rng = np.random.default_rng(args.seed)
    X, T = [], []
    t0 = time.time()
    for n, sc in enumerate(scenes(range(1000, 1000 + args.train))):
        search.geo.set_grid(search.node_grid)
        search.load_captures(sc["fmt"], torch.from_numpy(sc["y1"]).cuda(), torch.from_numpy(sc["y2"]).cuda())
        maps = search.coarse()
        ci, cj = L.cell_of(search.node_grid, sc["lat"], sc["lon"])
        xs, ts = make_crops(maps, ci, cj, args.crop, rng)
        X += xs
        T += [torch.tensor(t, dtype=torch.float32, device="cuda") for t in ts]
        if (n + 1) % 250 == 0:
            print(f"maps {n + 1}/{args.train} {time.time() - t0:.1f}s", flush=True)
    X = torch.stack(X)
    T = torch.stack(T).unsqueeze(1).contiguous()
    print(f"training set {tuple(X.shape)} in {time.time() - t0:.1f}s", flush=True)
    n = X.shape[0]
    steps = 0
    t1 = time.time()
    for ep in range(args.epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        losses = []
        lr = args.lr * (0.5 ** (ep // max(1, args.epochs // 3)))
        for b0 in range(0, n - args.batch + 1, args.batch):
            idx = perm[b0:b0 + args.batch]
            loss = net.train_step(X[idx].contiguous(), T[idx].contiguous(), args.pos_weight, lr)
            losses.append(loss)
            steps += 1
        torch.cuda.synchronize()
        print(f"epoch {ep} lr {lr:.2e} loss {float(torch.stack(losses).mean()):.5f} "
              f"({time.time() - t1:.1f}s, {steps} steps)", flush=True)
    search.close()
    return net, dict(train_scenes=args.train, crops=n, epochs=args.epochs, steps=steps,
                     train_s=time.time() - t1, maps_s=t1 - t0)


def evaluate(net, args, scenes, first):
    """The learned search (with ``net`` and with the sum of the coarse maps)
    against the full-grid search on the scenes of seeds 5, 100005, ..."""
    import torch
    from . import dg
    from . import learned as L

    search = L.LearnedSearch(first["grid"], first["ephem"], first["fs"], first["fc"], net, cells=args.cells)
    judge = dg.Geolocator(first["grid"], first["ephem"], first["fs"], first["fc"], algo="cdft",
                          contract="bf16x3", stream=search.geo.stream)
    cost = torch.empty((int(first["grid"]["nlat"]), int(first["grid"]["nlon"])), dtype=torch.float32,
                       device="cuda")
    sumnet = L.SumNet(search.K)
    rows = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    seeds = [5] + [100005 + i for i in range(args.eval - 1)]
    for sc in scenes(seeds):
        y1, y2 = torch.from_numpy(sc["y1"]).cuda(), torch.from_numpy(sc["y2"]).cuda()
        judge.load_captures(sc["fmt"], y1, y2)
        search.load_captures(sc["fmt"], y1, y2)
        torch.cuda.synchronize()
        ev[0].record(search.geo.stream)
        judge.cost_surface(out=cost)
        jf = judge.argmax_refine(cost, search.refine[0], search.refine[1])
        ev[1].record(search.geo.stream)
        best, _, peaks = search.search(net, fallback=False)   # the proposals alone
        ev[2].record(search.geo.stream)
        sbest, _, speaks = search.search(sumnet, fallback=False)
        ev[3].record(search.geo.stream)
        torch.cuda.synchronize()
        jn = (jf["i"], jf["j"])

        def covered(pk):
            for p in pk:
                g = search.region_grid(p["lat_deg"], p["lon_deg"])
                ci, cj = L.node_of(first["grid"], g["lat0_deg"], g["lon0_deg"])
                if abs(jn[0] - round(ci)) <= search.half and abs(jn[1] - round(cj)) <= search.half:
                    return True
            return False

        def err(f):
            return L.distance_m(f["refined_lat_deg"], f["refined_lon_deg"], sc["lat"], sc["lon"]) if f else 1e9

        r = dict(seed=sc["seed"], waveform=sc["waveform"], snr=sc["snr"],
                 judge_err_m=err(jf), net_err_m=err(best), sum_err_m=err(sbest),
                 net_recall=covered(peaks), sum_recall=covered(speaks),
                 net_same=bool(best) and L.distance_m(best["refined_lat_deg"], best["refined_lon_deg"],
                                                      jf["refined_lat_deg"], jf["refined_lon_deg"]) < 100.0,
                 sum_same=bool(sbest) and L.distance_m(sbest["refined_lat_deg"], sbest["refined_lon_deg"],
                                                       jf["refined_lat_deg"], jf["refined_lon_deg"]) < 100.0,
                 judge_ms=ev[0].elapsed_time(ev[1]), net_ms=ev[1].elapsed_time(ev[2]),
                 sum_ms=ev[2].elapsed_time(ev[3]))
        rows.append(r)
        print(json.dumps(r), flush=True)
    judge.close()
    search.close()
    keys = ["net_recall", "sum_recall", "net_same", "sum_same"]
    summary = {k: float(np.mean([r[k] for r in rows])) for k in keys}
    for k in ("judge_err_m", "net_err_m", "sum_err_m", "judge_ms", "net_ms", "sum_ms"):
        summary[k + "_median"] = float(np.median([r[k] for r in rows]))
    summary["n"] = len(rows)
    return summary, rows
