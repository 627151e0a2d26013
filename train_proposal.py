"""Train the learned proposal's network on the GPU and evaluate the learned
search against the full-grid search, on seeded synthetic scenes.

    python train_proposal.py --train 20000 --eval 200 --epochs 10 \\
        --channels 32,64,128,64 --tc \\
        --out paper_2508_06672_gb300/weights/proposal_2000km.npz

Scenes come from sim.learned (a 2000 km footprint, seeded emitter position,
waveform and SNR); a spawned process pool simulates them ahead of the GPU.
Training scenes are seeds 1000, 1001, ...; evaluation scenes 5, 100005, ...
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def scene(seed):
    import sim
    s = sim.learned(int(seed))
    return dict(seed=int(seed), y1=s.y1, y2=s.y2, grid=s.grid, ephem=s.ephem, fs=s.fs_hz, fc=s.fc_hz,
                fmt=s.fmt, lat=s.emitter_lat_deg, lon=s.emitter_lon_deg, waveform=s.meta["waveform"],
                snr=s.meta["snr_db"])


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--train", type=int, default=1500)
    ap.add_argument("--eval", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--pos-weight", type=float, default=100.0)
    ap.add_argument("--crop", type=int, default=128)
    ap.add_argument("--cells", type=int, default=512)
    ap.add_argument("--channels", default="32,64,64")
    ap.add_argument("--tc", action="store_true",
                    help="convolutions on the tensor cores (BF16 operands, FP32 accumulation)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=0)
    ap.add_argument("--out", default="")
    ap.add_argument("--weights", default="", help="evaluate these weights instead of training")
    ap.add_argument("--report", default="")
    ap.add_argument("--profile-kernels", action="store_true",
                    help="only run the coarse maps and the network forward on one scene, 3 times (a small "
                         "case for a profiler: ~0.5 GB of device memory)")
    args = ap.parse_args(argv)
    if args.profile_kernels:
        import torch
        from paper_2508_06672_gb300 import learned as L
        from paper_2508_06672_gb300.proposal import ProposalNet
        sc = scene(5)
        net = ProposalNet.load(args.weights or os.path.join(ROOT, "paper_2508_06672_gb300", "weights",
                                                            "proposal_2000km.npz"))
        search = L.LearnedSearch(sc["grid"], sc["ephem"], sc["fs"], sc["fc"], net, cells=args.cells)
        search.load_captures(sc["fmt"], torch.from_numpy(sc["y1"]).cuda(), torch.from_numpy(sc["y2"]).cuda())
        for _ in range(3):
            search.heatmap()
        torch.cuda.synchronize()
        search.close()
        print("profiled: coarse maps + network forward x 3")
        return
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.workers or max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        def scenes(seeds):
            return pool.imap(scene, seeds, chunksize=1)

        from paper_2508_06672_gb300 import training
        from paper_2508_06672_gb300.proposal import ProposalNet
        info = {}
        if args.weights:
            net = ProposalNet.load(args.weights)
        else:
            net, info = training.train(args, scenes, scene(1000))
            if args.out:
                os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
                net.save(args.out)
        summary, rows = training.evaluate(net, args, scenes, scene(5)) if args.eval > 0 else ({}, [])
    summary.update(info)
    print("SUMMARY " + json.dumps(summary), flush=True)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(dict(summary=summary, rows=rows, args=vars(args)), f, indent=1)


if __name__ == "__main__":
    main()
