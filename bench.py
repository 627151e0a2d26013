"""Throughput of direct geolocation on GB300: candidate*sample correlations/s.

One step = one pass of the whole hot path over the workload: the cost surface
(geometry, delay/Doppler alignment, correlation, accumulation over all K
snapshots; Sec. III, Eq. 11, Algorithm 1) and the argmax with a dense local
refinement. The default workload is the large footprint, the largest that the
method's configurations put on one GPU: a 4001 x 4001 grid at 400 m,
K = 50 snapshots of N = 131072 complex int8 samples at 20 MHz from a wideband
(18 MHz) noise jammer at -20 dB SNR. --workload mid runs the 1001 x 1001 /
100 m grid with K = 20 x N = 65536 complex int16 samples of a 10 MHz / 10 us
chirp at -15 dB.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dg|reference]

Rank 0 prints one JSON line. --impl reference times the CPU oracle on a
bounded sample of the same workload (same metric and unit).
Under torchrun each rank processes its own block of grid rows (weak scaling:
the grid grows with the number of GPUs).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_CAND_SAMPLE = 14          # conj product 6 + derotation 6 + accumulation 2
CDFT_COMBINE_FLOPS = 30             # per candidate x super-chunk: 6-bin interpolation 22 + phase MAC 8
FP32_PROBE_ITERS = 50000           # ~50 ms per probe launch on a GB300
METRIC = "candidate·sample correlations/s"
UNIT = "cand·samples/s"
REFINE_SPACING_M, REFINE_WINDOW_M = 10.0, 200.0


def workload(name, rank=0, world=1, grid=None):
    import sim

    if name == "mid":
        s = sim.mid()
        desc = ("mid: 1001x1001 grid at 100 m, K=20 x N=65536 complex int16, chirp 10 MHz / 10 us, "
                "fs 12.5 MHz, fc 1575.42 MHz, SNR -15 dB, 2 LEO receivers 50 km apart at 550 km")
    elif name == "tiny":
        s = sim.tiny()
        desc = "tiny: 101x101 grid at 1 km, K=1 x N=4096 complex64, 2 MHz noise, fs 5 MHz, SNR -5 dB"
    elif name == "large":
        s = sim.large()
        desc = ("large: 4001x4001 grid at 400 m, K=50 x N=131072 complex int8, 18 MHz noise, "
                "fs 20 MHz, SNR -20 dB")
    else:
        raise SystemExit(f"unknown workload {name}")
    if grid:
        # a smaller (or larger) square grid at the same spacing, same centre
        s.grid = dict(s.grid, nlat=grid, nlon=grid)
        desc += f" [grid overridden to {grid}x{grid}]"
    if world > 1:
        # weak scaling: a grid world times taller, this rank's block of rows
        s.grid = dict(s.grid, nlat=s.grid["nlat"] * world)
    return s, desc


# DRAM traffic of one contraction launch, from one ncu capture per workload
# (dram__bytes_read.sum + dram__bytes_write.sum); valid only for the kernel
# source it was measured on
CONTRACT_TRAFFIC = [
    {"source_sha1_16": "9879c696159e10c5", "workload": "mid", "contract": "fp16x3", "chunk": 1024,
     "bytes_per_launch": 241.93e6},
    # captured on a 1201^2 sub-grid of the large workload (both main batches of a surface: 4476.3 MB
    # for 8 702 208 (lag, chunk) rows = 514.4 B per row, 99 % of it the W rows written), scaled to
    # the large step's 17 565 632 rows over its 3 contraction launches
    {"source_sha1_16": "86624cc3027d5dc3", "workload": "large", "contract": "fp16x3", "chunk": 2048,
     "bytes_per_launch": 3.012e9},
]


def contract_traffic(workload, contract, chunk):
    import hashlib

    src = os.path.join(ROOT, "paper_2508_06672_gb300", "csrc", "dg_cdft_mma.cu")
    try:
        with open(src, "rb") as f:
            sha = hashlib.sha1(f.read()).hexdigest()[:16]
    except OSError:
        return None
    for t in CONTRACT_TRAFFIC:
        if (sha, workload, contract, chunk) == (t["source_sha1_16"], t["workload"], t["contract"], t["chunk"]):
            return t["bytes_per_launch"]
    return None


# arithmetic each contraction form performs, as the line's dtype
CONTRACT_DTYPE = {
    "fp32": "f32 (FP32 CUDA-core contraction)",
    "bf16": "bf16 (one bf16 tensor-core product, fp32 accumulate)",
    "fp16": "fp16 (one fp16 tensor-core product, fp32 accumulate)",
    "bf16x3": "bf16x3 (split bf16 products hi*hi + lo*hi + hi*lo, fp32 accumulate)",
    "fp16x3": "fp16x3 (split fp16 products hi*hi + lo*hi + hi*lo, fp32 accumulate)",
}


def fp32_peak(dev_index, stream=None, reps=5):
    """Measured FP32 FMA peak of the device (dg_fp32_peak: every SM full of
    independent FMA chains), median of `reps` launches, with the SM clock
    sampled meanwhile. Returns a dict."""
    import torch

    import paper_2508_06672_gb300 as P

    st = stream.cuda_stream if stream is not None else 0
    runs = []
    with ClockSampler(_smi_id(dev_index)) as clk:
        for _ in range(reps):
            runs.append(P.dg_fp32_peak(FP32_PROBE_ITERS, st))
    torch.cuda.synchronize(dev_index)
    tf = statistics.median(r[0] for r in runs)
    c = clk.summary()
    return {"tflops": tf, "sm_count": runs[0][2], "ms_per_launch": statistics.median(r[1] for r in runs),
            "sm_mhz": c["sm_mhz"], "reasons": c["reasons"],
            "basis": ("dg_fp32_peak: 8 resident 256-thread CTAs per SM, 8 independent FMA chains per thread, "
                      "2 flop per FMA / CUDA-event time, median of 5 launches")}


PEAK_BASIS_TENSOR = ("measured cuBLAS bf16 dense GEMM burst (MEASURED_PEAKS.json bf16_tflops); fp16 has the same "
                     "nominal dense rate (2.25 PFLOP/s)")


def tensor_peak(contract):
    """Dense 16-bit tensor peak: the measured bf16 burst figure (fp16 runs at
    the same nominal rate), else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s), else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ oracle (CPU)
def oracle_rate(scene, target_s, seed=0, max_pts=None, nthreads=None):
    """Time the FP64 oracle on a bounded sample of the workload's candidates
    (nthreads: every core this process may run on, unless given).
    Returns (cand*samples/s, seconds, points, cores)."""
    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    KN = scene.k_steps * scene.n_samples
    y1, y2 = oracle.iq_to_f64(scene.y1), oracle.iq_to_f64(scene.y2)
    args = (scene.grid, scene.ephem, scene.fs_hz, scene.fc_hz, y1, y2)
    # every core this process may run on, whatever OMP_NUM_THREADS says (a
    # launcher such as torchrun sets it to 1): the line reports this count
    cores = nthreads or host_cores()
    # calibrate on a few points, then size the sample for ~target_s
    cal = rng.integers(0, scene.G, max(4, cores))
    t0 = time.perf_counter()
    oracle.cost_points(*args, idx=cal, nthreads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    rate = cal.size * KN / dt
    npts = int(max(cores, min(target_s * rate / KN, max_pts or 1e12)))
    idx = rng.integers(0, scene.G, npts)
    t0 = time.perf_counter()
    oracle.cost_points(*args, idx=idx, nthreads=cores)
    dt = time.perf_counter() - t0
    return npts * KN / dt, dt, npts, cores


def run_reference(a, rank, world):
    """The reference arm: the CPU oracle on the same metric and workload."""
    if rank != 0:
        return
    scene, desc = workload(a.workload, grid=a.grid)
    KN = scene.k_steps * scene.n_samples
    rates = []
    npts = None
    for it in range(a.warmup + a.steps):
        r, dt, n, cores = oracle_rate(scene, a.reference_step_s, seed=it, max_pts=npts)
        npts = npts or n
        if it >= a.warmup:
            rates.append((r, dt))
    total_units = sum(r * dt for r, dt in rates)
    total_s = sum(dt for _, dt in rates)
    value = total_units / total_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total_s / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "G": scene.G, "K": scene.k_steps, "N": scene.n_samples},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{npts} random grid nodes x all {scene.k_steps} snapshots x {scene.n_samples} samples per step (FP64, OpenMP over nodes), {cpu_model()}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- GPU arm
def run_dg(a, rank, world, local_rank):
    import torch

    import paper_2508_06672_gb300 as P
    from paper_2508_06672_gb300.shard import allreduce_argmax, shard_rows

    dist = None
    if world > 1:
        import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    scene, desc = workload(a.workload, rank, world, a.grid)
    row0, nrows = shard_rows(scene.grid["nlat"], world, rank)
    G_rank = nrows * scene.grid["nlon"]
    KN = scene.k_steps * scene.n_samples
    stream = torch.cuda.Stream(dev)
    g = P.Geolocator(scene.grid, scene.ephem, scene.fs_hz, scene.fc_hz, algo=a.algo, row0=row0,
                     nrows=nrows, timing=True, stream=stream, device=local_rank, chunk=a.chunk,
                     contract=a.contract, tiles=a.tiles)
    y1d = torch.from_numpy(scene.y1).to(dev)
    y2d = torch.from_numpy(scene.y2).to(dev)
    y1h = torch.from_numpy(scene.y1).pin_memory()
    y2h = torch.from_numpy(scene.y2).pin_memory()
    with torch.cuda.stream(stream):
        g.load_captures(scene.fmt, y1d, y2d)
        cost = torch.empty((nrows, scene.grid["nlon"]), dtype=torch.float32, device=dev)
        flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step():
        g.cost_surface(cost)
        return g.argmax_refine(cost, REFINE_SPACING_M, REFINE_WINDOW_M)

    fp = fp32_peak(local_rank, stream)      # the FP32 ceiling of the ALU rooflines

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            step()
    barrier()
    g.reset_counters()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    fixes = []
    gpu_id = _smi_id(local_rank)
    with ClockSampler(gpu_id) as clk:
        barrier()
        t_wall = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(a.steps):
                flush.zero_()                     # L2 flush, outside the timed events
                ev[i][0].record(stream)
                fixes.append(step())
                ev[i][1].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    step_ms = [s.elapsed_time(e) for s, e in ev]
    sync_ms_per_step = sum(step_ms) / a.steps
    kt = {name: g.kernel_time(cls) for name, cls in (("corr", P.DG_K_CORR), ("plan", P.DG_K_CDFT_PLAN),
                                                     ("contract", P.DG_K_CDFT_CONTRACT),
                                                     ("combine", P.DG_K_CDFT_COMBINE),
                                                     ("accumulate", P.DG_K_ACCUM), ("argmax", P.DG_K_ARGMAX),
                                                     ("refine", P.DG_K_REFINE))}
    bucket_chunks, cand_chunks = g.cdft_work()
    chunk_lo, chunk_hi = g.cdft_chunks() if a.algo == "cdft" else (0, 0)
    corr_ms, corr_launches = kt["corr"]
    launches = g.launch_count()
    dev_s = sum(step_ms) / 1e3
    latency = full_grid_latency(g, cost, flush, stream)
    barrier()

    if a.graph:
        # the headline pass: each step is one CUDA-graph launch of the whole
        # step (dg_graph_*: surface, argmax, refinement on the device, fix)
        # and a read of its fix; the pass above gave the per-kernel times
        with torch.cuda.stream(stream):
            g.graph_capture(cost, REFINE_SPACING_M, REFINE_WINDOW_M)
            for _ in range(a.warmup):
                g.graph_launch()
                g.graph_fix()
        barrier()
        g.reset_counters()
        with ClockSampler(gpu_id) as clk:
            barrier()
            t_wall = time.perf_counter()
            with torch.cuda.stream(stream):
                for i in range(a.steps):
                    flush.zero_()                 # L2 flush, outside the timed events
                    ev[i][0].record(stream)
                    g.graph_launch()
                    ev[i][1].record(stream)
                    fixes[i] = g.graph_fix()
            barrier()
            t_wall = time.perf_counter() - t_wall
        step_ms = [s.elapsed_time(e) for s, e in ev]
        dev_s = sum(step_ms) / 1e3
        launches = g.launch_count()

        def e2e_step():
            g.load_captures(scene.fmt, y1h, y2h)  # same formats and lengths: the graph's buffers
            g.graph_launch()
            return g.graph_fix()                   # synchronises and copies the fix back
    else:
        def e2e_step():
            g.load_captures(scene.fmt, y1h, y2h)
            return step()                         # synchronises and copies the fix back

    # end to end through the public API: pinned host captures in, fix out
    with torch.cuda.stream(stream):
        for _ in range(2):
            e2e_step()
    barrier()
    e2e_ms = []
    for i in range(a.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            e2e_step()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    # the same, streamed: two contexts on two streams, each with its graph;
    # step i + 1's L2 flush, capture upload and launch are issued before step
    # i's fix is waited for, so the upload of one step overlaps the compute
    # of the other. Every step still includes its upload and its fix read.
    e2e_pipe_s = None
    if a.graph:
        stream2 = torch.cuda.Stream(dev)
        g2 = P.Geolocator(scene.grid, scene.ephem, scene.fs_hz, scene.fc_hz, algo=a.algo, row0=row0,
                          nrows=nrows, stream=stream2, device=local_rank, chunk=a.chunk, contract=a.contract,
                          tiles=a.tiles)
        with torch.cuda.stream(stream2):
            g2.load_captures(scene.fmt, y1d, y2d)
            cost2 = torch.empty_like(cost)
            flush2 = torch.empty_like(flush)
        g2.cost_surface(cost2)
        g2.argmax_refine(cost2, REFINE_SPACING_M, REFINE_WINDOW_M)
        g2.graph_capture(cost2, REFINE_SPACING_M, REFINE_WINDOW_M)
        pair = [(g, stream, flush), (g2, stream2, flush2)]

        def issue(k):
            gg, ss, ff = pair[k % 2]
            with torch.cuda.stream(ss):
                ff.zero_()
                gg.load_captures(scene.fmt, y1h, y2h)
                gg.graph_launch()

        for k in range(4):  # warm-up of the pair
            issue(k)
            pair[k % 2][0].graph_fix()
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        issue(0)
        for i in range(a.steps):
            if i + 1 < a.steps:
                issue(i + 1)
            pair[i % 2][0].graph_fix()
        e2e_pipe_s = (time.perf_counter() - t0) / a.steps
        g2.close()
    h2d = int(scene.y1.nbytes + scene.y2.nbytes)
    # two argmax records and two error words, or (graph) the fix record and
    # two error words
    d2h = 96 + 2 * 4 if a.graph else 2 * 48 + 2 * 4  # the fix (or two argmax records) and error words

    kernels = {}
    alu_peak = fp["tflops"]
    issued_per_step = None
    if a.algo == "cdft":
        # every kernel of the chunked-DFT path against its own roofline; the
        # dominant one is the headline
        # with the automatic choice every batch of this workload took the
        # same chunk (checked below); the flop count assumes one chunk
        chunk = chunk_hi
        nprod = 3 if a.contract.endswith("x3") else 1
        tensor = a.contract != "fp32"
        # contraction: one chunk x 64-bin complex DFT per (lag, chunk) row =
        # 512 * chunk real flops of algorithmic work; the split forms issue
        # three such products on the tensor cores
        contract_flops = 512 * chunk * bucket_chunks
        tc_peak = tensor_peak(a.contract)
        # combine: when the super-chunks leave about one per candidate the
        # kernel is a gather (order index, FDOA, surface write: 12 B per
        # candidate and snapshot, plus the W rows the super-chunk pass reads
        # and writes, 2 x 512 B per (lag, chunk)); otherwise it is FP32 work
        gk = G_rank * scene.k_steps
        combine_hbm = cand_chunks <= 2 * gk
        combine_units = (12 * gk + 1024 * bucket_chunks) / 1e12 if combine_hbm else CDFT_COMBINE_FLOPS * cand_chunks
        for name, flops, bound, peak, basis, unit in (
                ("contract", contract_flops, "tensor" if tensor else "alu", tc_peak if tensor else alu_peak,
                 "512 flop x chunk per (lag, chunk) row (one complex chunk x 64-bin DFT)", "TFLOP/s"),
                ("combine", combine_units * (1e12 if combine_hbm else 1), "hbm" if combine_hbm else "alu",
                 hbm_peak() if combine_hbm else alu_peak,
                 ("12 B per candidate x snapshot + 1024 B per (lag, chunk) (super-chunk pass)" if combine_hbm else
                  f"{CDFT_COMBINE_FLOPS} flop per candidate x super-chunk (6-bin interpolation 22 + phase MAC 8)"),
                 "GB/s" if combine_hbm else "TFLOP/s")):
            ms, n = kt[name]
            if n:
                scale = 1e9 if unit == "GB/s" else 1e12
                ach = flops * a.steps / (ms / 1e3) / scale
                kernels[name] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                                 "frac": ach / peak, "ms_per_step": ms / a.steps, "basis": basis}
                if name == "contract" and tensor and nprod > 1:
                    kernels[name]["issued_frac"] = nprod * ach / peak
        dom = max(("contract", "combine"), key=lambda n: kt[n][0])
        flops_per_step = contract_flops if dom == "contract" else combine_units * (1e12 if combine_hbm else 1)
        if dom == "contract" and tensor and nprod > 1:
            issued_per_step = nprod * contract_flops
        corr_ms, corr_launches = kt[dom]
        tc_name = "k_cdft_contract_hk (Hankel tiles)" if a.tiles == "hankel" and chunk <= 1024 else "k_cdft_contract_tc"
        roof_kernel = {"contract": (f"{tc_name} ({a.contract} tcgen05, {chunk}-sample chunks x 64 bins)"
                                    if tensor else f"k_cdft_contract_f32 (FP32 CUDA cores, {chunk}-sample chunks)"),
                       "combine": "k_cdft_superchunk + k_cdft_combine (per-candidate interpolation + super-chunk phase sum)"}[dom]
        roof_basis = kernels[dom]["basis"]
        roof_bound, roof_peak = kernels[dom]["bound"], kernels[dom]["peak"]
        roof_unit = kernels[dom]["unit"]
    else:
        roof_unit = "TFLOP/s"
        flops_per_step = FLOPS_PER_CAND_SAMPLE * G_rank * KN
        roof_kernel = "k_corr_direct (FP32, integer lag)"
        roof_basis = f"{FLOPS_PER_CAND_SAMPLE} flop per candidate*sample x G*K*N per launch"
        roof_bound, roof_peak = "alu", alu_peak
    worst = torch.tensor([dev_s, corr_ms / 1e3, sum(e2e_ms) / 1e3,
                          (e2e_pipe_s if e2e_pipe_s is not None else sum(e2e_ms) / 1e3 / a.steps)],
                         dtype=torch.float64)
    if dist:
        worst = worst.to(dev)
        dist.all_reduce(worst, op=dist.ReduceOp.MAX)
        worst = worst.cpu()
    dev_s, corr_s, e2e_s, e2e_step_s = (float(x) for x in worst)
    units = world * G_rank * KN * a.steps
    gfix = (fixes[-1]["cost"], row0 * scene.grid["nlon"] + fixes[-1]["index"])
    if dist:
        gfix = allreduce_argmax(*gfix)  # max-loc over the row blocks (after timing)

    if rank == 0:
        fix = fixes[-1]
        centre = (scene.grid["nlat"] // 2, scene.grid["nlon"] // 2)  # the emitter's node
        gi, gj = divmod(int(gfix[1]), scene.grid["nlon"])
        achieved = flops_per_step * a.steps / corr_s / (1e9 if roof_unit == "GB/s" else 1e12)
        peak = roof_peak
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": units / dev_s, "unit": UNIT, "n_gpus": world,
            "step": ("one CUDA-graph launch of surface + argmax + refinement (dg_graph_launch), fix read back"
                     if a.graph else "dg_cost_surface + dg_argmax_refine (host-synchronising calls)"),
            "ms_per_step_synchronous_calls": sync_ms_per_step,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * dev_s / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": CONTRACT_DTYPE[a.contract] if a.algo == "cdft" else "f32",
            "data": "synthetic",
            "config": {"workload": desc, "G": G_rank * world, "K": scene.k_steps, "N": scene.n_samples,
                       "fmt": scene.fmt, "delay": "integer", "algo": a.algo, "acc": "power",
                       "chunk": ((a.chunk if a.chunk else f"auto: {chunk_lo}..{chunk_hi}" if chunk_lo != chunk_hi
                                  else f"auto: {chunk_hi}") if a.algo == "cdft" else None),
                       "contract": a.contract if a.algo == "cdft" else None,
                       "tiles": a.tiles if a.algo == "cdft" else None,
                       "refine": f"{REFINE_SPACING_M:g} m spacing, +-{REFINE_WINDOW_M:g} m",
                       "l2": "flushed between timed steps (256 MB write outside the events)",
                       "parallelism": f"grid rows sharded over {world} GPU(s)", "seed": scene.meta["seed"]},
            "e2e": {"value": units / (e2e_step_s * a.steps), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "mode": ("streamed: two contexts on two streams, step i+1's upload and launch issued before "
                             "step i's fix is read (total wall time / steps)" if a.graph else
                             "one step at a time (upload, step, fix read), wall time per step"),
                    "serial": {"value": units / e2e_s,
                               "mode": "one step at a time (upload, graph launch, fix read), wall time per step"}},
            "gpu_launches": int(launches),
            "full_grid_latency": latency,
            "roofline": {"bound": roof_bound, "achieved": achieved, "peak": peak, "unit": roof_unit,
                         "frac": achieved / peak,
                         **({"issued_achieved": issued_per_step * a.steps / corr_s / 1e12,
                             "issued_frac": issued_per_step * a.steps / corr_s / 1e12 / peak,
                             "issued_basis": "the split form's three 16-bit products, 3 x 512 flop x chunk per "
                                             "(lag, chunk) row: tensor-pipe work, not algorithmic work"}
                            if issued_per_step else {}),
                         "traffic": (contract_traffic(a.workload, a.contract, chunk_hi)
                                     if a.algo == "cdft" and roof_bound == "tensor" and not a.grid else None),
                         "kernel": roof_kernel,
                         "peak_basis": (PEAK_BASIS_TENSOR if roof_bound == "tensor" else
                                        "measured HBM copy (MEASURED_PEAKS.json hbm_gbs)" if roof_bound == "hbm"
                                        else "measured FP32 FMA peak (dg_fp32_peak, see device.fp32_peak)"),
                         "achieved_basis": roof_basis + " / CUDA-event time of the launches",
                         **launch_fields(a, dom if a.algo == "cdft" else "corr", corr_launches, corr_s)},
            "kernel_ms_per_step": {n: v[0] / a.steps for n, v in kt.items() if v[1]},
            "cdft_work": ({"lag_chunk_rows": bucket_chunks, "candidate_superchunks": cand_chunks}
                          if a.algo == "cdft" else None),
            "kernels": kernels,
            "device": {"name": torch.cuda.get_device_name(dev), "sm_count": fp["sm_count"],
                       "fp32_peak": fp},
            "clocks": clocks,
            "fix": {"i": gi, "j": gj, "emitter_cell": list(centre),
                    "offset_cells": [gi - centre[0], gj - centre[1]],
                    "refined_latlon_deg": [fix["refined_lat_deg"], fix["refined_lon_deg"]]},
            "wall_s": t_wall,
        }
        if world == 1 and a.algo == "cdft" and not a.no_direct:
            line["direct_path"] = direct_reference(scene, local_rank, stream, alu_peak,
                                                   grid=DIRECT_SUBGRID.get(a.workload))
        if world == 1 and not a.no_cpu_baseline:
            r, dt, npts, cores = oracle_rate(scene, a.cpu_baseline_s)
            r1, dt1, npts1, _ = oracle_rate(scene, a.cpu_baseline_s / 3, seed=1, nthreads=1)
            line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"{npts} random grid nodes x all {scene.k_steps} snapshots x {scene.n_samples} samples ({dt:.1f} s, FP64, OpenMP over nodes), {cpu_model()}",
                                    "one_thread": {"value": r1, "unit": UNIT, "cores": 1,
                                                   "sample": f"{npts1} random grid nodes, same snapshots ({dt1:.1f} s)"}}
        print(json.dumps(line), flush=True)
    g.close()


# the direct path is timed on a sub-grid of workloads whose full grid would
# take it tens of seconds per surface (same spacing and centre)
DIRECT_SUBGRID = {"large": 1001}


def direct_reference(scene, local_rank, stream, alu_peak, steps=3, warmup=1, grid=None):
    """The direct (sample-by-sample) evaluation of the same surface, timed
    the same way, for context: cand*samples/s and its FP32 roofline."""
    import torch

    import paper_2508_06672_gb300 as P

    dev = torch.device("cuda", local_rank)
    gd = dict(scene.grid, nlat=grid, nlon=grid) if grid else scene.grid
    g = P.Geolocator(gd, scene.ephem, scene.fs_hz, scene.fc_hz, algo="direct", timing=True,
                     stream=stream, device=local_rank)
    with torch.cuda.stream(stream):
        g.load_captures(scene.fmt, torch.from_numpy(scene.y1).to(dev), torch.from_numpy(scene.y2).to(dev))
        cost = torch.empty((gd["nlat"], gd["nlon"]), dtype=torch.float32, device=dev)
        for _ in range(warmup):
            g.cost_surface(cost)
    torch.cuda.synchronize(dev)
    g.reset_counters()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(steps):
            g.cost_surface(cost)
        ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1) / steps
    corr_ms, n = g.kernel_time(P.DG_K_CORR)
    g.close()
    units = gd["nlat"] * gd["nlon"] * scene.k_steps * scene.n_samples
    ach = FLOPS_PER_CAND_SAMPLE * units * steps / (corr_ms / 1e3) / 1e12
    return {"value": units / (ms / 1e3), "unit": UNIT, "ms_per_surface": ms,
            "grid": f"{gd['nlat']}x{gd['nlon']}" + (" sub-grid (same spacing and centre)" if grid else ""),
            "roofline": {"bound": "alu", "kernel": "k_corr_direct", "achieved": ach, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": ach / alu_peak,
                         "peak_basis": "measured FP32 FMA peak (dg_fp32_peak)"}}


# ------------------------------------------------------- many uneven captures
BATCH_CAPTURES = 64


def _batch_scene(kw):
    import sim

    return sim.make_scene(**kw)


def batch_scenes(seed, n=BATCH_CAPTURES):
    """Seeded stand-in for a stream of uneven captures: per capture K in
    5..100 snapshots, N = 2^e samples with e in 12..18, a grid side in
    256..2048 at 50..500 m, a tone, chirp or noise emitter at -25..0 dB,
    complex int16 at 12.5 MHz. The parameters are drawn here in order; the
    captures are simulated by a spawned process pool (before any GPU work)."""
    import multiprocessing as mp

    rng = np.random.default_rng(seed)
    kws = []
    for i in range(n):
        side = int(rng.integers(256, 2049))
        kws.append(dict(seed=int(rng.integers(1 << 30)), fs_hz=12.5e6, n_samples=1 << int(rng.integers(12, 19)),
                        k_steps=int(rng.integers(5, 101)), fmt="ci16",
                        waveform=["tone", "chirp", "noise"][int(rng.integers(3))],
                        snr_db=float(rng.uniform(-25.0, 0.0)), grid_n=side,
                        grid_spacing_m=float(rng.uniform(50.0, 500.0)), bw_hz=2e6))
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        return pool.map(_batch_scene, kws, chunksize=1)


def run_batch(a, rank, world, local_rank):
    """All captures' steps as one CUDA graph (dg_batch_*), against the same
    steps issued one after the other through the synchronising calls."""
    import torch

    import paper_2508_06672_gb300 as P

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    scenes = batch_scenes(1000 + rank)
    units = sum(s.G * s.k_steps * s.n_samples for s in scenes)
    gs, costs, hosts = [], [], []
    for sc in scenes:
        st = torch.cuda.Stream(dev)
        g = P.Geolocator(sc.grid, sc.ephem, sc.fs_hz, sc.fc_hz, algo="cdft", contract=a.contract, tiles=a.tiles, stream=st,
                         device=local_rank, scratch_mib=1024)
        y1, y2 = torch.from_numpy(sc.y1).pin_memory(), torch.from_numpy(sc.y2).pin_memory()
        with torch.cuda.stream(st):
            g.load_captures(sc.fmt, y1, y2)
            costs.append(torch.empty((g.nrows, g.nlon), dtype=torch.float32, device=dev))
        gs.append(g)
        hosts.append((sc.fmt, y1, y2))
    torch.cuda.synchronize(dev)
    bstream = torch.cuda.Stream(dev)
    batch = P.Batch(gs, costs, REFINE_SPACING_M, REFINE_WINDOW_M, stream=bstream)
    with torch.cuda.stream(bstream):
        flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    for _ in range(a.warmup):
        batch.launch()
        batch.fixes()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    clk = ClockSampler(_smi_id(local_rank))
    torch.cuda.synchronize(dev)
    with clk:
        for i in range(a.steps):
            with torch.cuda.stream(bstream):
                flush.zero_()
                ev[i][0].record(bstream)
            batch.launch()
            ev[i][1].record(bstream)
            batch.fixes()
    dev_ms = [x.elapsed_time(y) for x, y in ev]
    # the same steps, one context after the other, synchronising calls
    seq_ms = []
    for _ in range(max(1, min(a.steps, 3))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for g, c in zip(gs, costs):
            with torch.cuda.stream(g.stream):
                g.cost_surface(c)
                g.argmax_refine(c, REFINE_SPACING_M, REFINE_WINDOW_M)
        torch.cuda.synchronize(dev)
        seq_ms.append(1e3 * (time.perf_counter() - t0))
    # end to end: pinned host captures in, every fix out, one graph launch
    e2e_ms = []
    h2d = sum(y1.numel() * y1.element_size() + y2.numel() * y2.element_size() for _, y1, y2 in hosts)
    for _ in range(max(1, min(a.steps, 3))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for g, (fmt, y1, y2) in zip(gs, hosts):
            with torch.cuda.stream(g.stream):
                g.load_captures(fmt, y1, y2)
        batch.launch()
        batch.fixes()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    nprod = 3 if a.contract.endswith("x3") else 1
    step_s = statistics.median(dev_ms) / 1e3
    # issued tensor flops: 512 x chunk per (lag, chunk) row of every context
    # algorithmic contraction flops: 512 x chunk per (lag, chunk) row of every context
    flops = sum(512 * g.cdft_work()[0] * g.cdft_chunks()[1] for g in gs) if a.contract != "fp32" else 0
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": units / step_s, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": CONTRACT_DTYPE[a.contract], "data": "synthetic",
            "config": {"workload": f"batch: {len(scenes)} uneven captures (K 5-100, N 2^12-2^18, grids 256-2048^2 "
                                   f"at 50-500 m, tone/chirp/noise, ci16, fs 12.5 MHz), one CUDA graph per step",
                       "captures": len(scenes), "cand_samples_per_step": units, "algo": "cdft",
                       "shared_contraction_rounds": batch.rounds(),
                       "contraction": ("one persistent tcgen05 launch per round over the tiles of every capture's "
                                       "r-th snapshot batch (each context's scratch target: 1 GiB)"
                                       if batch.rounds() else "one persistent launch per capture and snapshot batch"),
                       "contract": a.contract, "refine": f"{REFINE_SPACING_M:g} m spacing, +-{REFINE_WINDOW_M:g} m",
                       "l2": "flushed between timed steps (256 MB write inside the batch stream, before the start "
                             "event)", "seed": 1000 + rank},
            "e2e": {"value": units / (statistics.median(e2e_ms) / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": len(scenes) * 100},
            "gpu_launches": batch.launch_count() * a.steps,
            "roofline": {"bound": "tensor", "achieved": flops / step_s / 1e12, "peak": tensor_peak(a.contract),
                         "unit": "TFLOP/s", "frac": flops / step_s / 1e12 / tensor_peak(a.contract),
                         "issued_frac": nprod * flops / step_s / 1e12 / tensor_peak(a.contract),
                         "traffic": None,
                         "kernel": "k_cdft_contract_tc (algorithmic contraction flops over the whole step: a lower bound)",
                         "peak_basis": PEAK_BASIS_TENSOR},
            "sequential": {"ms_per_step": statistics.median(seq_ms),
                           "value": units / (statistics.median(seq_ms) / 1e3),
                           "note": "the same steps issued one context after the other (dg_cost_surface + "
                                   "dg_argmax_refine, host synchronisation per step)"},
            "clocks": clocks,
        }
        print(json.dumps(line))
    batch.close()
    for g in gs:
        g.close()


LEARNED_WEIGHTS = os.path.join(ROOT, "paper_2508_06672_gb300", "weights", "proposal_2000km.npz")
LEARNED_SEEDS = [5] + list(range(300000, 300199))   # held out: training used seeds 1000..


def _learned_scene(seed):
    import sim

    return sim.learned(seed)


def learned_scenes(seeds):
    """The held-out learned-workload scenes, simulated by a spawned process
    pool (before any GPU work)."""
    import multiprocessing as mp

    if len(seeds) <= 2:
        return [_learned_scene(sd) for sd in seeds]
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        return pool.map(_learned_scene, seeds, chunksize=1)


def run_learned(a, rank, world, local_rank):
    """The learned-proposal search against the full-grid search on the 2000 km
    footprint (sim.learned): per step one held-out scene, both searches on
    the same resident captures, CUDA events on the shared stream."""
    import torch

    n_sc = max(1, min(len(LEARNED_SEEDS), a.steps))
    scenes = learned_scenes(LEARNED_SEEDS[:n_sc])

    import paper_2508_06672_gb300 as P
    from paper_2508_06672_gb300 import learned as L
    from paper_2508_06672_gb300.proposal import ProposalNet

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    net = ProposalNet.load(LEARNED_WEIGHTS, device=dev)
    st = torch.cuda.Stream(dev)
    s0 = scenes[0]
    search = L.LearnedSearch(s0.grid, s0.ephem, s0.fs_hz, s0.fc_hz, net, stream=st)
    judge = P.Geolocator(s0.grid, s0.ephem, s0.fs_hz, s0.fc_hz, algo="cdft", contract="bf16x3", stream=st)
    cost = torch.empty((s0.grid["nlat"], s0.grid["nlon"]), dtype=torch.float32, device=dev)
    sumnet = L.SumNet(search.K, device=dev)
    dev_caps = [(torch.from_numpy(sc.y1).to(dev), torch.from_numpy(sc.y2).to(dev)) for sc in scenes]
    host_caps = [(torch.from_numpy(sc.y1).pin_memory(), torch.from_numpy(sc.y2).pin_memory()) for sc in scenes]
    with torch.cuda.stream(st):
        flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)

    def load(i, caps):
        with torch.cuda.stream(st):
            judge.load_captures(scenes[i].fmt, *caps[i])
            search.load_captures(scenes[i].fmt, *caps[i])

    for w in range(a.warmup):
        load(w % n_sc, dev_caps)
        judge.cost_surface(out=cost)
        judge.argmax_refine(cost, 25.0, 500.0)
        search.search()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    learned_ms, full_ms, rec, rec_sum, err_l, err_f, same, fell = [], [], [], [], [], [], [], []
    l0 = search.geo.launch_count() + search.hm.launch_count()
    nn_launches = 2 * len(net.params) - 1
    clk = ClockSampler(_smi_id(local_rank))
    with clk:
        for i in range(a.steps):
            sc = scenes[i % n_sc]
            load(i % n_sc, dev_caps)
            with torch.cuda.stream(st):
                flush.zero_()
            torch.cuda.synchronize(dev)
            ev[0].record(st)
            judge.cost_surface(out=cost)
            jf = judge.argmax_refine(cost, 25.0, 500.0)
            ev[1].record(st)
            with torch.cuda.stream(st):
                flush.zero_()
            ev[1].synchronize()
            e_mid = torch.cuda.Event(enable_timing=True)
            e_mid.record(st)
            lf, _, peaks = search.search()
            ev[2].record(st)
            fell.append(search.fell_back)
            torch.cuda.synchronize(dev)
            full_ms.append(ev[0].elapsed_time(ev[1]))
            learned_ms.append(e_mid.elapsed_time(ev[2]))

            def covered(pk):
                for p in pk:
                    g = search.region_grid(p["lat_deg"], p["lon_deg"])
                    ci, cj = L.node_of(s0.grid, g["lat0_deg"], g["lon0_deg"])
                    if abs(jf["i"] - round(ci)) <= search.half and abs(jf["j"] - round(cj)) <= search.half:
                        return True
                return False

            rec.append(covered(peaks))
            err_f.append(L.distance_m(jf["refined_lat_deg"], jf["refined_lon_deg"], sc.emitter_lat_deg,
                                      sc.emitter_lon_deg))
            err_l.append(L.distance_m(lf["refined_lat_deg"], lf["refined_lon_deg"], sc.emitter_lat_deg,
                                      sc.emitter_lon_deg))
            same.append(L.distance_m(lf["refined_lat_deg"], lf["refined_lon_deg"], jf["refined_lat_deg"],
                                     jf["refined_lon_deg"]) < 100.0)
            if i < n_sc:
                _, _, speaks = search.search(sumnet, fallback=False)
                rec_sum.append(covered(speaks))
    launches = search.geo.launch_count() + search.hm.launch_count() - l0
    launches_per_search = launches / (a.steps + len(rec_sum)) + nn_launches
    # end to end: pinned host captures in, the fix out
    e2e = []
    for i in range(min(a.steps, n_sc)):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(st):
            search.load_captures(scenes[i].fmt, *host_caps[i])
        search.search()
        e2e.append(1e3 * (time.perf_counter() - t0))
    h2d = sum(t.numel() * t.element_size() for t in host_caps[0])
    # the network's forward on the 512 x 512 coarse maps, timed alone
    x = search.maps.view(1, search.K, search.cells, search.cells)
    with torch.cuda.stream(st):
        for _ in range(3):
            net.forward(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(20):
            net.forward(x)
        e1.record(st)
    torch.cuda.synchronize(dev)
    fwd_ms = e0.elapsed_time(e1) / 20
    fwd_flops = sum(2 * 9 * w.shape[0] * w.shape[1] * search.cells * search.cells for w, _ in net.params)
    fp = fp32_peak(local_rank, st)
    alu_peak = fp["tflops"]
    clocks = clk.summary()
    # the plain method's full-grid search (DIRECT FP32, sample by sample) on
    # a 1001^2 sub-grid of the first scene's footprint, scaled to the full grid
    sub = 1001
    dref = direct_reference(s0, local_rank, st, alu_peak, steps=1, warmup=1, grid=sub)
    scale = s0.grid["nlat"] * s0.grid["nlon"] / float(sub * sub)
    plain = {"ms_extrapolated": dref["ms_per_surface"] * scale, "sub_grid": f"{sub}x{sub}",
             "sub_grid_ms": dref["ms_per_surface"], "cand_samples_per_s": dref["value"],
             "basis": "DIRECT FP32 cost surface (dg_cost_surface, CUDA events) on a sub-grid of the same "
                      "footprint, spacing and centre, times the full grid's node count over the sub-grid's; "
                      "its argmax is the CDFT search's (parity), so its localisation error is the full "
                      "search's"}
    if rank == 0:
        med_l, med_f = statistics.median(learned_ms), statistics.median(full_ms)
        line = {
            "metric": "learned-proposal search latency (2000 km footprint; full-grid search timed beside it)",
            "value": med_l, "unit": "ms", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": med_l, "higher_is_better": False, "scaling": "replicas", "vs_baseline": None,
            "dtype": ("bf16 network convolutions (tensor cores, fp32 accumulate)" if net.tc else
                      "f32 network") + ", CDFT contraction bf16x3", "data": "synthetic",
            "config": {"workload": "learned: 2000 km square footprint (4001^2 nodes at 500 m), K = 20 x N = 65536 "
                                   "ci16 at 12.5 MHz, noise / 2 ms chirp / GPS C/A at -21..-12 dB; 512^2 coarse "
                                   f"cells -> network {net.channels} -> top 8 regions of 50 x 50 km at 500 m -> "
                                   "25 m re-evaluation (+-500 m)",
                       "scenes": n_sc, "seeds": LEARNED_SEEDS[:n_sc], "weights": os.path.relpath(LEARNED_WEIGHTS, ROOT),
                       "l2": "flushed before each timed search (256 MB write outside the events)"},
            "full_grid_ms": med_f, "speedup_vs_full_grid": med_f / med_l,
            "plain_full_grid": dict(plain, speedup_of_learned=plain["ms_extrapolated"] / med_l),
            "mean_ms": float(np.mean(learned_ms)), "full_grid_mean_ms": float(np.mean(full_ms)),
            "fallback": {"rule": f"no region proposed, the best region's argmax within {search.edge} nodes "
                                 f"of its border, the best proposal's logit under {search.min_logit}, or the best "
                                 f"region's maximum less than {search.min_region_gap} (relative) above the "
                                 "runner-up's: the full-grid search runs on the same context",
                         "rate": float(np.mean(fell)), "count": int(sum(fell)),
                         "median_ms_when_taken": (float(np.median([t for t, f in zip(learned_ms, fell) if f]))
                                                  if any(fell) else None)},
            "recall": float(np.mean(rec)), "recall_coarse_sum_without_network": float(np.mean(rec_sum)),
            "recall_with_fallback": float(np.mean([r or f for r, f in zip(rec, fell)])),
            "recall_basis": ("recall: the full-grid argmax lies inside one of the proposed regions; "
                             "recall_with_fallback: that, or the fallback ran the full-grid search"),
            "same_fix_as_full_grid": float(np.mean(same)),
            "error_m": {"learned_p50": float(np.median(err_l)), "learned_p90": float(np.percentile(err_l, 90)),
                        "full_grid_p50": float(np.median(err_f)), "full_grid_p90": float(np.percentile(err_f, 90))},
            "e2e": {"value": statistics.median(e2e), "unit": "ms", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 100},
            "gpu_launches": int(round(launches_per_search * a.steps)),
            "roofline": net_roofline(net, fwd_flops, fwd_ms, alu_peak),
            "device": {"name": torch.cuda.get_device_name(dev), "sm_count": fp["sm_count"], "fp32_peak": fp},
            "cpu_baseline": None,
            "clocks": clocks,
        }
        print(json.dumps(line))
    search.close()
    judge.close()


def full_grid_latency(g, cost, flush, stream, runs=10, warmup=2):
    """Full-grid latency: dg_cost_surface alone (no argmax or refinement),
    CUDA events on the library's stream around each call, L2 flushed before
    each; median and mean of `runs` after `warmup` untimed calls."""
    import torch

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(runs)]
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            g.cost_surface(cost)
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            g.cost_surface(cost)
            e1.record(stream)
    stream.synchronize()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    return {"median_ms": statistics.median(ms), "mean_ms": float(np.mean(ms)), "runs": runs, "warmup": warmup,
            "basis": "dg_cost_surface alone (no argmax or refinement), CUDA events, L2 flushed before each"}


def launch_fields(a, dom, class_launches, class_s):
    """Launches of the roofline's kernel and its mean time per launch. On
    the tensor-core path every batch of snapshots launches its DFT-operand
    table kernel (~0.01 ms) and then the contraction, both timed in the
    contraction's class: the contraction's own launches are half of them."""
    tensor = a.algo == "cdft" and a.contract != "fp32" and dom == "contract"
    n = class_launches // 2 if tensor and a.tiles != "hankel" else class_launches
    out = {"launches": n, "ms_per_launch": 1e3 * class_s / max(1, n)}
    if n != class_launches:
        out["launches_basis"] = ("contraction kernel launches (one per batch of snapshots); the class's time "
                                 "also holds the batch's DFT-operand table kernel")
    return out


def net_roofline(net, fwd_flops, fwd_ms, alu_peak):
    """Roofline of the network's forward on the 512^2 maps, timed alone: the
    tensor-core convolution against the dense bf16 peak, or the FP32 one
    against the measured FP32 FMA peak."""
    ach = fwd_flops / (fwd_ms / 1e3) / 1e12
    if net.tc:
        peak = tensor_peak("bf16")
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": "k_conv3x3_tc (BF16 tcgen05, the network's forward on the 512^2 maps, "
                                           "timed alone, with its per-layer weight conversion)",
                "ms_per_forward": fwd_ms, "peak_basis": PEAK_BASIS_TENSOR}
    return {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": ach / alu_peak,
            "traffic": None, "kernel": "k_conv3x3_tiled (the network's forward on the 512^2 maps, timed alone)",
            "ms_per_forward": fwd_ms, "peak_basis": "measured FP32 FMA peak (dg_fp32_peak, see device.fp32_peak)"}


def _smi_id(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return local_rank


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["dg", "reference"], default="dg")
    ap.add_argument("--workload", choices=["large", "mid", "tiny", "batch", "learned"], default="large")
    ap.add_argument("--algo", choices=["direct", "cdft"], default="cdft")
    ap.add_argument("--chunk", type=int, default=0, help="CDFT samples per chunk; 0 = automatic")
    ap.add_argument("--contract", choices=["fp32", "bf16", "fp16", "bf16x3", "fp16x3"], default="fp16x3")
    ap.add_argument("--tiles", choices=["auto", "rows", "lags", "hankel"], default="auto",
                    help="CDFT tensor-core tiles (auto: Hankel where lag-type tiles fit)")
    ap.add_argument("--no-direct", action="store_true", help="skip the direct-path reference measurement")
    ap.add_argument("--grid", type=int, default=0, help="override the grid to GRID x GRID nodes")
    ap.add_argument("--cpu-baseline-s", type=float, default=15.0)
    ap.add_argument("--reference-step-s", type=float, default=6.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="time the host-synchronising calls instead of the whole-step CUDA graph")
    a = ap.parse_args()
    if a.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if a.workload == "batch":
        run_batch(a, rank, world, local_rank)
    elif a.workload == "learned":
        run_learned(a, rank, world, local_rank)
    else:
        run_dg(a, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
