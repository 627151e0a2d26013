"""bench.py on the CPU: the reference arm's JSON line, and no silent fallback.

The reference arm times the oracle on a bounded sample of the default
workload and prints one JSON line with the same metric, unit and direction as
the library's arm. Without a GPU the library's arm must fail (non-zero exit)
instead of measuring something else. Two helpers of the line: the clock
summary taken from nvidia-smi samples, and the contraction's DRAM traffic,
reported only for the kernel source it was captured on."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "3", "--reference-step-s", "0.3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "candidate·sample correlations/s" and d["unit"] == "cand·samples/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"].startswith("large: 4001x4001")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_library_arm_fails_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run("--steps", "1", "--warmup", "3", "--no-direct", "--no-cpu-baseline")
    assert r.returncode != 0
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_clock_summary_reads_the_sampled_lines():
    b = _bench()
    c = b.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2055, 2070, 1200.5, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbled line", "0, [N/A], 2070, 1, 0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines = ["0, 1200, 2070, 700, 0x8, Active, Not Active, Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_contraction_traffic_only_for_the_source_it_was_measured_on(tmp_path, monkeypatch):
    import hashlib

    b = _bench()
    src = os.path.join(ROOT, "paper_2508_06672_gb300", "csrc", "dg_cdft_mma.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha1(f.read()).hexdigest()[:16]
    t = {"source_sha1_16": sha, "workload": "large", "contract": "fp16x3", "chunk": 1024, "bytes_per_launch": 1.5e9}
    monkeypatch.setattr(b, "CONTRACT_TRAFFIC", [t])
    assert b.contract_traffic(t["workload"], t["contract"], t["chunk"]) == t["bytes_per_launch"]
    assert b.contract_traffic(t["workload"], "bf16", t["chunk"]) is None
    assert b.contract_traffic("tiny", t["contract"], t["chunk"]) is None
    assert b.contract_traffic(t["workload"], t["contract"], 256) is None
    # another kernel source: no traffic figure
    src = tmp_path / "paper_2508_06672_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "dg_cdft_mma.cu").write_text("// a changed kernel\n")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.contract_traffic(t["workload"], t["contract"], t["chunk"]) is None
    # every recorded figure names a workload, a form and a chunk
    for e in _bench().CONTRACT_TRAFFIC:
        assert set(e) == {"source_sha1_16", "workload", "contract", "chunk", "bytes_per_launch"}


def test_reference_arm_under_torchrun_prints_on_rank_0_only():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
                        "--reference-step-s", "0.3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    # torchrun sets OMP_NUM_THREADS=1; the line reports every core of the process's affinity, and
    # the oracle is given that many threads explicitly
    assert d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))


def test_roofline_counts_the_contractions_own_launches():
    """Each batch of snapshots on the tensor-core path launches its DFT-operand
    table kernel and then the contraction, both timed in the contraction's
    class: the roofline's launches are the contraction's, half of them."""
    import types

    b = _bench()
    cdft = types.SimpleNamespace(algo="cdft", contract="fp16x3", tiles="auto")
    f = b.launch_fields(cdft, "contract", 6, 0.06)
    assert f["launches"] == 3 and abs(f["ms_per_launch"] - 20.0) < 1e-9 and "launches_basis" in f
    for a, dom in ((types.SimpleNamespace(algo="cdft", contract="fp32", tiles="auto"), "contract"),
                   (cdft, "combine"), (types.SimpleNamespace(algo="direct", contract="fp16x3", tiles="auto"), "corr")):
        f = b.launch_fields(a, dom, 6, 0.06)
        assert f["launches"] == 6 and "launches_basis" not in f
