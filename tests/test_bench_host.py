"""Host logic of bench.py without a GPU: the maximum over replicas under a
two-rank gloo process group, the clock-sample summary (median SM clock and
throttle reasons), the FP32 peak, the traffic lookup keyed by the far-field
kernel's source and tiling, and the reference arm's JSON line (the oracle timed
on a bounded sample) with its silence on ranks other than 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(torch, dist, world, values[rank], torch.device("cpu"))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_is_the_slowest_replica_on_every_rank():
    import torch.multiprocessing as mp
    world, values = 2, [0.25, 0.75]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), values, out), nprocs=world, join=True,
                           start_method="spawn")
        assert dict(out) == {0: 0.75, 1: 0.75}


def test_max_over_ranks_single_rank_passes_through():
    assert bench.max_over_ranks(None, None, 1, 0.125, None) == 0.125


def test_clock_summary_median_max_and_reasons():
    c = bench.ClockSampler(0)
    rows = [
        (10.0, ["0", "1000", "2070", "500", "Not Active", "Not Active", "Not Active", "Not Active"]),  # before
        (11.0, ["0", "2070", "2070", "900", "Not Active", "Not Active", "Not Active", "Active"]),
        (11.2, ["0", "2055", "2070", "950", "Not Active", "Not Active", "Not Active", "Not Active"]),
        (11.4, ["0", "2070", "2070", "940", "Not Active", "Not Active", "Not Active", "Active"]),
        (20.0, ["0", "1500", "2070", "300", "Active", "Not Active", "Not Active", "Not Active"]),  # after
    ]
    c.rows = rows
    s = c.summary(10.5, 11.5)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s = c.summary(0.0, 30.0)
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"] and s["samples"] == 5 and s["sm_mhz"] == 2055.0
    c.rows = []
    assert c.summary(0.0, 1.0) is None


def test_fp32_peak():
    assert bench.peak_fp32_tflops(152, 2070) == pytest.approx(80.54784)


def test_traffic_lookup_needs_the_measured_tiling_and_source():
    h = bench.far_source_hash()
    for key, val in bench.NCU_TRAFFIC.items():
        src, tiling, split, tile, mb = key.split("/")
        th, tpt = tiling.split("x")
        t = {"threads": int(th), "targets_per_thread": int(tpt), "split": int(split), "tile": int(tile),
             "min_blocks": int(mb[2:])}
        assert bench.ncu_traffic(t) == (val if src == h else None)
        assert bench.ncu_traffic(dict(t, split=int(split) + 1)) is None
        assert bench.ncu_traffic(dict(t, min_blocks=int(mb[2:]) + 1)) is None
    assert bench.ncu_traffic({}) is None


def _run_reference(env_extra):
    env = dict(os.environ, OMP_NUM_THREADS="1", **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "1"], capture_output=True, text=True, env=env, timeout=600)


def test_reference_arm_prints_the_oracle_line():
    r = _run_reference({"RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "s"
    assert line["higher_is_better"] is False and line["value"] > 0
    assert line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == bench.host_cores() and cb["value"] == line["value"]
    assert cb["sample"]
    # value = 4 x the mean quarter-apply step x the oracle solve's operator applies
    gs = bench.golden_solve()
    assert line["value"] == pytest.approx(4 * line["ms_per_step"] / 1e3 * gs["operator_applies"])
    assert line["ms_per_step"] * (line["steps"] + line["warmup"]) < 600e3
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_on_other_ranks():
    r = _run_reference({"RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_self_vsh_rate():
    prof = {"launches": {"self": 63}, "ms": {"self": 4.33}}
    r = bench.self_vsh_rate(prof, 61952)
    assert r["bytes_per_apply"] == 2 * 3 * 61952 * 8
    assert r["ms_per_apply"] == pytest.approx(4.33 / 63)
    assert r["gb_per_s"] == pytest.approx(2 * 3 * 61952 * 8 * 63 / 4.33e-3 / 1e9)
    assert bench.self_vsh_rate({"launches": {"self": 0}, "ms": {"self": 0.0}}, 10) is None
    assert bench.self_vsh_rate({"launches": {}, "ms": {}}, 10) is None


def test_stage_rooflines_from_a_profile():
    """Each stage's achieved rate is its algorithmic work over its profiled time."""
    prof = {"ms": {"near": 10.0, "completion": 5.0, "arnoldi": 4.0, "self": 2.0, "precond": 3.0},
            "launches": {"near": 50, "completion": 50, "self": 50, "precond": 40},
            "arnoldi_vectors": 1000}
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "source": "measured"}
    n, p, near, pairs = 256, 10, 1118, 559
    r = bench.stage_rooflines(prof, n, p, near, pairs, 80.0, peaks)
    npn = 242
    assert r["near"]["achieved"] == pytest.approx(near * npn * 3 * 121 * 20 * 50 / 10e-3 / 1e12)
    assert r["completion"]["achieved"] == pytest.approx(n * npn * n * 32 * 50 / 5e-3 / 1e12)
    assert r["arnoldi"]["achieved"] == pytest.approx(1000 * 3 * n * npn * 8 / 4e-3 / 1e9)
    assert r["arnoldi"]["frac"] == pytest.approx(r["arnoldi"]["achieved"] / 6000.0)
    assert r["self"]["peak"] == pytest.approx(2000.0 * 1.1 / 2.25)
    assert r["self"]["achieved"] == pytest.approx(3 * 2 * 726 * 726 * n * 50 / 2e-3 / 1e12)
    assert r["precond"]["bytes_per_apply"] > pairs * 146 * 146 * 4
    assert bench.stage_rooflines({"ms": {}, "launches": {}}, n, p, near, None, 80.0, peaks) == {}
