"""Host logic of the benchmark (no GPU): the comment-insensitive kernel-source hash that keys the
committed DRAM-traffic record, the traffic lookup, the flop model, and the reference arm's JSON line
(the oracle timed on host cores) on the small workload."""

import json
import math
import subprocess
import sys
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_only_ignores_comments_and_layout():
    a = "int f(int x) {  // one\n  return x + 1; /* two\n lines */ }\n"
    b = "int f(int x) { return x + 1; }  // other words"
    c = "int f(int x) { return x + 2; }"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def test_traffic_record_applies_only_to_the_hashed_sources(monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    entry = rec["4det-60min-2048Hz"]["pass_a"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: entry["kernel_hash"])
    assert bench.ncu_traffic("pass_a", "4det-60min-2048Hz") == entry["bytes_per_launch"]
    assert entry["bytes_per_launch"] == entry["read"] + entry["write"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic("pass_a", "4det-60min-2048Hz") is None
    assert bench.ncu_traffic("pass_a", "no-such-workload") is None


def test_flop_model():
    n, d, nb = 1 << 23, 4, 3973120
    got = bench.flop_per_eval(n, d, nb)
    assert got == 2 * 5 * n * 23 + nb * (14 * d + 20) + 12 * n + 4 * n
    assert 2.3e9 < got < 2.4e9
    assert math.isclose(bench.FP32_PEAK_TFLOPS, 80.55, rel_tol=1e-3)


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "small-4det-4096", "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["steps"] == 2 and out["warmup"] == 1 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["value"] == out["value"]


def test_uneven_segments_cycle_15_30_60_minutes():
    lengths = [bench._segment_workload(s, (1.4, 1.6, 12.0)) for s in range(6)]
    assert [w.n_fft for w in lengths] == [1 << 21, 1 << 22, 1 << 23] * 2
    assert [w.n_samples for w in lengths[:3]] == [15 * 60 * 2048, 30 * 60 * 2048, 60 * 60 * 2048]
    assert all(w.n_samples <= w.n_fft and w.fs == 2048.0 for w in lengths)
    assert lengths[0].m1 == 1.4 and lengths[0].m2 == 1.6 and lengths[0].snr == 12.0


def test_oracle_judgements_report_fitness_and_argmax():
    import synthdata as sd
    from oracle import fcas_oracle as o
    w = sd.SMALL
    th = sd.make_particles(w, 2, seed=5)
    got = bench.oracle_judgements({"pts": (w.name, 5, {}, th.tolist())})
    data = sd.make_dataset(w, seed=5)
    setup = o.OracleSetup(data["det"], data["psd"], data["data"], w.n_fft, w.fs, w.f_low, w.f_high)
    for (v, t), p in zip(got["pts"], th):
        assert (v, t) == o.fitness(setup, p)


def test_traffic_record_is_the_stated_scaling_of_its_capture():
    """The committed DRAM record holds 64-particle launches scaled from 8-particle captures of one
    kernel each: pass A's spectrum and basis reads once per launch, its intermediate writes times 8;
    pass B's intermediate reads times 8, its writes as captured. Both records come from one set of
    kernel sources, and each read/write is at least the algorithmic bytes of what it scales."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))["4det-60min-2048Hz"]
    a, b = rec["pass_a"], rec["pass_b"]
    assert a["kernel_hash"] == b["kernel_hash"]
    scale = a["particles_per_launch"] // a["captured"]["particles"]
    assert scale == 8 and b["particles_per_launch"] // b["captured"]["particles"] == scale
    assert a["read"] == a["captured"]["read"] and a["write"] == scale * a["captured"]["write"]
    assert b["read"] == scale * b["captured"]["read"] and b["write"] == b["captured"]["write"]
    per_particle = (1 << 23) * 16                      # one particle's intermediate, FP32 form
    assert 0.9 * 64 * per_particle <= a["write"] <= 1.01 * 64 * per_particle
    assert 64 * per_particle <= b["read"] <= 1.01 * 64 * per_particle
