"""The benchmark's reference arm (the FP64 CPU oracle on bounded column samples) runs on the
host alone and prints one JSON line with the keys the benchmark contract asks for."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *extra],
                       capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env={k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_json_line():
    d = _run("--steps", "2", "--warmup", "0", "--ref-columns", "8", "--workload", "water32")
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "density matrices/s" and d["steps"] == 2 and d["n_gpus"] == 1
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) <= 1e-9 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "8 of 32" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("32 water-like molecules")


def test_reference_arm_other_ranks_print_nothing():
    env = {k: v for k, v in os.environ.items()}
    env.update(RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "water32"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT, env=env)
    assert r.returncode == 0 and not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def _bench_module():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_records_follow_the_kernel_source():
    # The roofline's `traffic` comes from a committed ncu record only while the record's hash
    # names the current kernel source; a shard record is scaled by the launch's GEMM count.
    b = _bench_module()
    rec = json.load(open(os.path.join(ROOT, "profiles", "ns_tc_traffic.json")))
    by = {r["workload"]: r for r in rec["records"]}
    t, note = b._profiled_traffic("water1024", "fp16x3", 1.0)
    if t is not None:  # the record matches the source: the launch's bytes as recorded
        assert t == by["water1024"]["dram_bytes_read"] + by["water1024"]["dram_bytes_write"]
        c3 = by["water4096x23"]
        t3, note3 = b._profiled_traffic("water4096x23", "fp16x3", 2.0 * c3["gemms"])
        if t3 is not None:
            assert abs(t3 - 2.0 * (c3["dram_bytes_read"] + c3["dram_bytes_write"])) <= 1e-6 * t3
            assert "scaled" in note3
    else:
        assert note == "kernel changed since the ncu capture"
    assert b._profiled_traffic("water1024", "fp16", 1.0) == (None, "no ncu record for this precision")
    assert b._profiled_traffic("slab6000", "fp16x3", 1.0)[0] is None
