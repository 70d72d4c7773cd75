"""The bench's reference arm (the FP64 oracle timed on the host cores) keeps the
JSON-line contract on the CPU: one line from rank 0 with the keys the measured
arm also prints, and nothing from the other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--dims", "4", "4", "4", "4",
           "--steps", "2", "--warmup", "1"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_json_line():
    p = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is False
    assert d["value"] > 0 and d["unit"] == "s"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["lattice"] == [4, 4, 4, 4]
    # the measured arm prints the same config object for the same workload
    sys.path.insert(0, ROOT)
    import bench

    assert d["config"] == bench.workload_config((4, 4, 4, 4), bench.MASS, 1)
    assert d["cpu_baseline"]["host_cpu"] and d["cpu_baseline"]["host_logical_cores"] >= 1


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_all_core_oracle_timing_reproduces_the_oracle():
    """The host-core timing splits the lattice into t-slabs, one process each, and applies the
    oracle's A, unchanged, to every slab widened by the reach of A (6 t-slices with Naik);
    the interior rows put together are the oracle's A on the whole lattice."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1010_4782_gb300 import inputs

    dims = (4, 4, 2, 32)
    fat, lng = inputs.asqtad_form_fields(dims)
    b = inputs.gaussian_even_source(dims, 0)
    per_a, w, y = bench.oracle_apply_A_all_cores(fat, lng, b, dims, 0.1, reps=1)
    assert w >= 2 or (os.cpu_count() or 1) < 2
    assert per_a > 0
    ref = oracle.Operator(fat, lng, 0.1, dims).apply_A(b)
    assert np.array_equal(y, ref)


def test_recorded_traffic_matches_the_kernel_sources():
    """Every ncu traffic figure the bench reports was captured from the kernel
    sources as they stand: a kernel edited since its capture would make the bench
    report `traffic: null`, so the capture must be repeated with the edit."""
    sys.path.insert(0, ROOT)
    import bench

    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        recorded = json.load(f)
    assert recorded
    for key, entry in recorded.items():
        files = bench.MULTI_SOURCES if key.startswith("multi_") else bench.DSLASH_SOURCES
        assert entry["source_hash"] == bench.dslash_source_hash(files), key
        assert entry["dram_bytes_per_launch"] > 0 and entry["how"], key
        assert bench.recorded_traffic(key, files) == float(entry["dram_bytes_per_launch"]), key
