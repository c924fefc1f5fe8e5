"""The bench's reference arm (the oracle on the host cores) runs on CPU: its
JSON line carries the contract's keys, and under torchrun only rank 0 works
and prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "grid48",
        "--steps", "1", "--warmup", "3"]


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run(ARGS, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_line_has_the_contract_keys():
    p = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["unit"] == "trees/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"].startswith("grid48")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "trees/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC


def test_reference_arm_other_ranks_exit_without_work():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_per_class_bounds_match_the_library():
    """bench.py --per-class groups the batch by the library's size classes."""
    import re
    sys.path.insert(0, ROOT)
    import bench
    src = open(os.path.join(ROOT, "paper_2006_13679_gb300", "csrc", "ust_common.cuh")).read()
    consts = {m.group(1): m.group(2) for m in re.finditer(r"constexpr int (\w+) = ([^;]+);", src)}
    body = re.search(r"kClassMaxN\[kNumClasses\] = \{([^}]*)\}", src).group(1)
    bounds = tuple(int(eval(consts.get(t.strip(), t.strip()), {})) for t in body.split(","))
    assert bounds == bench.BATCH_CLASS_MAX_N
    assert len(bounds) == int(consts["kNumClasses"])


def test_traffic_capture_follows_the_sampler_code():
    """The DRAM traffic a capture measured is reported only while the
    sampler's code (comments left out) hashes as it did then: a comment edit
    keeps it, a code edit drops it, and other workloads never get it."""
    sys.path.insert(0, ROOT)
    import bench

    sha = bench.sampler_sha1()
    assert sha is not None
    caps = [c for c in bench.TRAFFIC_CAPTURES if c["sha1"] == sha and "rmat22" in c["applies_to"]]
    n, trees = 2394915, 9475
    t = bench.traffic_per_launch("rmat22", n, trees)
    if caps:
        assert t == caps[0]["bytes_per_vertex_tree"] * n * trees
    else:
        assert t is None  # the code changed since the capture: no traffic figure
    assert bench.traffic_per_launch("hyperbolic20", n, trees) is None
    code = "int a; // one\n/* two\n three */ int b;\n\nint c;  // four\n"
    assert bench.code_of(code) == "int a;\n int b;\nint c;"
    assert bench.code_of(code.replace("one", "uno")) == bench.code_of(code)
    assert bench.code_of(code.replace("int c", "int d")) != bench.code_of(code)
