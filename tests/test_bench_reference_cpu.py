"""The reference arm of bench.py (the FP64 oracle on the host cores) keeps the
JSON-line contract: one line on rank 0 with the metric, value, units, timing,
cpu_baseline and e2e keys; other ranks exit 0 without work."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
           "--steps", "2", "--warmup", "1"]
    return subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["unit"] == "TFLOP/s"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("L8_N8_Sz0_M64")


def test_reference_arm_loads_no_library():
    """The oracle arm times the oracle alone: the GPU library is never loaded."""
    code = ("import runpy, sys\nsys.argv = ['bench.py', '--impl', 'reference', '--workload', 'c1', "
            "'--steps', '1', '--warmup', '0']\n"
            "try:\n    runpy.run_path('bench.py', run_name='__main__')\nexcept SystemExit as e:\n"
            "    assert not e.code\n"
            "import sys as _s\n"
            "maps = open('/proc/self/maps').read()\n"
            "assert 'libdmrg_gb300' not in maps, 'library loaded'\n"
            "assert 'paper_2001_04890_gb300.binding' not in _s.modules\n"
            "print('CLEAN')")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env=dict(os.environ, RANK="0", WORLD_SIZE="1"))
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip().splitlines()[-1] == "CLEAN"


def test_large_workload_reference_arm_times_the_oracle_on_its_own_workload():
    """For workloads whose blocks the oracle cannot build on the host, the reference
    arm names the workload it timed instead."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c5a",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["config"]["workload"].startswith("L24_N24_Sz0_M512")
    assert "cannot build the L76_N113_Sz1_M3000" in d["config"]["step"]


def test_reference_arm_other_ranks_do_nothing():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_sweep_summary_takes_every_site_once():
    """The sweeps mode's entropy summary reads site s from a step whose two sites include s."""
    import importlib.util
    import numpy as np
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for L in (3, 6, 9):
        positions = list(range(0, L - 2)) + list(range(L - 2, 0, -1))   # one sweep, both directions
        rec = {"entropies": np.array([[k, k + 1, -1.0] for k in positions], dtype=float)}
        assert bench._site_entropies(rec, L) == [float(s) for s in range(L)]


def test_launch_shape_keys_match_the_recorded_traffic():
    """A fixed launch shape given on the command line (five or six numbers) maps to
    the key of the recorded DRAM traffic, and every workload with recorded
    tensor-core traffic also has its algorithmic bytes."""
    import bench
    t5 = bench._fixed_tune("8192,200000,1,1,1")
    t6 = bench._fixed_tune("8192,200000,1,1,1,0")
    assert t5 == t6 and t6["tc_tiny"] == 0 and bench._fixed_tune("8192,200000,1,1,1,1")["tc_tiny"] == 1
    assert ("c5b", 2, 6000, bench._shape_key(t5)) in bench.TRAFFIC_PER_LAUNCH
    for (wl, prec, M, shape) in bench.TRAFFIC_PER_LAUNCH:
        assert len(shape) == 6 and M == bench.WORKLOADS[wl]["M"]
        if prec == 2:
            assert wl in bench.ALG_BYTES and bench.ALG_BYTES[wl] < bench.TRAFFIC_PER_LAUNCH[(wl, prec, M, shape)]
