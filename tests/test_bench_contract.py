"""The reference arm of bench.py (the CPU oracle, no GPU): one JSON line with the keys the
benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    # the small star tree (same node shapes as the 4 x 20 tree) keeps this CPU test short; the
    # line's keys are the same for every workload
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "sf_5state_4x4_d10_D20"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"] == "sf_5state_4x4_d10_D20"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["nproc"] >= 1 and cb["cpu_model"]
    assert cb["single_thread"] > 0 and cb["all_threads"] > 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_default_workload_is_the_largest_single_gpu_configuration():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.HEADLINE == "sf_er_5state_8x60_d20_D40"
    p = bench.make_problems(bench.HEADLINE)[0]
    assert p.er_tree and len(p.envs) == 8 and all(e.L == 60 and e.d == 20 and e.D == 40 for e in p.envs)
    assert p.dt == 0.25 and bench.WORKLOADS[bench.HEADLINE]["prec"] == "bf16x3"
