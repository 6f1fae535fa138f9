"""bench.py --impl reference (the oracle timed on the host cores) prints the
one JSON line of the benchmark contract: the same metric, unit, direction and
workload config as the GPU arm, with cpu_baseline and e2e filled in; and
--gpus 2 outside torchrun starts two ranks itself (gloo here, no GPU), of
which rank 0 alone prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.join(os.path.dirname(__file__), "..")


def _run(*extra, timeout=600):
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--cpu-seconds", "0.3", "--grid", "31", *extra],
                         capture_output=True, text=True, timeout=timeout, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_prints_the_contract_line():
    d = _run()
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "s"
    assert d["higher_is_better"] is False and d["n_gpus"] == 1
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    c = d["config"]
    assert c["n"] == 25230 and "31x31x32" in c["workload"] and "sym storage, fp32_ru, tol 1e-10" in c["workload"]


def test_default_workload_is_the_largest_single_gpu_system():
    import bench
    sys.argv = ["bench.py"]
    a = bench.parse()
    assert (a.grid, a.format, a.precision) == ("256", "sym", "fp32_ru")
    g = bench.GRIDS[a.grid]
    assert (g.nx, g.ny, g.nz, g.n_incl) == (256, 256, 256, 4)


def test_two_ranks_started_without_torchrun():
    d = _run("--gpus", "2", timeout=900)
    assert d["impl"] == "reference" and d["n_gpus"] == 2
