"""bench.py's JSON line on the CPU: the reference arm (the oracle timed on a
bounded sample) prints the contract's keys with the same metric and workload
config as the GPU arm, and the launch-count helper adds up."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "points/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("junction512: AB junction, N_G=512, 320 slices, 128 E x 32 k_par")


def test_refine_launch_count():
    sys.path.insert(0, ROOT)
    import bench
    # init + finish, a backward pass of bw launches per interface, per pass a residual and a
    # forward pass (2N+1 launches), and a backward pass after every pass but the last
    N = 10
    for batched, bw in ((True, 3), (False, 2)):
        assert (bench.refine_launches(N, 2, batched, sliced=False)
                == 2 + bw * (N + 1) + 2 * (2 * N + 2) + bw * (N + 1))
    # the residual as slice products: four launches per interface in place of one
    assert (bench.refine_launches(N, 2, True, sliced=True)
            == bench.refine_launches(N, 2, True, sliced=False) + 2 * (4 * (N + 1) - 1))
    assert bench.refine_launches(N, 0) == 0
