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


def test_kernel_table_keeps_side_stream_launches_out_of_the_shares():
    """The per-kernel table: average launch time x launches per step, shares
    of the summed time; a launch on the side stream (the eigensolver's partial
    wave, whose events include its wait for free SMs) is listed last, without
    a share."""
    import bench
    kprof = {"kb_trail (x)": (30.0, 3, 6), "k_heev (x)": (1000.0, 1, 1),
             "k_heev_tail (x)": (1500.0, 1, 1), "kb_panel": (1.0, 2, 4)}
    rows = bench.kernel_table(kprof, steps=2)
    names = [r["kernel"] for r in rows]
    assert names[0] == "k_heev (x)" and names[-1] == "k_heev_tail (x)"
    assert rows[-1]["share"] is None
    tot = 500.0 + 30.0 + 1.0            # per step: 1000 x 1 / 2, 10 x 6 / 2, 0.5 x 4 / 2
    assert abs(rows[0]["share"] - 500.0 / tot) < 1e-12
    assert abs(sum(r["share"] for r in rows[:-1]) - 1.0) < 1e-12


def test_algorithmic_counts():
    """The roofline's algorithmic counts: the eigensolver's (16/3 + 6 x 0.97 +
    8) n^3 flops per matrix, an overlap's n^3 complex multiply-adds, and the
    sweep's per-kind totals add up to the per-point formula (the trailing
    update's n^3/3 and the back substitution's n^2 (n + n_c)/2 multiply-adds
    among them)."""
    import bench
    n = 512
    assert abs(bench.heev_flops_per_matrix(n) - (16 / 3 + 5.82 + 8) * n ** 3) < 1e-6 * n ** 3
    assert bench.overlap_flops_per_pair(n) == 8.0 * n ** 3
    nc, npts, N = 8, 4, 3
    tot = bench.sweep_kind_totals(n, nc, npts, N, False, 8)
    flops = sum(f for (f, _) in tot.values())
    # [W|Y] on N interfaces; LU (panel, panel apply, trailing) and back
    # substitution on N + 1, 8 flop per complex multiply-add
    lu_tri = (n ** 3 / 3.0 + n * n * (n + nc) / 2.0) * 8.0 * (N + 1) * npts
    assert flops > 8.0 * 2 * n ** 3 * N * npts + 0.9 * lu_tri
    assert tot["kb_trail"][1] > 0 and tot["kb_bsupd"][1] > 0


def test_paired_blocks_move_fewer_bytes_for_the_same_updates():
    """Panels and back-substitution blocks in pairs (the tensor-core form):
    the LU does the same multiply-adds as one panel at a time, with the first
    panel's update of the second panel's 32 rows moved from the trailing
    update into the second panel's apply; the back-substitution updates do
    the same multiply-adds; the wide read-modify-write passes happen about
    half as often, so their bytes drop by nearly half.  Ragged sizes keep the
    identities."""
    import bench
    nc, npts, N = 8, 2, 1
    for n in (64, 96, 100, 512):
        one = bench.sweep_kind_totals(n, nc, npts, N, False, 8, paired=False)
        two = bench.sweep_kind_totals(n, nc, npts, N, False, 8, paired=True)
        lu1 = one["kb_trail"][0] + one["kb_panel_apply"][0]
        lu2 = two["kb_trail"][0] + two["kb_panel_apply"][0]
        assert abs(lu1 - lu2) <= 1e-9 * lu1, n
        assert two["kb_panel_apply"][0] > one["kb_panel_apply"][0]
        assert abs(one["kb_bsupd"][0] - two["kb_bsupd"][0]) <= 1e-9 * one["kb_bsupd"][0], n
        # (at n = 64 the back substitution's one pair is the one update)
        assert two["kb_trail"][1] < one["kb_trail"][1], n
        assert two["kb_bsupd"][1] < one["kb_bsupd"][1] or (n == 64 and two["kb_bsupd"] == one["kb_bsupd"]), n
        assert two["kb_panel"][0] == one["kb_panel"][0]
    one = bench.sweep_kind_totals(512, nc, npts, N, False, 8, paired=False)
    two = bench.sweep_kind_totals(512, nc, npts, N, False, 8, paired=True)
    assert 0.45 < two["kb_trail"][1] / one["kb_trail"][1] < 0.6
