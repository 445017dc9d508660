"""Throughput benchmark of the transmission hot path.

Workload (one GPU): the synthetic AB side-contact junction with N_G = 512
plane waves and 320 slices, 128 energies x 32 k_par points (4096 (E, k_par)
points).  One step = one k_par point with all its 128 energies: the slice
Hamiltonians, their eigenmodes and interface overlaps for that k_par, then
the left-to-right star-product sweep over all 321 interfaces for the 128
points, and T = Tr(t^H t).  Metric: (E, k_par)-points/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
    python bench.py --impl reference   # the CPU oracle on the host cores
    python bench.py --config uneven [--instances K]   # uneven-batch form
    python bench.py --config grad [--grad-points P]   # adjoint form (FP64)
    python bench.py --config scan                     # second workload (Tbar scans)
    python bench.py --config modes [--slices N]       # the mode stage alone (FP64)
    python bench.py --composition doubling --instances P   # Eq. recurrence2 (FP64)

The uneven-batch line times pw_transmission_batch over the first K of the
2048 seeded instances of uneven N_G (128..768) and slice count (60..400), one
(E, k_par) point each; a step is one call over those K instances.

Under torchrun each rank takes its own k_par points (weak scaling, no data
exchange); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synthetic import junction, minimal_cell, uneven_batch  # noqa: E402

METRIC = "(E,k∥)-points/s at N_G=512, 320 slices: mixed-precision vs FP64, at 1e-8 rel T"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
GOLDEN_512 = os.path.join(ROOT, "tests", "golden", "junction512_k5.json")
# every 11th launch of each kernel kind is bracketed by CUDA events: a prime, so that
# the sample walks through every position of the per-interface launch patterns (15
# trailing and back-substitution updates, 16 panels, applies and diagonal blocks, 8
# overlap chunks), with few events in the timed region
PROFILE_STRIDE = 11
MIXED_DEFAULT_VARIANT = 2    # the library's default launch variant of the mixed form
T_FLOOR = 1e-6          # relative error of T is taken against max(|T|, T_FLOOR)
# DRAM traffic of kernels captured with ncu: dram__bytes_read + dram__bytes_write of the
# captured launches over their algorithmic bytes (profiles/kb_trail_tc_junction512_small.md,
# panels in pairs: 596.3/626.5, 20.0/29.4, 437.0/474.5 MB); the roofline's `traffic` is this
# ratio times the step's average algorithmic bytes per launch.  A kernel changed since its
# capture has no entry.
KERNEL_TRAFFIC = {"kb_trail": 0.93}
# DRAM bytes per matrix of the FP64 eigensolver from its ncu capture (64 matrices of
# N_G = 512, one launch: 186.2 + 152.3 MB, profiles/k_heev_junction512_64matrices.md);
# the roofline's `traffic` is this times the matrices of the timed launch
KERNEL_TRAFFIC_PER_MATRIX = {"k_heev": (186.19e6 + 152.32e6) / 64}
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def workload(name):
    if name == "junction512":
        return junction(ng=512, n_slices=320, n_e=128, n_k=32), 128, 32
    if name == "junction401":
        return junction(ng=0, ecut=29.34, n_slices=240, n_e=128, n_k=32), 128, 32
    if name == "junction48":
        return junction(ng=48, n_slices=16, n_e=128, n_k=32), 128, 32
    if name == "minimal":
        inst = minimal_cell(energies=np.linspace(0.3, 6.0, 128),
                            kpar=np.zeros((128, 2)))
        return inst, 128, 1
    raise ValueError(name)


def shard_kpoints(rank, world, n_k, n_steps, first_step=0):
    """k_par indices processed by `rank` in steps first_step .. first_step+n_steps-1:
    step s of rank r takes k = (r + s * world) mod n_k, so the ranks of one step
    hold disjoint k_par points (weak scaling: each rank has a full step)."""
    return [(rank + (first_step + s) * world) % n_k for s in range(n_steps)]


def instance_weight(inst):
    """Work of one uneven-batch instance, n^3 (N_s + 1): the sweep's GEMM and LU
    cost per interface times its interfaces."""
    n = inst.ng_exact if inst.ng_exact > 0 else 0
    return float(n) ** 3 * (inst.n_slices + 1)


def shard_instances(weights, rank, world):
    """Indices of the instances rank `rank` of `world` evaluates: the
    instances, largest weight first, each go to the rank with the least
    weight so far (lowest rank on ties), so every rank gets a disjoint set and
    the ranks' total weights differ by at most the largest single weight."""
    load = [0.0] * world
    mine = []
    for i in sorted(range(len(weights)), key=lambda j: (-weights[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += weights[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def reduce_sum(values, world, device):
    """Sum over ranks of a vector of doubles (the host-side exchange of the
    summed transmission and of the gradient)."""
    import torch
    t = torch.as_tensor(np.asarray(values, dtype=np.float64).reshape(-1), device=device).clone()
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def reduce_max(value, world, device):
    """Max over ranks of a scalar (the slowest rank's time sets the job time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


QL_ROTATIONS_PER_N2 = 0.97


def heev_flops_per_matrix(n):
    """Algorithmic flops of one Hermitian eigendecomposition by the tridiagonal
    route: Householder reduction 16/3 n^3; implicit QL, about 0.97 n^2
    rotations (counted on the CPU for the tridiagonal forms of four junction
    slices at N_G = 512), each 6 flops on every row of the real eigenvector
    matrix; back-transformation of n vectors 8 n^3."""
    return (16.0 / 3.0 + 6.0 * QL_ROTATIONS_PER_N2 + 8.0) * n ** 3


def overlap_flops_per_pair(n):
    """O_p = U_p^H U_{p+1}: n^3 complex multiply-adds, 8 flops each."""
    return 8.0 * n ** 3


# kernel kinds whose launches run beside others on a side stream: their event
# times include the wait for free SMs and are kept out of the kernel-time shares
OVERLAPPED_KINDS = ("k_heev_tail",)
# kernel kinds that run in FP64 in both forms (the mixed form's modes and
# overlaps are FP64 unless sweep variant bit 5 selects double-float)
FP64_KINDS = ("k_heev", "k_overlaps")


def refine_launches(N, iters, batched=True, sliced=True):
    """Launches of the mixed form's refinement: init; a backward pass; per pass
    the residual and a forward pass (fwd_b at every interface, fwd_a after the
    first), then (except after the last pass) a backward pass; the finish.  A
    backward step is bwd_a + bwd_b per interface, or bwd_a, the batched
    tensor-core product and its combine when every point of the launch shares
    its overlaps (one k_par per step here).  The residual is one launch, or,
    as exact slice products on the tensor cores (shared overlaps, N_G a
    multiple of 4 up to 512), four per interface (slice O, slice y, product,
    combine)."""
    if iters <= 0:
        return 0
    bw = 3 if batched else 2
    res = 4 * (N + 1) if sliced else 1
    return 2 + bw * (N + 1) + iters * (res + 2 * N + 1) + (iters - 1) * bw * (N + 1)


def sweep_flops_per_point(n, nopen_left):
    """Algorithmic flops of one interface step of the sweep for one point:
    R [Q | P] (2 n^3 complex multiply-adds), LU of W (n^3 / 3), forward and
    back substitution on n + n_open right-hand sides (n^2 (n + n_open));
    8 real flops per complex multiply-add."""
    return 8.0 * (2.0 * n ** 3 + n ** 3 / 3.0 + n * n * (n + nopen_left))


def sweep_kind_totals(n, nc, npts, N, big, esz, paired=False):
    """Algorithmic work of one step's sweep per kernel kind (all N+1
    interfaces, npts points): {kind: (flops, bytes)}.  CMA = 8 flop.  Bytes are
    what each launch must move at least: the matrix region it updates read and
    written once, its operands read once.  `big` (sweep variant bit 3):
    LAPACK-ordered pivots, the LU updates W's columns only, the right-hand
    sides n + nc eliminated in 128-row blocks after the LU; else 32-row
    blocks, the LU's trailing updates carry all 2n + nc columns.  `paired`
    (the tensor-core form without bit 3): the LU's 32-column panels in pairs,
    the first panel's update reaching only the second panel's columns and its
    32 rows (in the second panel's apply), the rest with K = 64; and the back
    substitution's 32-row blocks in pairs from the bottom, a 32-row update
    inside each pair and one update of the rows above it with K = 64."""
    NB, FB = 32, 128
    ncols, nrhs = 2 * n + nc, n + nc
    ucols = n if big else ncols
    tr_f = tr_b = pa_f = pn_f = 0.0

    def trail(r0, c0, k, cend):   # M[r0:n, c0:cend] -= (rows x k) (k x cols)
        nonlocal tr_f, tr_b
        rows, cols = n - r0, cend - c0
        tr_f += rows * cols * k
        tr_b += esz * (2.0 * rows * cols + rows * k + k * cols)
    j0 = 0
    while j0 < n:
        nb = min(NB, n - j0)
        c0 = j0 + nb
        pn_f += (n - j0) * nb * nb / 2.0
        pa_f += nb * nb / 2.0 * (ucols - c0)
        if paired and c0 < n:
            j1, nb2 = c0, min(NB, n - c0)
            c1 = j1 + nb2
            trail(j1, j1, nb, c1)                                 # the second panel's columns
            pn_f += (n - j1) * nb2 * nb2 / 2.0
            pa_f += (nb2 * nb + nb2 * nb2 / 2.0) * (ucols - c1)   # its 32 rows, then the solve
            if c1 < n:
                trail(c1, c1, nb + nb2, ucols)
            j0 = c1
            continue
        if c0 < n:
            trail(c0, c0, nb, ucols)
        j0 = c0
    bs = FB if big else NB
    up_f = up_b = dg_f = fs_f = fs_b = fd_f = 0.0

    def update(rows, k):   # rows x nrhs -= (rows x k) (k x nrhs)
        nonlocal up_f, up_b
        up_f += rows * nrhs * k
        up_b += esz * (2.0 * rows * nrhs + rows * k + k * nrhs)
    for j0 in range(0, n, bs):
        fb = min(bs, n - j0)
        dg_f += fb * fb / 2.0 * nrhs
        if j0 > 0 and not paired:
            update(j0, fb)
        if big:
            fd_f += fb * fb / 2.0 * nrhs
            c1 = j0 + fb
            if c1 < n:
                fs_f += (n - c1) * nrhs * fb
                fs_b += esz * (2.0 * (n - c1) * nrhs + (n - c1) * fb + fb * nrhs)
    if paired:
        jb = ((n - 1) // NB) * NB
        while jb > 0:
            j0 = jb - NB
            kb = min(NB, n - jb)
            update(NB, kb)              # block b-1 from block b
            if j0 > 0:
                update(j0, NB + kb)     # the rows above the pair
            jb = j0 - NB
    I = (N + 1) * npts
    out = {
        "kb_wy": (8.0 * 2 * n ** 3 * N * npts, esz * (n * n + 2.0 * n * n) * N * npts),
        "kb_trail": (8.0 * tr_f * I, tr_b * I),
        "kb_panel": (8.0 * pn_f * I, None),
        "kb_panel_apply": (8.0 * pa_f * I, None),
        "kb_bsupd": (8.0 * up_f * I, up_b * I),
        "kb_bsdiag": (8.0 * dg_f * I, None),
    }
    if big:
        out["kb_fsupd_tc"] = (8.0 * fs_f * I, fs_b * I)
        out["kb_fsdiag"] = (8.0 * fd_f * I, None)
    return out


def kernel_table(kprof, steps):
    """Per-kernel totals of the timed region from the library's sampled CUDA
    events: average launch time of the timed launches x all launches."""
    rows = []
    for name, (ms, timed, launches) in kprof.items():
        if timed <= 0:
            continue
        avg = ms / timed
        rows.append({"kernel": name, "launches_per_step": launches / steps, "avg_launch_ms": avg,
                     "ms_per_step": avg * launches / steps, "timed_launches": timed})
    side = [r for r in rows if r["kernel"].split(" ")[0] in OVERLAPPED_KINDS]
    rows = [r for r in rows if r not in side]
    tot = sum(r["ms_per_step"] for r in rows) or 1.0
    for r in rows:
        r["share"] = r["ms_per_step"] / tot
    rows.sort(key=lambda r: -r["ms_per_step"])
    for r in side:
        r["share"] = None
        r["note"] = "side stream, overlapped; time includes the wait for free SMs"
    return rows + side


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, device_index=0):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.p = None
        self.dev = device_index

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax = float(r[1])
                for nm, v in zip(names, r[4:8]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_oracle_rate(inst, n_e, sample_ifaces=24, sample_slices=24):
    """Points/s of the CPU oracle, timed on a bounded sample of one point:
    `sample_slices` slice eigendecompositions (amortised over the n_e energies
    of a k_par, as in the workload) and `sample_ifaces` interface S-matrices
    with their star products, scaled to all N+2 slices and N+1 interfaces."""
    from oracle import pw_oracle as O
    m = O.Model(inst)
    k = inst.kpar[0]
    E = float(inst.energies[min(n_e // 2, len(inst.energies) - 1)])
    tabs = m.all_tables()
    t0 = time.perf_counter()
    modes = [O.slice_modes(O.hamiltonian(m.mn, m.G, k, tabs[q], m.half))
             for q in range(sample_slices + 1)]
    t_eig = (time.perf_counter() - t0) / (sample_slices + 1)
    S = O.identity_s(m.n)
    t0 = time.perf_counter()
    for p in range(sample_ifaces):
        S = O.star(S, m.interface_s(modes, E, p))
    t_if = (time.perf_counter() - t0) / sample_ifaces
    per_point = t_if * (m.N + 1) + t_eig * (m.N + 2) / n_e
    return 1.0 / per_point, {
        "sample": f"1 point: {sample_slices + 1} slice eigendecompositions and {sample_ifaces} "
                  f"interface S + star products of N_G={m.n}, scaled to {m.N + 2} slices "
                  f"(amortised over {n_e} energies) and {m.N + 1} interfaces",
        "seconds_per_point": per_point, "n": m.n, "N": m.N}


def golden_junction512():
    """Stored oracle T of the 128 energies at one k_par of the N_G = 512,
    320-slice junction (None when the file is absent)."""
    try:
        with open(GOLDEN_512) as f:
            return json.load(f)
    except OSError:
        return None


def fp64_sample(pw, torch, inst, n_e, stream, gold, npts):
    """The plain FP64 GPU form on a bounded sample of one step: `npts`
    energies of one k_par through the whole path (eigenmodes and overlaps of
    the k_par in FP64, the FP64 sweep), timed with CUDA events.  Points/s for
    a full step of n_e energies = n_e / (mode stage + n_e x sweep time per
    point); the sampled T are compared with the stored oracle values."""
    kk = gold["k_index"] if gold is not None else 0
    sel = np.unique(np.linspace(0, n_e - 1, npts).astype(int))
    idx = kk * n_e + sel
    with pw.Context.from_instance(inst, precision=pw.FP64, stream=stream.cuda_stream) as c64:
        T64 = torch.empty(len(sel), dtype=torch.float64, device="cuda")
        c64.set_profiling(True)
        c64.get_profile(reset=True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        c64.transmission(inst.energies[idx], inst.kpar[idx], T64)
        ev1.record(stream)
        torch.cuda.synchronize()
        prof = c64.get_profile(reset=True)
        kprof = c64.get_kernel_profile(reset=True)
        c64.set_profiling(False)
        T64 = T64.cpu().numpy()
    total_ms = ev0.elapsed_time(ev1)
    modes_ms = prof["modes_ms"] + prof["overlap_ms"]
    sweep_ms = max(total_ms - modes_ms, 1e-9)
    step_ms = modes_ms + n_e * sweep_ms / len(sel)
    out = {"value": n_e / (step_ms / 1e3), "unit": "points/s", "step_ms_estimate": step_ms,
           "sample": f"1 k_par (index {kk}) x {len(sel)} of its {n_e} energies through the whole FP64 path "
                     f"(eigenmodes and overlaps of the k_par, FP64 sweep), CUDA events; a full step is the "
                     f"mode stage plus {n_e} x the sweep time per point",
           "modes_ms": modes_ms, "sweep_ms_per_point": sweep_ms / len(sel),
           "kernels": kernel_table(kprof, 1)[:6]}
    if gold is not None:
        ref = np.array([gold["T"][i] if gold["T"][i] is not None else np.nan for i in sel])
        rel = np.abs(T64 - ref) / np.maximum(np.abs(ref), T_FLOOR)
        ok = ~np.isnan(ref)
        out["vs_oracle"] = {"points": int(ok.sum()),
                            "max_rel_err_T": float(np.max(rel[ok])) if ok.any() else None}
    return out


def workload_config(name, n, N, n_e, n_k, world):
    """The `config` object both arms report for the junction workloads."""
    return {"workload": f"{name}: AB junction, N_G={n}, {N} slices, "
                        f"{n_e} E x {n_k} k_par ({n_e * n_k} points); step = 1 k_par x {n_e} E",
            "global_batch": n_e * world,
            "l2": f"inputs larger than L2 (overlaps of one k_par: {(N + 1) * n * n * 16 / 1e9:.2f} GB)",
            "parallelism": f"replicas over k_par x{world}"}


def run_reference(args):
    """The CPU oracle as the reference arm: each step is the bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    inst, n_e, n_k = workload(args.config)
    cores = os.cpu_count()
    rates, secs = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r, info = cpu_oracle_rate(inst, n_e, sample_ifaces=8, sample_slices=8)
        if i >= args.warmup:
            rates.append(r)
            secs.append(time.perf_counter() - t0)
    v = float(np.mean(rates))
    config = workload_config(args.config, info["n"], info["N"], n_e, n_k, 1)
    config["precision"] = "fp64 (CPU oracle)"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": cores, "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_uneven(args, torch, pw, local):
    """The uneven-batch form: the first K of the 2048 instances per step, one
    call per step; under torchrun each rank takes its share of the K
    instances by weight n^3 (N_s + 1) (no data exchange), and the summed T of
    all ranks is added up on the host at the end."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    allk = uneven_batch(2048)[:args.instances]
    mine = shard_instances([instance_weight(x) for x in allk], rank, world)
    insts = [allk[i] for i in mine]
    prec = pw.MIXED_FP32 if args.precision == "mixed" else pw.FP64
    E = np.array([float(x.energies[0]) for x in insts])
    k = np.array([x.kpar[0] for x in insts])
    stream = torch.cuda.current_stream()
    b = pw.Batch.from_instances(insts, prec, 0 if prec == pw.FP64 else 4, stream=stream.cuda_stream)
    T = torch.empty(len(insts), dtype=torch.float64, device="cuda")
    err = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        b.transmission(E, k, T, err_out=err, allow_threshold=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stage = None
    ev0.record(stream)
    for _ in range(args.steps):
        b.transmission(E, k, T, err_out=err, allow_threshold=True)
        st = b.stats()
        stage = st if stage is None else {kk: stage[kk] + st[kk] if kk != "variant" else st[kk]
                                           for kk in st}
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = reduce_max(ev0.elapsed_time(ev1), world, "cuda")
    sumT = reduce_sum([float(torch.nan_to_num(T).sum().item())], world, "cuda")[0]
    if rank != 0:
        b.close()
        return
    ng = [x.ng_exact for x in allk]
    ns = [x.n_slices for x in allk]
    line = {
        "metric": "uneven-batch instances/s (one (E,k_par) point each)",
        "value": args.steps * len(allk) / (ms / 1e3), "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64" if prec == pw.MIXED_FP32 else "c128", "data": "synthetic",
        "sumT": sumT,
        "config": {"workload": f"uneven: first {len(allk)} of 2048 seeded instances, N_G "
                               f"{min(ng)}..{max(ng)}, {min(ns)}..{max(ns)} slices",
                   "parallelism": f"instances sharded by n^3 (N_s+1) over {world} rank(s)",
                   "precision": args.precision, "l2": "inputs larger than L2",
                   "sum_n3_slices": float(sum(float(a) ** 3 * (b_ + 2) for a, b_ in zip(ng, ns)))},
        "stages_ms": {kk: vv for kk, vv in stage.items() if kk != "variant"},
        "variant_per_ng": stage["variant"],
        "clocks": clk,
        "accuracy": {"err_est_max": float(torch.nan_to_num(err).max().item())},
    }
    print(json.dumps(line))
    b.close()


def kline(n_k, ax):
    """The k_par mesh of Eq. T2_d: n_k points k_x = (2j - n_k + 1) pi / (n_k a_x),
    k_y = 0 (symmetric in +-k, neither 0 nor the zone edge)."""
    kx = (2.0 * np.arange(n_k) - (n_k - 1)) * np.pi / (n_k * ax)
    return np.stack([kx, np.zeros_like(kx)], axis=1)


def scan_tbar(pw, torch, inst, E, n_k, prec, stream, refine=0):
    """Tbar (Eq. T1_d / T2_d) of one junction at energy E over an n_k-point
    k_x mesh through the library: T of every mesh point by pw_transmission,
    then the FP64 device sums of pw_reduce_transmission.  Returns (Tbar,
    channel points, T per point)."""
    k = kline(n_k, inst.a1[0])
    Es = np.full(n_k, E)
    T = torch.empty(n_k, dtype=torch.float64, device="cuda")
    nop = torch.empty((n_k, 2), dtype=torch.int32, device="cuda")
    with pw.Context.from_instance(inst, precision=prec, refine_iters=refine, stream=stream.cuda_stream) as ctx:
        ctx.transmission(Es, k, T, None, nop, allow_threshold=True)
        red = pw.reduce_transmission(T, nop, stream=stream.cuda_stream)
        torch.cuda.synchronize()
    r = red.cpu().numpy()
    return float(r[1]), int(r[2]), T.cpu().numpy()


def scan_plan(quick=False):
    """The second workload (synthetic analogues of the overlap-area and
    interlayer-distance scans, and the k-mesh convergence of Tbar): lists of
    (label, junction keyword arguments, n_k).  Overlap in rectangular cells
    (two primitive cells each), 16 slices per cell, N_G = 128."""
    ng = 48 if quick else 128
    spc = 4 if quick else 16
    nk = 8 if quick else 32
    ovs = (1, 3) if quick else (1, 2, 4, 6, 8)
    gaps = (3.35, 4.5) if quick else (3.0, 3.35, 4.0, 5.0)
    plan = []
    for st in ("AA", "AB"):
        for ov in ovs:
            plan.append((f"overlap/{st}/{ov}", dict(ng=ng, n_slices=spc * (ov + 4), cells=ov + 4, stacking=st,
                                                   n_e=1, n_k=1), nk))
        for g in gaps:
            plan.append((f"gap/{st}/{g}", dict(ng=ng, n_slices=spc * 8, cells=8, stacking=st, gap_angstrom=g,
                                               n_e=1, n_k=1), nk))
    for m in ((4, 8) if quick else (8, 16, 32, 64, 128)):
        plan.append((f"kmesh/AA/{m}", dict(ng=ng, n_slices=spc * 8, cells=8, stacking="AA", n_e=1, n_k=1), m))
    return plan


def run_scan(args, torch, pw, local):
    """The second workload on one GPU: Tbar against overlap area and gap for
    AA and AB stacking, and Tbar against the k mesh, at E_ref; every point
    through pw_transmission (mixed form), Tbar by pw_reduce_transmission."""
    stream = torch.cuda.current_stream()
    prec = pw.MIXED_FP32 if args.precision == "mixed" else pw.FP64
    plan = scan_plan(quick=args.instances < 0)
    E = 0.2
    out, npts = {}, 0
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    for label, kw, nk in plan:
        inst = junction(**kw)
        tbar, nch, _ = scan_tbar(pw, torch, inst, E, nk, prec, stream)
        out[label] = {"Tbar": tbar, "channel_points": nch, "n_k": nk}
        npts += nk
    secs = time.perf_counter() - t0
    clk = clocks.stop()
    line = {"metric": "second workload: Tbar scans (points/s through the whole path)",
            "value": npts / secs, "unit": "points/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * secs, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64" if prec == pw.MIXED_FP32 else "c128", "data": "synthetic",
            "config": {"workload": "Tbar vs overlap (cells) and gap for AA/AB, Tbar vs k mesh; "
                                   f"E = {E} Ry, {len(plan)} junctions, {npts} points",
                       "precision": args.precision},
            "scan": out, "clocks": clk}
    print(json.dumps(line))


def run_modes(args, torch, pw, local):
    """The mode stage alone (rows a2, a3): the N + 2 slice eigendecompositions
    and N + 1 overlaps of one k_par of the N_G = 512 junction in FP64
    (pw_slice_modes, the same kernels in both forms); a step is one k_par."""
    inst, n_e, n_k = workload("junction512")
    if args.slices:
        inst.z_edges = np.linspace(inst.z_edges[0], inst.z_edges[-1], args.slices + 1)
    stream = torch.cuda.current_stream()
    ctx = pw.Context.from_instance(inst, precision=pw.FP64, stream=stream.cuda_stream)
    n, N = ctx.ng, ctx.n_slices
    nq = N + 2

    def kpar(s):
        return inst.kpar[(s % n_k) * n_e]

    for s in range(args.warmup):
        ctx.slice_modes(kpar(s))
    torch.cuda.synchronize()
    ctx.set_profiling(True, stride=1)
    ctx.get_kernel_profile(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for s in range(args.steps):
        ctx.slice_modes(kpar(args.warmup + s))
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    rows = kernel_table(ctx.get_kernel_profile(reset=True), args.steps)
    ctx.set_profiling(False)
    flops = heev_flops_per_matrix(n) * nq + overlap_flops_per_pair(n) * (nq - 1)
    try:
        own = pw.measure_peaks()
    except Exception:       # noqa: BLE001  (reported as missing)
        own = {}
    fp64_peak = max(own.get("fp64_fma") or 0.0, own.get("fp64_mma") or 0.0) or None
    tf = flops / (ms / args.steps / 1e3) / 1e12
    line = {
        "metric": "slice eigendecompositions per second (mode stage: eigenmodes and overlaps, FP64)",
        "value": args.steps * nq / (ms / 1e3), "unit": "matrices/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": f"junction512 mode stage: N_G={n}, {nq} slice Hamiltonians and {nq - 1} "
                               f"overlaps of one k_par; step = 1 k_par",
                   "eig_wave": pw.eig_wave(n)},
        "tflops": tf, "fp64_peak_tflops": fp64_peak,
        "frac_of_fp64_peak": tf / fp64_peak if fp64_peak else None,
        "algorithmic_flops_per_step": flops,
        "kernels": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()} for r in rows],
        "clocks": clk,
    }
    print(json.dumps(line))
    ctx.close()


def run_grad(args, torch, pw, local):
    """The adjoint form (pw_grad, FP64, checkpointed recomputation): the summed
    T of one k_par x P energies of the N_G = 512, 320-slice junction (its
    64 E x 16 k_par gradient workload) and the derivatives of that sum by
    every well depth and by the sheet gap; one step is one call."""
    inst = junction(ng=512, n_slices=320, n_e=64, n_k=16)
    P = max(1, min(args.grad_points, 64))
    stream = torch.cuda.current_stream()
    ctx = pw.Context.from_instance(inst, precision=pw.FP64, stream=stream.cuda_stream)
    nw = len(inst.v0)

    def pts(s):
        # energies from the middle of the window, where both electrodes have open channels
        kk = 5 + s % 8
        idx = np.arange(kk * 64 + 32, kk * 64 + 32 + P) % (64 * 16)
        return inst.energies[idx], inst.kpar[idx]

    for s in range(args.warmup):
        ctx.grad(*pts(s), n_wells=nw, gap=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    res = None
    for s in range(args.steps):
        res = ctx.grad(*pts(args.warmup + s), n_wells=nw, gap=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ws = ctx.workspace_bytes()
    n, N = ctx.ng, ctx.n_slices
    nc = 8   # incident columns of these points, padded to 4 (n_open <= 5)
    full = 16.0 * ((N + 1) * (n * n + n * nc) + 4 * (N + 2) * n * nc)
    line = {
        "metric": "points/s of the adjoint (sum of T and its derivatives by 48 well depths and the gap, FP64)",
        "value": args.steps * P / (ms / 1e3), "unit": "points/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": f"junction512 gradient: AB junction, N_G={n}, {N} slices, 64 E x 16 k_par; "
                               f"step = 1 k_par x {P} E",
                   "checkpoint_interval": "ceil(sqrt(N+1))"},
        "sum_T_last_step": res[0], "dgap_last_step": res[2],
        "memory": {"workspace_bytes": ws, "per_point_bytes": ws / P,
                   "store_every_interface_per_point_bytes": full},
        "clocks": clk,
    }
    print(json.dumps(line))
    ctx.close()


def run_doubling(args, torch, pw, local):
    """The layer doubling of Eq. recurrence2 (FP64, one point after another)
    on points of the chosen workload: a latency path, timed per point."""
    inst, n_e, n_k = workload(args.config)
    if args.slices:
        inst.z_edges = np.linspace(inst.z_edges[0], inst.z_edges[-1], args.slices + 1)
    stream = torch.cuda.current_stream()
    ctx = pw.Context.from_instance(inst, precision=pw.FP64, stream=stream.cuda_stream)
    npts = max(1, args.instances)
    E, k = inst.energies[:npts], inst.kpar[:npts]
    T = torch.empty(npts, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ctx.transmission_doubling(E, k, T, allow_threshold=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    levels = None
    for _ in range(args.steps):
        levels = ctx.transmission_doubling(E, k, T, allow_threshold=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    # the same points by the sweep, for the comparison of T
    Ts = torch.empty(npts, dtype=torch.float64, device="cuda")
    ctx.transmission(E, k, Ts, allow_threshold=True)
    torch.cuda.synchronize()
    d = (T - Ts).abs() / Ts.abs().clamp(min=T_FLOOR)
    line = {
        "metric": "points/s by layer doubling (Eq. recurrence2, FP64)",
        "value": args.steps * npts / (ms / 1e3), "unit": "points/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": f"{args.config}: N_G={ctx.ng}, {ctx.n_slices} slices, {npts} points",
                   "composition": "doubling"},
        "mixed_levels": [int(x) for x in levels],
        "max_rel_diff_T_vs_sweep": float(torch.nan_to_num(d).max().item()),
        "clocks": clk,
    }
    print(json.dumps(line))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--config", default="junction512",
                    choices=["junction512", "junction401", "junction48", "minimal", "uneven", "scan", "grad",
                             "modes"])
    ap.add_argument("--grad-points", type=int, default=8,
                    help="grad config: energies of one k_par per pw_grad call")
    ap.add_argument("--instances", type=int, default=96,
                    help="uneven config: how many of the 2048 instances one step covers")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--refine", type=int, default=0,
                    help="most FP64 refinement passes of the mixed form (0: library default, "
                         "-1: none)")
    ap.add_argument("--sweep-variant", type=int, default=-1,
                    help="sweep launch variant (bit 0: 512-thread SIMT tiles, bit 1: [W|Y], LU and "
                         "back-substitution GEMMs on the tcgen05 tensor cores); -1: library default")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the comparison with the stored oracle values and the FP64 sample")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU sample")
    ap.add_argument("--fp64-points", type=int, default=16,
                    help="energies of the FP64 GPU sample (one k_par)")
    ap.add_argument("--slices", type=int, default=0,
                    help="override the slice count (profiling of small cases only)")
    ap.add_argument("--composition", default="sweep", choices=["sweep", "doubling"],
                    help="doubling: time the layer doubling of Eq. recurrence2 (FP64, --instances points)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    import __graft_entry__ as g
    g.build()
    import paper_1504_01462_gb300 as pw

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.config == "uneven":
        return run_uneven(args, torch, pw, local)
    if args.config == "scan":
        return run_scan(args, torch, pw, local)
    if args.config == "grad":
        return run_grad(args, torch, pw, local)
    if args.config == "modes":
        return run_modes(args, torch, pw, local)
    if args.composition == "doubling":
        return run_doubling(args, torch, pw, local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    inst, n_e, n_k = workload(args.config)
    if args.slices:
        inst.z_edges = np.linspace(inst.z_edges[0], inst.z_edges[-1], args.slices + 1)
    prec = pw.MIXED_FP32 if args.precision == "mixed" else pw.FP64
    stream = torch.cuda.current_stream()
    ctx = pw.Context.from_instance(inst, precision=prec, refine_iters=args.refine,
                                   stream=stream.cuda_stream)
    if args.sweep_variant >= 0:
        ctx.set_sweep_variant(args.sweep_variant)
    n, N = ctx.ng, ctx.n_slices
    npts = len(inst.energies)

    def step_points(s):
        kk = shard_kpoints(rank, world, n_k, 1, first_step=s)[0]
        idx = np.arange(kk * n_e, (kk + 1) * n_e)
        return inst.energies[idx], inst.kpar[idx]

    T = torch.empty(n_e, dtype=torch.float64, device="cuda")
    nop = torch.empty((n_e, 2), dtype=torch.int32, device="cuda")
    err = torch.zeros(n_e, dtype=torch.float64, device="cuda")
    for s in range(args.warmup):
        E, k = step_points(s)
        ctx.transmission(E, k, T, None, nop, err)
    barrier()

    # ---- device-timed region: K steps, CUDA events on the library's stream
    # (every PROFILE_STRIDE-th launch of each kernel kind is also bracketed by
    # events, for the per-kernel table and the roofline of the dominant kernel)
    ctx.set_profiling(True, stride=PROFILE_STRIDE)
    ctx.get_profile(reset=True)
    ctx.get_kernel_profile(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    flops_launch = []
    err_max = 0.0
    for s in range(args.steps):
        E, k = step_points(args.warmup + s)
        ctx.transmission(E, k, T, None, nop, err)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.get_profile(reset=True)
    kprof = ctx.get_kernel_profile(reset=True)
    ctx.set_profiling(False)
    nopen_last = nop.cpu().numpy()
    err_max = float(err.max().item())
    fb_points, fb_spread = ctx.fp64_fallback()
    flops_per_launch = sum(sweep_flops_per_point(n, int(nl)) for nl in nopen_last[:, 0])
    ms_max = reduce_max(ms, world, "cuda")
    total_points = args.steps * n_e * world
    value = total_points / (ms_max / 1e3)

    # ---- end to end through the public API: host inputs, host T, wall clock
    T_host = torch.empty(n_e, dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for s in range(0 if args.no_e2e else args.steps):
        E, k = step_points(args.warmup + s)
        ctx.transmission(E, k, T, None, None)
        T_host.copy_(T, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = max(time.perf_counter() - t0, 1e-9)
    e2e_value = total_points / reduce_max(e2e_s, world, "cuda")

    # ---- accuracy and the FP64 GPU form, outside every timed region (rank 0):
    # the stored oracle T of all 128 energies at the golden k_par (written by
    # tests/golden/make_fullsize_golden.py) against this form's T, and the FP64
    # GPU form timed on a bounded sample of the same step
    accuracy_vs_oracle = None
    fp64_arm = None
    if rank == 0 and not args.no_accuracy and args.config in ("junction512", "junction401") and not args.slices:
        gold = golden_junction512() if args.config == "junction512" else None
        if gold is not None:
            kk = gold["k_index"]
            idx = np.arange(kk * n_e, (kk + 1) * n_e)
            ctx.transmission(inst.energies[idx], inst.kpar[idx], T, None, nop, err)
            torch.cuda.synchronize()
            have = np.array([t is not None for t in gold["T"]])
            ref = np.array([t if t is not None else np.nan for t in gold["T"]])
            got = T.cpu().numpy()
            rel = np.abs(got - ref) / np.maximum(np.abs(ref), T_FLOOR)
            accuracy_vs_oracle = {"points": int(have.sum()), "k_index": int(kk),
                                  "max_rel_err_T": float(np.nanmax(rel[have])) if have.any() else None,
                                  "T_floor": T_FLOOR,
                                  "T_min_nonzero": float(np.min(ref[have & (ref > 0)])) if (have & (ref > 0)).any()
                                  else None}
        if args.config == "junction401":
            path = os.path.join(ROOT, "tests", "golden", "junction401.json")
            if os.path.exists(path):
                with open(path) as f:
                    g4 = json.load(f)
                E4, k4 = np.array(g4["energies"]), np.array(g4["kpar"]).reshape(-1, 2)
                T4 = torch.empty(len(E4), dtype=torch.float64, device="cuda")
                ctx.transmission(E4, k4, T4)
                torch.cuda.synchronize()
                ref = np.array(g4["T"], dtype=np.float64)
                rel = np.abs(T4.cpu().numpy() - ref) / np.maximum(np.abs(ref), T_FLOOR)
                accuracy_vs_oracle = {"points": len(E4), "max_rel_err_T": float(rel.max()), "T_floor": T_FLOOR,
                                      "stored": "tests/golden/junction401.json"}
        if prec == pw.MIXED_FP32 and not args.no_fp64:
            ctx.close()
            torch.cuda.empty_cache()
            fp64_arm = fp64_sample(pw, torch, inst, n_e, stream, gold, args.fp64_points)

    if rank == 0:
        variant = args.sweep_variant if args.sweep_variant >= 0 else (MIXED_DEFAULT_VARIANT if prec == pw.MIXED_FP32
                                                                      else 0)
        tensor = prec == pw.MIXED_FP32 and (variant & 2) != 0
        peaks = measured_peaks()
        hbm = peaks.get("hbm_gbs") or 6800.0
        try:
            own = pw.measure_peaks()
        except Exception:       # noqa: BLE001  (reported as missing)
            own = {}
        fp32_peak = own.get("fp32_fma") or SM_COUNT * FP32_LANES_PER_SM * 2 * 2070.0 * 1e6 / 1e12
        fp64_peak = max(own.get("fp64_fma") or 0.0, own.get("fp64_mma") or 0.0) or 1.25
        # TF32 dense = measured bf16 x the nominal TF32/BF16 ratio (1.1 / 2.25); the hi/lo
        # split executes three TF32 products per algorithmic product
        tf32_split = (peaks.get("bf16_tflops") or 1900.0) * (1.1 / 2.25) / 3.0
        esz = 8 if prec == pw.MIXED_FP32 else 16
        nc = max(4, ((int(nopen_last[:, 0].max()) + 3) // 4) * 4) if len(nopen_last) else 4
        rows = kernel_table(kprof, args.steps)
        model = sweep_kind_totals(n, nc, n_e, N, tensor and (variant & 8) != 0, esz,
                                  paired=tensor and not (variant & 8))
        # the mode stage of one k_par: N + 2 slice Hamiltonians, the FP64
        # solver's main launch taking the full waves (the rest on the side
        # stream), and N + 1 overlaps
        nq = N + 2
        try:
            wave = pw.eig_wave(n)
        except Exception:       # noqa: BLE001  (no split assumed)
            wave = 0
        fp64_modes = prec == pw.FP64 or not (variant & 32)
        n_main = nq - nq % wave if fp64_modes and wave and nq > wave else nq
        heev_launches = sum(c for (name, (_, _, c)) in kprof.items() if name.startswith("k_heev ("))
        kmodes = heev_launches / max(args.steps, 1)
        if kmodes and fp64_modes:
            model["k_heev"] = (heev_flops_per_matrix(n) * n_main * kmodes, None)
            model["k_overlaps"] = (overlap_flops_per_pair(n) * (nq - 1) * kmodes, None)

        def roof(row):
            key = row["kernel"].split(" ")[0]
            flops, nbytes = model.get(key, (None, None))
            tsec = row["ms_per_step"] / 1e3
            obj = {"kernel": row["kernel"], "avg_launch_ms": row["avg_launch_ms"],
                   "launches_per_step": row["launches_per_step"], "ms_per_step": row["ms_per_step"],
                   "share_of_kernel_time": row["share"], "traffic": None}
            if flops is None or tsec <= 0:
                obj.update({"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                            "note": "no algorithmic model for this kernel"})
                return obj
            on_tc = tensor and key in ("kb_wy", "kb_trail", "kb_bsupd", "kb_fsupd_tc")
            fp64_kind = prec == pw.FP64 or (key in FP64_KINDS and not (variant & 32))
            cpeak = tf32_split if on_tc else (fp64_peak if fp64_kind else fp32_peak)
            csrc = ("of measured: bf16 burst x 1.1/2.25 (nominal TF32/BF16) / 3 products" if on_tc else
                    "of measured: FP64 microbenchmark, the faster of DFMA and DMMA (pw_measure_peaks)"
                    if fp64_kind else "of measured: FP32 FMA microbenchmark (pw_measure_peaks)")
            ai = flops / nbytes if nbytes else None
            if ai is not None and ai * hbm / 1e3 < cpeak:
                ach = nbytes / tsec / 1e9
                per_launch = nbytes / (row["launches_per_step"] or 1)
                obj.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                            "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs",
                            "traffic": (KERNEL_TRAFFIC[key] * per_launch if key in KERNEL_TRAFFIC and on_tc
                                        and not (variant & 8) else None),
                            "traffic_source": ("ncu DRAM/algorithmic ratio of the captured launches x the step's "
                                               "average algorithmic bytes per launch" if key in KERNEL_TRAFFIC
                                               else None),
                            "algorithmic_bytes_per_launch": per_launch,
                            "tflops": flops / tsec / 1e12, "intensity_flop_per_byte": ai})
            else:
                ach = flops / tsec / 1e12
                obj.update({"bound": "tensor" if on_tc else "alu", "achieved": ach, "peak": cpeak,
                            "unit": "TFLOP/s", "frac": ach / cpeak, "peak_source": csrc,
                            "algorithmic_flops_per_launch": flops / (row["launches_per_step"] or 1)})
                if key in KERNEL_TRAFFIC_PER_MATRIX and fp64_modes and n == 512:
                    obj.update({"traffic": KERNEL_TRAFFIC_PER_MATRIX[key] * n_main,
                                "traffic_source": "ncu DRAM bytes per matrix of a 64-matrix capture x the "
                                                  "matrices of the timed launch"})
            return obj

        dominant = roof(rows[0]) if rows else None
        runner_up = roof(rows[1]) if len(rows) > 1 else None
        speedup = (value / fp64_arm["value"]) if fp64_arm else None
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64" if prec == pw.MIXED_FP32 else "c128", "data": "synthetic",
            "config": dict(workload_config(args.config, n, N, n_e, n_k, world), precision=args.precision,
                           sweep_variant=variant),
            "roofline": dominant,
            "roofline_next": runner_up,
            "kernels": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()} for r in rows],
            "stages_ms": {"sweep": prof["sweep_ms"], "modes": prof["modes_ms"],
                          "overlaps": prof["overlap_ms"], "refine": prof["refine_ms"],
                          "note": "totals over the timed steps; with one k_par per call the eigensolver's "
                                  "partial wave and the overlaps run on their own streams beside the sweep, "
                                  "so their time is inside the sweep stage"},
            "fp64_gpu": fp64_arm,
            "speedup_vs_fp64": speedup,
            "measured_peaks_tflops": own or None,
            "accuracy": {"refine_passes_per_step": (prof["refine_stages"] / max(args.steps, 1)
                                                    if prec == pw.MIXED_FP32 else 0),
                         "err_est_max_last_step": err_max,
                         "fp64_fallback_last_step": {"points": fb_points, "max_lu_diag_spread": fb_spread},
                         "vs_oracle": accuracy_vs_oracle,
                         "target_rel_T": 1e-8 if prec == pw.MIXED_FP32 else 1e-10},
            "clocks": clk,
            "gpu_launches": int(sum(c for (_, _, c) in kprof.values())),
            "e2e": (None if args.no_e2e else
                    {"value": e2e_value, "unit": "points/s",
                     "h2d_bytes_per_step": n_e * 32,
                     "d2h_bytes_per_step": n_e * (8 + 4) + 2 * n * 8 + (N + 2) * 4}),
            "sweep_step": {"tflops": flops_per_launch * (N + 1) * args.steps / (prof["sweep_ms"] / 1e3) / 1e12,
                           "note": "algorithmic flops of all sweep phases / sweep-stage time"},
        }
        if not args.no_cpu_baseline:
            r, info = cpu_oracle_rate(inst, n_e)
            line["cpu_baseline"] = {"value": r, "unit": "points/s", "cores": os.cpu_count(),
                                    "kind": "oracle", "sample": info["sample"]}
        print(json.dumps(line))
    ctx.close()   # (no-op when already closed)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
