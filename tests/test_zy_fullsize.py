"""Parity at the workloads' full sizes, against oracle values stored by
tests/golden/make_fullsize_golden.py (the oracle needs about a minute per point
here, too long to recompute inside a test run):

* the N_G = 512, 320-slice AB junction, one k_par x 128 energies in one call
  (the launch configuration the benchmark times), mixed form with its default
  refinement: every stored energy against the oracle to 1e-8 relative on T
  (T = 0 points included: there an electrode has no open channel), the
  open-channel counts exactly, and every point for the properties that hold
  at any size (T finite, 0 <= T <= the open channels of either electrode, the
  refinement's error estimate below the target); the FP64 form on eight of
  the energies (the smallest non-zero T, two T = 0 points, the largest T and
  four spread ones) to 1e-10 relative;
* the N_G = 401 (whole shells), 240-slice junction at four seeded points,
  FP64 to 1e-10 and mixed to 1e-8 relative.

Runs after the other GPU tests (file name) because it holds the device for
the longest."""
import json
import os

import numpy as np
import pytest

from tests.parity import TOL_FP64, TOL_MIXED, rel_T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def pw():
    import __graft_entry__ as g
    g.build()
    import paper_1504_01462_gb300 as pw
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pw


def _run(pw, inst, prec, E, k, with_err=False):
    with pw.Context.from_instance(inst, precision=prec) as ctx:
        T = torch.empty(len(E), dtype=torch.float64, device="cuda")
        nop = torch.empty((len(E), 2), dtype=torch.int32, device="cuda")
        err = torch.zeros(len(E), dtype=torch.float64, device="cuda")
        ctx.transmission(E, k, T, None, nop, err)
        torch.cuda.synchronize()
        shape = (ctx.ng, ctx.n_slices)
        return shape, T.cpu().numpy(), nop.cpu().numpy(), err.cpu().numpy()


def test_full_size_step_against_oracle(pw):
    from synthetic import junction
    gold = _golden("junction512_k5.json")
    inst = junction(ng=512, n_slices=320, n_e=128, n_k=32)
    n_e, kk = 128, gold["k_index"]
    idx = np.arange(kk * n_e, (kk + 1) * n_e)
    E, k = inst.energies[idx], inst.kpar[idx]
    assert np.array_equal(E, np.array(gold["energies"]))
    shape, T, nop, err = _run(pw, inst, pw.MIXED_FP32, E, k)
    assert shape == (512, 320)
    assert np.all(np.isfinite(T))
    assert np.all(T >= -1e-9)
    assert np.all(T <= np.minimum(nop[:, 0], nop[:, 1]) + 1e-9)
    assert np.all((err >= 0) & (err < TOL_MIXED)), err.max()

    have = np.array([t is not None for t in gold["T"]])
    assert have.sum() >= 16, "too few stored oracle points"
    ref = np.array([t if t is not None else np.nan for t in gold["T"]])
    nop_ref = np.array([x if x is not None else [-1, -1] for x in gold["nopen"]])
    assert np.array_equal(nop[have], nop_ref[have])
    rel = rel_T(T[have], ref[have])
    assert np.all(rel < TOL_MIXED), (rel.max(), np.nonzero(have)[0][np.argmax(rel)])

    # FP64 form on eight stored energies
    cand = np.nonzero(have)[0]
    pos = cand[ref[cand] > 0]
    zero = cand[ref[cand] == 0]
    sel = set()
    if len(pos):
        sel |= {int(pos[np.argmin(ref[pos])]), int(pos[np.argmax(ref[pos])])}
        sel |= {int(x) for x in pos[np.linspace(0, len(pos) - 1, 4).astype(int)]}
    sel |= {int(x) for x in zero[:2]}
    sel = sorted(sel)
    _, T64, _, _ = _run(pw, inst, pw.FP64, E[sel], k[sel])
    rel64 = rel_T(T64, ref[sel])
    assert np.all(rel64 < TOL_FP64), (rel64, sel)


def test_config2_junction401_against_oracle(pw):
    from synthetic import junction, junction_ecut_for
    gold = _golden("junction401.json")
    assert all(t is not None for t in gold["T"])
    inst = junction(ng=0, ecut=junction_ecut_for(401), n_slices=240, n_e=128, n_k=32)
    E = np.array(gold["energies"])
    k = np.array(gold["kpar"])
    ref = np.array(gold["T"])
    shape, T64, nop, _ = _run(pw, inst, pw.FP64, E, k)
    assert shape == (401, 240)
    assert np.array_equal(nop, np.array(gold["nopen"]))
    assert np.all(rel_T(T64, ref) < TOL_FP64), (T64, ref)
    _, Tm, _, err = _run(pw, inst, pw.MIXED_FP32, E, k)
    assert np.all(rel_T(Tm, ref) < TOL_MIXED), (Tm, ref)
    assert np.all(err < TOL_MIXED)


def test_config5_gradient_full_size_against_central_differences(pw):
    """The adjoint at the gradient workload's size (AB junction, N_G = 512,
    320 slices, FP64, checkpointed recomputation by default), one point with
    open channels: d(sum T)/dV0 of two wells and d/dgap against central
    differences of the FP64 GPU path's T (itself checked against the oracle
    above) with steps 1e-6 Ry and 1e-5 angstrom, to 1e-6."""
    import copy
    from synthetic import junction
    base = junction(ng=512, n_slices=320, n_e=64, n_k=16)
    i_pt = 5 * 64 + 40
    E = base.energies[i_pt:i_pt + 1]
    k = base.kpar[i_pt:i_pt + 1]
    nw = len(base.v0)
    with pw.Context.from_instance(base, precision=pw.FP64) as ctx:
        sumT, g, dgap = ctx.grad(E, k, n_wells=nw, gap=True)
        ws = ctx.workspace_bytes()
    assert sumT > 1e-3
    # about 4 sqrt(321) n^2 + 4 (N+2) n n_c complex doubles (0.41 GB) instead of
    # the 3 x 321 n^2 (4 GB) of storing every interface and slice
    assert ws < 0.5e9, ws

    def T_of(inst):
        _, T, _, _ = _run(pw, inst, pw.FP64, E, k)
        return float(T[0])

    h = 1e-6
    for w in (0, nw - 1):
        ip, im = copy.deepcopy(base), copy.deepcopy(base)
        ip.v0[w] += h
        im.v0[w] -= h
        fd = (T_of(ip) - T_of(im)) / (2 * h)
        assert abs(fd - g[w]) < 1e-6 * max(1.0, abs(fd)), (w, fd, g[w])
    hg = 1e-5   # angstrom
    Tp = T_of(junction(ng=512, n_slices=320, n_e=64, n_k=16, gap_angstrom=3.35 + hg))
    Tm = T_of(junction(ng=512, n_slices=320, n_e=64, n_k=16, gap_angstrom=3.35 - hg))
    from synthetic import ANGSTROM
    fd_gap = (Tp - Tm) / (2 * hg * ANGSTROM)     # per bohr, the unit of the gap motion
    assert abs(fd_gap - dgap) < 1e-6 * max(1.0, abs(fd_gap)), (fd_gap, dgap)
