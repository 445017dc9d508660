"""pw_grad (adjoint of the summed transmission with respect to the device
wells' depths and to the sheet gap) against the oracle's adjoint and central
differences."""
import copy

import numpy as np
import pytest

from oracle import pw_oracle as O
from synthetic import junction, minimal_cell
from tests.parity import TOL_FP64, rel_T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pw():
    import __graft_entry__ as g
    g.build()
    import paper_1504_01462_gb300 as pw
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pw


def _oracle_grad(inst, E, k, w):
    m = O.Model(inst)
    dH = O.well_depth_derivatives(m)
    tot, g = 0.0, np.zeros(len(inst.v0))
    for Ei, ki, wi in zip(E, k, w):
        T, gi = O.grad_T(m, np.asarray(ki), float(Ei), dH)
        tot += wi * T
        g += wi * gi
    return tot, g


def test_grad_minimal_cell_against_oracle_adjoint_and_fd(pw):
    E = np.array([2.3, 4.1, 0.7, 2.9])
    k = np.array([[0.1, -0.2], [0.0, 0.3], [0.0, 0.0], [0.1, -0.2]])
    w = np.array([1.0, 0.5, 2.0, 1.5])
    inst = minimal_cell(n_wells=3, n_slices=6, energies=E, kpar=k)
    with pw.Context.from_instance(inst) as ctx:
        sumT, g = ctx.grad(E, k, w, n_wells=len(inst.v0))
    ref_T, ref_g = _oracle_grad(inst, E, k, w)
    assert rel_T(sumT, ref_T) < TOL_FP64
    assert np.abs(g - ref_g).max() < 1e-9 * max(1.0, np.abs(ref_g).max())
    h = 1e-5
    for i in range(len(inst.v0)):
        ip, im = copy.deepcopy(inst), copy.deepcopy(inst)
        ip.v0[i] += h
        im.v0[i] -= h
        fd = (np.dot(w, O.transmission(ip)) - np.dot(w, O.transmission(im))) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd))


def test_grad_small_junction_against_oracle_adjoint(pw):
    inst = junction(ng=48, n_slices=16, n_e=3, n_k=4)
    sel = [1, 5, 6, 9]
    E, k = inst.energies[sel], inst.kpar[sel]
    with pw.Context.from_instance(inst) as ctx:
        sumT, g = ctx.grad(E, k, None, n_wells=len(inst.v0))
    ref_T, ref_g = _oracle_grad(inst, E, k, np.ones(len(sel)))
    assert rel_T(sumT, ref_T) < TOL_FP64
    assert np.abs(g - ref_g).max() < 1e-8 * max(1.0, np.abs(ref_g).max())


def _oracle_gap(inst, E, k):
    m = O.Model(inst)
    dH = O.well_shift_derivative(m, inst.gap_rate_wells)
    lr = tuple(map(tuple, inst.gap_rate_leads))
    tot, g = 0.0, 0.0
    for Ei, ki in zip(E, k):
        T, gi = O.grad_T(m, np.asarray(ki), float(Ei), [dH], [lr])
        tot += T
        g += gi[0]
    return tot, g


def test_gap_derivative_small_junction(pw):
    """d sum T / d gap: wells of each sheet and its electrode move by half the
    gap; against the oracle's adjoint and central differences over the
    generated geometry (step 1e-5 angstrom)."""
    from synthetic.junction import ANGSTROM
    inst = junction(ng=48, n_slices=16, n_e=3, n_k=4)
    sel = [1, 5, 6, 9]
    E, k = inst.energies[sel], inst.kpar[sel]
    with pw.Context.from_instance(inst) as ctx:
        sumT, dV0, dgap = ctx.grad(E, k, None, n_wells=len(inst.v0), gap=True)
    ref_T, ref_g = _oracle_gap(inst, E, k)
    assert rel_T(sumT, ref_T) < TOL_FP64
    assert abs(dgap - ref_g) < 1e-8 * max(1.0, abs(ref_g))
    h = 1e-5
    vals = []
    for gap in (3.35 + h, 3.35 - h):
        J = junction(ng=48, n_slices=16, n_e=3, n_k=4, gap_angstrom=gap)
        vals.append(float(np.sum(O.transmission(J, points=sel))))
    fd = (vals[0] - vals[1]) / (2 * h * ANGSTROM)
    assert abs(fd - dgap) < 1e-6 * max(1.0, abs(fd))


def test_shift_derivative_asymmetric_cell(pw):
    """Arbitrary transverse motion (x and y) of wells and both electrodes of a
    cell without symmetry; and a rigid translation of everything gives 0."""
    from synthetic import Lead
    E = np.array([2.3, 4.1])
    k = np.array([[0.1, -0.2], [0.0, 0.3]])
    inst = minimal_cell(n_wells=4, n_slices=6, energies=E, kpar=k)
    rng = np.random.default_rng(7)
    inst.lead_left = Lead(rng.uniform(0, 5, (2, 2)), np.array([1.5, 2.0]), np.array([0.6, 0.6]), 1.3)
    inst.lead_right = Lead(rng.uniform(0, 5, (3, 2)), np.array([1.0, 2.5, 1.2]),
                           np.array([0.6, 0.5, 0.7]), 0.9)
    inst.gap_rate_wells = rng.uniform(-1, 1, (len(inst.v0), 2))
    inst.gap_rate_leads = np.array([[0.4, -0.7], [-0.2, 0.5]])
    with pw.Context.from_instance(inst) as ctx:
        sumT, _, dgap = ctx.grad(E, k, None, gap=True)
    ref_T, ref_g = _oracle_gap(inst, E, k)
    assert rel_T(sumT, ref_T) < TOL_FP64
    assert abs(ref_g) > 1e-3
    assert abs(dgap - ref_g) < 1e-9 * max(1.0, abs(ref_g))
    inst.gap_rate_wells = np.tile([0.3, 1.0], (len(inst.v0), 1))
    inst.gap_rate_leads = np.array([[0.3, 1.0], [0.3, 1.0]])
    with pw.Context.from_instance(inst) as ctx:
        _, _, rigid = ctx.grad(E, k, None, gap=True)
    assert abs(rigid) < 1e-10


def test_grad_rejects_gap_and_tables(pw):
    """No geometry motion given at setup: the gap derivative is refused."""
    inst = minimal_cell(n_wells=2, n_slices=3)
    import ctypes
    with pw.Context.from_instance(inst) as ctx:
        E = np.array([2.0])
        k = np.zeros((1, 2))
        s = np.zeros(1)
        gap = np.zeros(1)
        dp = ctypes.POINTER(ctypes.c_double)
        st = pw.lib().pw_grad(ctx.handle, 1, E.ctypes.data_as(dp), k.ctypes.data_as(dp), None,
                              s.ctypes.data_as(dp), None, gap.ctypes.data_as(dp))
        assert st == 1


def test_autograd_function_over_pw_grad(pw):
    """torch.autograd through SummedTransmission: gradients of V0 and of the
    gap (per angstrom) equal the adjoint's and central differences of the
    forward value."""
    from paper_1504_01462_gb300.autograd import summed_transmission
    from synthetic.junction import ANGSTROM
    base = junction(ng=48, n_slices=16, n_e=3, n_k=4)
    sel = [1, 5, 6]
    E, k = base.energies[sel], base.kpar[sel]

    def make(v0, gap):
        inst = junction(ng=48, n_slices=16, n_e=3, n_k=4, gap_angstrom=gap)
        inst.v0 = v0.copy()
        inst.gap_rate_wells = inst.gap_rate_wells * ANGSTROM     # per angstrom
        inst.gap_rate_leads = inst.gap_rate_leads * ANGSTROM
        return pw.Context.from_instance(inst)

    v0 = torch.tensor(base.v0, dtype=torch.float64, requires_grad=True)
    gap = torch.tensor(3.35, dtype=torch.float64, requires_grad=True)
    out = summed_transmission(v0, gap, make, E, k)
    out.backward()
    with make(base.v0, 3.35) as ctx:
        sumT, dV0, dgap = ctx.grad(E, k, None, n_wells=len(base.v0), gap=True)
    assert rel_T(out.item(), sumT) < 1e-12
    assert torch.allclose(v0.grad, torch.as_tensor(dV0), rtol=0, atol=1e-12)
    h = 1e-5
    with torch.no_grad():
        fp = summed_transmission(v0, gap + h, make, E, k).item()
        fm = summed_transmission(v0, gap - h, make, E, k).item()
    assert abs((fp - fm) / (2 * h) - gap.grad.item()) < 1e-6 * max(1.0, abs(gap.grad.item()))


@pytest.mark.parametrize("interval", [1, 3, 0])
def test_grad_checkpointed_recomputation_equals_stored_sweep(pw, interval):
    """pw_grad recomputes its sweeps in segments of C interfaces from stored
    states; every C (1, a ragged 3 on 17 interfaces, and the default
    ceil(sqrt(17)) = 5) gives the same sum and gradient as storing every
    interface (C = N + 1), and both match the oracle's adjoint."""
    inst = junction(ng=48, n_slices=16, n_e=3, n_k=4)
    sel = [1, 5, 6, 9]
    E, k = inst.energies[sel], inst.kpar[sel]
    nw = len(inst.v0)
    with pw.Context.from_instance(inst) as ctx:
        ctx.set_grad_checkpoint(inst.n_slices + 1)
        s_full, g_full, dg_full = ctx.grad(E, k, n_wells=nw, gap=True)
        ctx.set_grad_checkpoint(interval)
        s_ck, g_ck, dg_ck = ctx.grad(E, k, n_wells=nw, gap=True)
    assert rel_T(s_ck, s_full) < 1e-13
    assert np.abs(g_ck - g_full).max() < 1e-12 * max(1.0, np.abs(g_full).max())
    assert abs(dg_ck - dg_full) < 1e-12 * max(1.0, abs(dg_full))
    ref_T, ref_g = _oracle_grad(inst, E, k, np.ones(len(E)))
    assert rel_T(s_ck, ref_T) < TOL_FP64
    assert np.abs(g_ck - ref_g).max() < 1e-9 * max(1.0, np.abs(ref_g).max())


def test_grad_memory_grows_as_sqrt_of_slices(pw):
    """Workspace of pw_grad for one point at 80 and 320 slices (N_G = 256):
    with the default segments it grows by about sqrt(4) = 2 (the stores and
    the gradient's slice chunks are ~4 sqrt(N+1) n^2; only the n x n_c
    amplitudes grow linearly), storing every interface grows it by about 4."""
    out = {}
    for ns in (80, 320):
        inst = junction(ng=256, n_slices=ns, n_e=1, n_k=1)
        for mode, interval in (("ckpt", 0), ("full", ns + 1)):
            with pw.Context.from_instance(inst) as ctx:
                ctx.set_grad_checkpoint(interval)
                ctx.grad(inst.energies, inst.kpar, n_wells=len(inst.v0))
                out[(mode, ns)] = ctx.workspace_bytes()
    r_ck = out[("ckpt", 320)] / out[("ckpt", 80)]
    r_full = out[("full", 320)] / out[("full", 80)]
    assert r_ck < 2.6, out
    assert r_full > 3.3, out
    assert out[("ckpt", 320)] < 0.3 * out[("full", 320)], out
