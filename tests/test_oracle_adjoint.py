"""Pins of the oracle's adjoint (the derivative of T with respect to the
device wells' depths) against central finite differences of the oracle's own
T, which needs no adjoint at all."""
import copy

import numpy as np
import pytest

from oracle import pw_oracle as O
from synthetic import minimal_cell


@pytest.mark.parametrize("E,k", [(2.3, (0.1, -0.2)), (4.1, (0.0, 0.3)), (0.7, (0.0, 0.0))])
def test_adjoint_matches_central_differences(E, k):
    inst = minimal_cell(n_wells=3, n_slices=6, energies=(E,), kpar=(k,))
    m = O.Model(inst)
    T, g = O.grad_T(m, inst.kpar[0], E, O.well_depth_derivatives(m))
    assert abs(T - O.transmission(inst)[0]) < 1e-11 * max(1.0, T)
    h = 1e-5
    fd = []
    for i in range(len(inst.v0)):
        ip = copy.deepcopy(inst)
        ip.v0[i] += h
        im = copy.deepcopy(inst)
        im.v0[i] -= h
        fd.append((O.transmission(ip)[0] - O.transmission(im)[0]) / (2 * h))
    assert np.abs(np.array(fd) - g).max() < 1e-7 * max(1.0, np.abs(g).max())


def test_dense_amplitudes_reproduce_sweep():
    """The dense solve's transmitted block equals S11 of the star-product sweep,
    and right incidence on the transposed problem has the transposed S-matrix's
    reflection equal to the original's S22 transposed (reciprocity of S)."""
    inst = minimal_cell(n_wells=3, n_slices=5, energies=(2.0,), kpar=((0.2, 0.1),))
    m = O.Model(inst)
    modes = m.modes(inst.kpar[0])
    S = m.total_s(modes, 2.0)
    n = m.n
    I = np.eye(n, dtype=complex)
    a, b = O.dense_amplitudes(m, modes, 2.0, I, np.zeros((n, n), complex))
    assert np.abs(a[-1] - S[0]).max() < 1e-11
    assert np.abs(b[0] - S[2]).max() < 1e-11
    tmodes = [(Ep, U.conj()) for Ep, U in modes]
    a2, b2 = O.dense_amplitudes(m, tmodes, 2.0, np.zeros((n, n), complex), I)
    # the transposed problem's transmission (right to left) is S11 of the original, transposed
    kL = O.kz(2.0, modes[0][0])
    kR = O.kz(2.0, modes[-1][0])
    oL = O.open_channels(2.0, modes[0][0])
    oR = O.open_channels(2.0, modes[-1][0])
    tt = b2[0][np.ix_(oL, oR)] * np.sqrt(kL[oL][:, None].real / kR[oR][None, :].real)
    t = S[0][np.ix_(oR, oL)] * np.sqrt(kR[oR][:, None].real / kL[oL][None, :].real)
    assert np.abs(tt - t.T).max() < 1e-11


def _junction_T(gap, ng=31, ns=12, idx=6):
    from synthetic import junction
    inst = junction(ng=ng, n_slices=ns, n_e=4, n_k=4, gap_angstrom=gap)
    m = O.Model(inst)
    return inst, m, float(inst.energies[idx]), inst.kpar[idx]


def test_gap_derivative_matches_central_differences():
    """d T / d gap of the side-contact junction (both sheets and both
    electrodes move by half the gap) against central differences of T over the
    generated geometry; the electrode term alone is a sizeable part of it."""
    from synthetic.junction import ANGSTROM
    inst, m, E, k = _junction_T(3.35)
    dH = O.well_shift_derivative(m, inst.gap_rate_wells)
    lr = tuple(inst.gap_rate_leads)
    T, g = O.grad_T(m, k, E, [dH, None, dH], [None, lr, lr])
    assert T > 1.0
    assert abs(g[1]) > 0.2 * abs(g[2])          # the electrodes' share is not negligible
    assert abs(g[0] + g[1] - g[2]) < 1e-14 * max(1.0, abs(g[2]))
    h = 1e-4                                     # angstrom
    vals = []
    for gap in (3.35 + h, 3.35 - h):
        _, mg, Eg, kg = _junction_T(gap)
        vals.append(O.grad_T(mg, kg, Eg, [])[0])
    fd = (vals[0] - vals[1]) / (2 * h * ANGSTROM)
    assert abs(fd - g[2]) < 1e-6 * max(abs(fd), 1e-3)


def test_electrode_translation_matches_central_differences():
    """Only the right electrode moved along y (device fixed): the contact-plane
    jump term against central differences with the electrode's wells moved."""
    inst, m, E, k = _junction_T(3.35)
    T, g = O.grad_T(m, k, E, [None], [((0.0, 0.0), (0.0, 1.0))])
    h = 1e-4
    vals = []
    for s in (h, -h):
        ip = copy.deepcopy(inst)
        ip.lead_right.wells_xy[:, 1] += s
        vals.append(O.grad_T(O.Model(ip), k, E, [])[0])
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(g[0]) > 1e-4
    assert abs(fd - g[0]) < 1e-6 * max(abs(fd), 1e-3)


def _asymmetric_cell():
    """Minimal cell with random wells in both electrodes (no symmetry ties the
    parts of a translation together)."""
    from synthetic import Lead
    inst = minimal_cell(n_wells=4, n_slices=6, energies=(2.3,), kpar=((0.1, -0.2),))
    rng = np.random.default_rng(7)
    inst.lead_left = Lead(rng.uniform(0, 5, (2, 2)), np.array([1.5, 2.0]), np.array([0.6, 0.6]), 1.3)
    inst.lead_right = Lead(rng.uniform(0, 5, (3, 2)), np.array([1.0, 2.5, 1.2]),
                           np.array([0.6, 0.5, 0.7]), 0.9)
    return inst


def test_rigid_translation_leaves_T_unchanged():
    """Moving every well and both electrodes together is a translation of the
    whole system: its derivative vanishes, while each part alone does not."""
    inst = _asymmetric_cell()
    m = O.Model(inst)
    E, k = float(inst.energies[0]), inst.kpar[0]
    rates = np.tile([0.3, 1.0], (len(inst.v0), 1))
    dH = O.well_shift_derivative(m, rates)
    r = (0.3, 1.0)
    zero = (0.0, 0.0)
    T, g = O.grad_T(m, k, E, [dH, dH, None, None],
                    [(r, r), None, (r, zero), (zero, r)])
    assert T > 0.5
    assert min(abs(g[1]), abs(g[2]), abs(g[3])) > 1e-3
    assert abs(g[0]) < 1e-11 * abs(g[1])
    assert abs(g[1] + g[2] + g[3] - g[0]) < 1e-13


def test_asymmetric_electrode_shift_matches_central_differences():
    """Left electrode moved along x and y at once, asymmetric cell."""
    inst = _asymmetric_cell()
    m = O.Model(inst)
    E, k = float(inst.energies[0]), inst.kpar[0]
    r = np.array([0.4, -0.7])
    T, g = O.grad_T(m, k, E, [None], [(tuple(r), (0.0, 0.0))])
    h = 1e-5
    vals = []
    for s in (h, -h):
        ip = copy.deepcopy(inst)
        ip.lead_left.wells_xy += s * r[None, :]
        vals.append(O.transmission(ip)[0])
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(g[0]) > 1e-3
    assert abs(fd - g[0]) < 1e-7 * max(abs(fd), 1e-3)
