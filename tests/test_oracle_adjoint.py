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
