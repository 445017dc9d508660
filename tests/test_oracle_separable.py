"""Pins of the oracle's separable (nonlocal) projector terms: particular
solutions of Eq. nloc, the general solution Eq. gsol_p0 and the coefficients
C of Eq. calm_0 solved with the interface matching.  Checked against the
local path when D = 0, the closed-form scattering of a one-dimensional
separable potential (a projector on a single plane wave with a box profile
in z over free slices), flux conservation for Hermitian D, the invariance of
T under cutting a z-uniform region into more slices, and real-space
quadrature of the Gaussian projectors' plane-wave coefficients."""
import math

import numpy as np
import pytest

from oracle import pw_oracle as O
from oracle import separable as NL
from synthetic import explicit_tables, minimal_cell, random_tables

A4 = 4.0
B4 = 2 * math.pi / A4


def _free_instance(dz, E, k):
    z = np.concatenate([[0.0], np.cumsum(dz)])
    tabs = np.zeros((len(dz), 5, 5), complex)
    return explicit_tables([A4, 0.0], [0.0, A4], 2.0 * B4 * B4 * (1 + 1e-9), z, tabs, None, None, (2, 2),
                           [E], [k])


def test_no_projector_strength_is_the_local_path():
    inst = minimal_cell(energies=(2.3, 3.9), kpar=((0.1, -0.2), (0.0, 0.0)))
    m = O.Model(inst)
    area = O.cell_area(inst.a1, inst.a2)
    ref = O.transmission(inst)
    zN = float(np.sum(m.dz))
    for i in range(2):
        E, k = float(inst.energies[i]), np.asarray(inst.kpar[i])
        projs = [NL.gaussian_projector(m.G, k, area, (1.2, 2.1, 1.7), 0.5, 0.0, zN)]
        _, _, T, _, C = NL.transmission_nonlocal(m.modes(k), m.dz, E, projs, [[0.0]], area)
        assert abs(T - ref[i]) < 1e-12 * max(1.0, ref[i])
        assert np.abs(C).max() == 0.0


@pytest.mark.parametrize("D,box", [(0.9, (1, 4)), (-2.5, (1, 4)), (1.7, (0, 6)), (-0.6, (2, 3))])
def test_one_dimensional_separable_potential_closed_form(D, box):
    """Free slices and one projector on the plane wave G0 with a box profile
    chi over whole slices: channel G0 obeys psi'' + k0^2 psi = C chi with
    C = D A int chi psi, so (Green's function e^{ik|u|}/2ik)
      C = D A I+ / (1 - D A J),  t0 = 1 + C I- / (2 i k0),
      I+- = int chi e^{+-ik0 z},  J = int int chi g chi = (1/ik)(-L/(ik) + (e^{ikL} - 1)/(ik)^2),
    and every other open channel passes: T = n_open - 1 + |t0|^2."""
    dz = np.array([0.3, 0.25, 0.4, 0.35, 0.3, 0.2])
    E, k = 3.1, np.array([0.13, -0.07])
    inst = _free_instance(dz, E, k)
    m = O.Model(inst)
    area = O.cell_area(inst.a1, inst.a2)
    g0 = 3
    k0 = math.sqrt(E - float(np.sum((k + m.G[g0]) ** 2)))
    z = np.concatenate([[0.0], np.cumsum(dz)])
    z1, z2 = z[box[0]], z[box[1]]

    def W(zz):
        zz = np.asarray(zz, float)
        out = np.zeros((m.n, len(zz)), complex)
        out[g0] = ((zz >= z1) & (zz <= z2)).astype(float)
        return out
    _, _, T, _, _ = NL.transmission_nonlocal(m.modes(k), m.dz, E, [W], [[D]], area)
    L, ik = z2 - z1, 1j * k0
    Ip = (np.exp(ik * z2) - np.exp(ik * z1)) / ik
    Im = (np.exp(-ik * z1) - np.exp(-ik * z2)) / ik
    J = (1 / ik) * (-L / ik + (np.exp(ik * L) - 1) / ik ** 2)
    C = D * area * Ip / (1 - D * area * J)
    t0 = 1 + C * Im / (2 * ik)
    n_open = int(np.sum(np.sum((k + m.G) ** 2, 1) < E))
    assert abs(T - (n_open - 1 + abs(t0) ** 2)) < 1e-12


def _gaussian_setup(seed):
    rng = np.random.default_rng(seed)
    nsl = 5
    dz = rng.uniform(0.3, 0.6, nsl)
    z = np.concatenate([[0.0], np.cumsum(dz)])
    tabs = random_tables(rng, nsl, (2, 2), 0.4)
    E, k = 3.3, np.array([0.07, 0.19])
    inst = explicit_tables([A4, 0.0], [0.0, A4], 2.0 * B4 * B4 * (1 + 1e-9), z, tabs, None, None, (2, 2),
                           [E], [k])
    m = O.Model(inst)
    area = O.cell_area(inst.a1, inst.a2)
    zN = z[-1]
    projs = [NL.gaussian_projector(m.G, k, area, (1.1, 2.3, 0.45 * zN), 0.45, 0.0, zN),
             NL.gaussian_projector(m.G, k, area, (3.0, 0.6, 0.6 * zN), 0.5, 0.0, zN)]
    return m, E, k, area, projs


@pytest.mark.parametrize("D", [np.diag([0.8, -1.3]), np.array([[0.8, 0.3 + 0.2j], [0.3 - 0.2j, -1.3]])])
def test_hermitian_projector_terms_conserve_flux(D):
    m, E, k, area, projs = _gaussian_setup(3)
    t, r, T, _, _ = NL.transmission_nonlocal(m.modes(k), m.dz, E, projs, D, area)
    unit = np.sum(np.abs(t) ** 2, 0) + np.sum(np.abs(r) ** 2, 0)
    assert np.abs(unit - 1.0).max() < 1e-12
    # the z quadrature has converged
    _, _, T8, _, _ = NL.transmission_nonlocal(m.modes(k), m.dz, E, projs, D, area, q=8)
    _, _, T24, _, _ = NL.transmission_nonlocal(m.modes(k), m.dz, E, projs, D, area, q=24)
    assert abs(T8 - T) < 1e-11 and abs(T24 - T) < 1e-11


def test_cutting_a_uniform_region_into_more_slices():
    """A z-uniform device cut into one, two or three slices, with projectors
    that straddle the cuts: T does not change."""
    rng = np.random.default_rng(5)
    tab = random_tables(rng, 1, (2, 2), 0.4)[0]
    E, k = 3.3, np.array([0.07, 0.19])
    Ts = []
    for cuts in ([1.5], [0.6, 0.9], [0.4, 0.5, 0.6]):
        z = np.concatenate([[0.0], np.cumsum(cuts)])
        inst = explicit_tables([A4, 0.0], [0.0, A4], 2.0 * B4 * B4 * (1 + 1e-9), z, [tab] * len(cuts),
                               None, None, (2, 2), [E], [k])
        m = O.Model(inst)
        area = O.cell_area(inst.a1, inst.a2)
        projs = [NL.gaussian_projector(m.G, k, area, (1.1, 2.3, 0.75), 0.3, 0.0, 1.5)]
        _, _, T, _, _ = NL.transmission_nonlocal(m.modes(k), m.dz, E, projs, [[1.4]], area, q=24)
        Ts.append(T)
    assert max(Ts) - min(Ts) < 1e-11


def test_gaussian_projector_coefficients_against_quadrature():
    """(1/A) int_cell e^{-i(k+G).r} sum_R e^{ik.R} W(r - tau - R) d^2 r of the
    Gaussian, by a midpoint rule over the cell with the images summed."""
    inst = minimal_cell()
    m = O.Model(inst)
    area = O.cell_area(inst.a1, inst.a2)
    k = np.array([0.1, -0.2])
    tau, s = (1.2, 2.1, 1.7), 0.6
    W = NL.gaussian_projector(m.G, k, area, tau, s, 0.0, 4.0)
    zq = np.array([1.3])
    got = W(zq)[:, 0]
    a = inst.a1[0]
    g = (np.arange(96) + 0.5) * a / 96
    X, Y = np.meshgrid(g, g, indexing="ij")
    tot = np.zeros_like(X, dtype=np.complex128)
    for i in range(-3, 4):
        for j in range(-3, 4):
            R = np.array([i * a, j * a])
            tot += np.exp(1j * (k @ R)) * np.exp(-((X - tau[0] - R[0]) ** 2 + (Y - tau[1] - R[1]) ** 2
                                                   + (zq[0] - tau[2]) ** 2) / (2 * s * s))
    for gi in range(0, m.n, 4):
        q = m.G[gi] + k
        want = (np.exp(-1j * (q[0] * X + q[1] * Y)) * tot).sum() * (a / 96) ** 2 / area
        assert abs(got[gi] - want) < 1e-9
