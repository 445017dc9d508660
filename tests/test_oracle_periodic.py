"""Pins of the oracle's periodic electrodes (App. B complex bands by the
generalised Bloch eigenproblem Eq. cmp, tilted cells, band folding; App. C
transmission between periodic electrodes).  Each test checks it against
something other than itself: the z-invariant electrodes of ``pw_oracle``
(a z-invariant electrode is a periodic one of any period), the closed-form
Bloch factors e^{+-ik d} of a uniform cell, flux conservation, the pairing of
the Bloch factors of a Hermitian problem, the invariance of T when one
electrode period is moved into the device, the reflectionless perfect crystal
(straight and tilted), and the direct supercell problem against the folded
primitive one."""
import math

import numpy as np
import pytest

from oracle import complex_bands as CB
from oracle import pw_oracle as O
from synthetic import junction, minimal_cell, random_tables

A = 4.0
B = 2 * math.pi / A
HALF = (2, 2)
B1 = np.array([B, 0.0])
B2 = np.array([0.0, B])


def _basis():
    return O.gvectors([A, 0.0], [0.0, A], 2.0 * B * B * (1 + 1e-9))


def _flux_ok(t, r, tol=1e-12):
    unit = np.sum(np.abs(t) ** 2, 0) + np.sum(np.abs(r) ** 2, 0)
    return np.abs(unit - 1.0).max() < tol


@pytest.mark.parametrize("which", ["minimal", "junction"])
def test_uniform_cells_reproduce_z_invariant_electrodes(which):
    """An electrode that is uniform along z is periodic with any period and
    any cut into slices: T equals the z-invariant electrodes' T of the star
    product path, and the flux is conserved."""
    if which == "minimal":
        inst = minimal_cell(energies=(2.3, 3.9), kpar=((0.1, -0.2), (0.0, 0.0)))
    else:
        inst = junction(ng=48, n_slices=20, n_e=2, n_k=1)
    m = O.Model(inst)
    ref = O.transmission(inst)
    for i in range(len(inst.energies)):
        E, k = float(inst.energies[i]), np.asarray(inst.kpar[i])
        for left, right in ((([m.vl], [0.7]), ([m.vr], [1.3])),
                            (([m.vl] * 2, [0.35, 0.35]), ([m.vr] * 3, [0.2, 0.5, 0.4]))):
            t, r, T, _ = CB.transmission_periodic(m.mn, m.G, m.half, k, E, m.tables, m.dz, left, right)
            assert abs(T - ref[i]) < 1e-12 * max(1.0, ref[i])
            assert _flux_ok(t, r, 1e-11)


def test_uniform_cell_bloch_factors_closed_form():
    """One uniform slice of thickness d: the Bloch factors are e^{ik_n d}
    (right-going, k_n of the slice modes, evanescent ones decaying) and
    e^{-ik_n d} (left-going)."""
    inst = minimal_cell(energies=(2.3,), kpar=((0.1, -0.2),))
    m = O.Model(inst)
    E, k, d = 2.3, np.array([0.1, -0.2]), 0.83
    _, st = CB.electrode_states(m.mn, m.G, m.half, k, E, ([m.vl], [d]), "last")
    En, _ = O.slice_modes(O.hamiltonian(m.mn, m.G, k, m.vl, m.half))
    kn = O.kz(E, En)
    for got, want in ((st["lamR"], np.exp(1j * kn * d)), (st["lamL"], np.exp(-1j * kn * d))):
        g = np.sort_complex(got)
        w = np.sort_complex(want)
        assert np.abs(g - w).max() < 1e-12
    assert st["propR"].sum() == int(np.sum(En < E))


def _random_setup(seed):
    rng = np.random.default_rng(seed)
    mn, G = _basis()
    cellL = (random_tables(rng, 3, HALF, 0.5), [0.3, 0.5, 0.4])
    cellR = (random_tables(rng, 2, HALF, 0.5), [0.6, 0.35])
    dev = random_tables(rng, 5, HALF, 0.5)
    dd = rng.uniform(0.2, 0.6, 5)
    return mn, G, cellL, cellR, dev, dd


@pytest.mark.parametrize("seed,E,k", [(4, 3.7, (0.13, -0.21)), (5, 2.6, (0.0, 0.3))])
def test_periodic_electrodes_conserve_flux_and_pair_bloch_factors(seed, E, k):
    """Different z-periodic electrodes on both sides of a random device: the
    flux-normalised t and r conserve the incident flux; the Bloch factors of a
    Hermitian cell pair as lambda <-> 1 / conj(lambda), n of the 2n go right."""
    mn, G, cellL, cellR, dev, dd = _random_setup(seed)
    k = np.asarray(k)
    t, r, T, info = CB.transmission_periodic(mn, G, HALF, k, E, dev, dd, cellL, cellR)
    assert t.shape[1] >= 1 and _flux_ok(t, r)
    for side in ("left", "right"):
        st = info[side]
        lam = np.concatenate([st["lamR"], st["lamL"]])
        inv = 1.0 / np.conj(lam)
        d = np.min(np.abs(lam[None, :] - inv[:, None]), axis=1) / np.maximum(1.0, np.abs(inv))
        assert d.max() < 1e-10
        assert len(st["lamR"]) == len(mn)
        assert np.all(np.abs(st["lamR"][~st["propR"]]) < 1.0)


def test_moving_an_electrode_period_into_the_device():
    """The electrodes are semi-infinite: one more of their periods on either
    side of the device changes nothing."""
    mn, G, cellL, cellR, dev, dd = _random_setup(4)
    k, E = np.array([0.13, -0.21]), 3.7
    _, _, T, _ = CB.transmission_periodic(mn, G, HALF, k, E, dev, dd, cellL, cellR)
    dev2 = np.concatenate([cellL[0], dev])
    dd2 = np.concatenate([cellL[1], dd])
    _, _, T2, _ = CB.transmission_periodic(mn, G, HALF, k, E, dev2, dd2, cellL, cellR)
    dev3 = np.concatenate([dev, cellR[0], cellR[0]])
    dd3 = np.concatenate([dd, cellR[1], cellR[1]])
    _, _, T3, _ = CB.transmission_periodic(mn, G, HALF, k, E, dev3, dd3, cellL, cellR)
    assert abs(T2 - T) < 1e-12 * max(1.0, T)
    assert abs(T3 - T) < 1e-12 * max(1.0, T)


def test_perfect_crystal_is_reflectionless():
    """Device = three periods of the electrode on both sides: every
    propagating right-going Bloch state is transmitted (T = their number,
    r = 0)."""
    mn, G, cellL, _, _, _ = _random_setup(6)
    k, E = np.array([0.05, 0.12]), 3.1
    dev = np.concatenate([cellL[0]] * 3)
    dd = np.concatenate([cellL[1]] * 3)
    t, r, T, info = CB.transmission_periodic(mn, G, HALF, k, E, dev, dd, cellL, cellL)
    nprop = int(info["left"]["propR"].sum())
    assert nprop >= 2
    assert abs(T - nprop) < 1e-11
    assert np.abs(r).max() < 1e-11


def _tilted_cells(seed, s):
    rng = np.random.default_rng(seed)
    base = random_tables(rng, 1, HALF, 0.6)[0]
    M, d = 3, [0.4, 0.3, 0.5]

    def cell(kappa):   # cell kappa: slice j is the base moved by (kappa M + j) s
        return [CB.translate_table(base, B1, B2, (kappa * M + j) * np.asarray(s)) for j in range(M)]
    return cell, d, M * np.asarray(s)


def test_tilted_cell_perfect_crystal():
    """A screw-periodic electrode: each slice is the previous one moved by s,
    so the cell repeats along a3 = (3 s, d) with a3_perp off the lattice.
    With the tilt phases e^{-i G . a3_perp} on the next cell (App. B) the
    perfect crystal is reflectionless; treating a3 as straight is not."""
    mn, G = _basis()
    cell, d, a3p = _tilted_cells(9, (0.37, 0.21))
    D = CB.tilt_phases(G, a3p)
    k, E = np.array([0.11, 0.07]), 3.3
    dev = cell(1) + cell(2)
    t, r, T, info = CB.transmission_periodic(mn, G, HALF, k, E, dev, d + d, (cell(0), d), (cell(3), d), D, D)
    nprop = int(info["left"]["propR"].sum())
    assert abs(T - nprop) < 1e-11 and np.abs(r).max() < 1e-11
    _, r0, T0, _ = CB.transmission_periodic(mn, G, HALF, k, E, dev, d + d, (cell(0), d), (cell(3), d))
    assert np.abs(r0).max() > 1e-2


def test_tilt_by_a_lattice_vector_is_no_tilt():
    """a3_perp equal to a transverse lattice vector: D = 1, and a cell whose
    slices step by a third of it is reflectionless as a perfect crystal."""
    mn, G = _basis()
    cell, d, a3p = _tilted_cells(9, (A / 3, 0.0))
    D = CB.tilt_phases(G, a3p)
    assert np.abs(D - 1.0).max() < 1e-12
    k, E = np.array([0.11, 0.07]), 3.3
    _, r, T, info = CB.transmission_periodic(mn, G, HALF, k, E, cell(1) + cell(2), d + d,
                                             (cell(0), d), (cell(3), d))
    assert abs(T - info["left"]["propR"].sum()) < 1e-11


def test_band_folding_matches_the_supercell_problem():
    """An electrode with half the supercell's period along x: its supercell
    plane waves fall into two classes that do not couple, each the primitive
    cell's problem at k_perp + g_c.  The folded classes give the supercell's
    Bloch factors and, through their fields, the same T for a device that has
    only the supercell's period."""
    rng = np.random.default_rng(11)
    mn, G = _basis()
    tab = random_tables(rng, 3, HALF, 0.6)
    tab[:, 1::2, :] = 0.0          # odd dm vanish: the potential repeats after a/2 along x
    cell = (list(tab), [0.3, 0.45, 0.25])
    c = [[2, 0], [0, 1]]           # b1 = 2 B1, b2 = B2
    labels = CB.coset_labels(mn, c)
    assert len(set(labels)) == 2
    k, E = np.array([0.11, 0.07]), 3.3
    for ref in ("last", "first"):
        _, st1 = CB.electrode_states(mn, G, HALF, k, E, cell, ref)
        _, st2 = CB.electrode_states_folded(mn, G, HALF, k, E, cell, ref, c)
        l1 = np.sort_complex(np.concatenate([st1["lamR"], st1["lamL"]]))
        l2 = np.sort_complex(np.concatenate([st2["lamR"], st2["lamL"]]))
        assert np.abs(l1 - l2).max() < 1e-12
        assert st1["propR"].sum() == st2["propR"].sum()
    dev = random_tables(rng, 4, HALF, 0.6)
    dd = [0.3] * 4
    L1 = CB.electrode_states(mn, G, HALF, k, E, cell, "last")
    R1 = CB.electrode_states(mn, G, HALF, k, E, cell, "first")
    L2 = CB.electrode_states_folded(mn, G, HALF, k, E, cell, "last", c)
    R2 = CB.electrode_states_folded(mn, G, HALF, k, E, cell, "first", c)
    _, _, Ta = CB.transmission_from_states(mn, G, HALF, k, E, dev, dd, L1, R1, cell[1][0])
    tb, rb, Tb = CB.transmission_from_states(mn, G, HALF, k, E, dev, dd, L2, R2, cell[1][0])
    assert abs(Ta - Tb) < 1e-12 * max(1.0, Ta)
    assert _flux_ok(tb, rb)


@pytest.mark.parametrize("seed,E,k", [(21, 2.9, (0.17, -0.11)), (22, 1.4, (0.0, 0.25))])
def test_bloch_factors_against_the_period_propagator(seed, E, k):
    """The 2n Bloch factors of Eq. cmp (from the S-matrix chain of one period)
    are the eigenvalues of the exact state propagator [c; c'](z + d) =
    M [c; c'](z) over the period, M the product of the slices' matrix
    exponentials evaluated with 40 digits (no modes, no S-matrices)."""
    import mpmath as mp
    rng = np.random.default_rng(seed)
    mn, G = O.gvectors([A, 0.0], [0.0, A], 1.0 * B * B * (1 + 1e-9))
    assert len(mn) == 5
    tabs = random_tables(rng, 3, HALF, 0.5)
    dz = [0.35, 0.5, 0.3]
    kk = np.asarray(k)
    _, st = CB.electrode_states(mn, G, HALF, kk, E, (tabs, dz), "last")
    lam = np.concatenate([st["lamR"], st["lamL"]])
    mp.mp.dps = 40
    n = len(mn)
    M = mp.eye(2 * n)
    for t, d in zip(tabs, dz):
        H = O.hamiltonian(mn, G, kk, t, HALF)
        gen = mp.zeros(2 * n, 2 * n)
        for i in range(n):
            gen[i, n + i] = 1
            for j in range(n):
                gen[n + i, j] = mp.mpc(complex(H[i, j]))
            gen[n + i, i] -= mp.mpf(E)
        M = mp.expm(gen * mp.mpf(d)) * M
    ev = mp.eig(M, left=False, right=False)
    ref = np.array([complex(x) for x in ev])
    for x in ref:
        j = np.argmin(np.abs(lam - x))
        assert abs(lam[j] - x) < 1e-11 * max(1.0, abs(x)), (x, lam[j])
    assert len(lam) == len(ref) == 2 * n
