"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a hand
count, quadrature of the real-space potential, the textbook rectangular
barrier, the free-electron channel count, flux conservation, reciprocity,
a second formulation (one dense linear system), an independent 40-digit
matrix-exponential solve, and the star product's algebraic identities."""
import math

import numpy as np
import pytest
from scipy.special import roots_legendre

from oracle import pw_oracle as O
from oracle.brute import brute_transmission
from synthetic import (explicit_barrier, explicit_tables, junction, junction_ecut_for,
                       minimal_cell, random_tables)


# ---------------------------------------------------------------------------
# a1: basis and Fourier tables
# ---------------------------------------------------------------------------
def test_gset_minimal_cell_hand_count():
    """a = 5 bohr square, |G|^2 <= 5 (2pi/a)^2: shells m^2+n^2 = 0,1,2,4,5 hold
    1 + 4 + 4 + 4 + 8 = 21 vectors."""
    inst = minimal_cell()
    mn, G = O.gvectors(inst.a1, inst.a2, inst.ecut, 0)
    assert len(mn) == 21
    s = (mn ** 2).sum(1)
    assert [int((s == v).sum()) for v in (0, 1, 2, 4, 5)] == [1, 4, 4, 4, 8]
    assert list(s) == sorted(s)                      # ordered by shell
    # full shells are inversion symmetric
    assert set(map(tuple, mn)) == set(map(tuple, -mn))


def test_gset_junction_counts():
    """Junction cell 2.46 A x 20 A: the cutoffs 29.34 and 35.82 Ry hold 401 and
    513 vectors; the exact-size set of 512 drops the last (m, n) of the last
    shell of the 513."""
    for ng in (401, 513):
        inst = junction(ecut=junction_ecut_for(ng))
        mn, _ = O.gvectors(inst.a1, inst.a2, inst.ecut, 0)
        assert len(mn) == ng
        assert set(map(tuple, mn)) == set(map(tuple, -mn))
    inst = junction(ecut=35.82)
    full, _ = O.gvectors(inst.a1, inst.a2, inst.ecut, 0)
    inst = junction(ng=512)
    ex, _ = O.gvectors(inst.a1, inst.a2, 0.0, 512)
    assert np.array_equal(ex, full[:512])


def _oblique_setup():
    a1 = np.array([4.0, 0.0])
    a2 = np.array([1.0, 3.5])
    wells = np.array([[0.7, 1.1, 0.5], [2.9, 2.2, 1.4], [3.6, 0.2, 0.1]])
    v0 = np.array([2.0, 1.3, 0.7])
    sig = np.array([0.5, 0.7, 0.45])
    return a1, a2, wells, v0, sig


def _grid(a1, a2, N):
    u = (np.arange(N) + 0.5) / N
    uu, vv = np.meshgrid(u, u, indexing="ij")
    return uu[..., None] * a1 + vv[..., None] * a2      # (N, N, 2)


def _transverse_sum(r, a1, a2, xy, s, images=3):
    out = np.zeros(r.shape[:2])
    for i in range(-images, images + 1):
        for j in range(-images, images + 1):
            c = xy + i * a1 + j * a2
            out += np.exp(-((r - c) ** 2).sum(-1) / (2 * s * s))
    return out


def test_slice_potential_against_quadrature():
    """V^p(G) in closed form equals (1/A) int_cell d^2r <V>_slice(r) e^{-iG.r}
    computed by quadrature of the real-space wells (periodic images summed,
    slice average by Gauss-Legendre)."""
    a1, a2, wells, v0, sig = _oblique_setup()
    z_lo, z_hi = 0.3, 0.9
    half = (2, 2)
    V = O.slice_vg_wells(a1, a2, half, wells, v0, sig, z_lo, z_hi)
    N = 128
    r = _grid(a1, a2, N)
    xg, wg = roots_legendre(60)
    zq = 0.5 * (z_hi - z_lo) * xg + 0.5 * (z_hi + z_lo)
    wq = 0.5 * (z_hi - z_lo) * wg
    Vr = np.zeros((N, N))
    for (x, y, z), v, s in zip(wells, v0, sig):
        zavg = (wq * np.exp(-(zq - z) ** 2 / (2 * s * s))).sum() / (z_hi - z_lo)
        Vr += -v * zavg * _transverse_sum(r, a1, a2, np.array([x, y]), s)
    b1, b2 = O.reciprocal(a1, a2)
    for m in range(-2, 3):
        for n in range(-2, 3):
            G = m * b1 + n * b2
            num = (Vr * np.exp(-1j * (r @ G))).mean()
            assert abs(num - V[m + 2, n + 2]) < 1e-12, (m, n, num, V[m + 2, n + 2])


def test_lead_potential_against_quadrature():
    """An electrode's table equals the z-average over one period of the
    z-periodic array of wells (all z-images summed), by quadrature."""
    from synthetic.junction import Lead
    a1, a2, wells, v0, sig = _oblique_setup()
    period = 2.3
    lead = Lead(wells[:, :2].copy(), v0, sig, period)
    half = (2, 1)
    V = O.lead_vg(a1, a2, half, lead)
    N = 128
    r = _grid(a1, a2, N)
    xg, wg = roots_legendre(80)
    zq = 0.5 * period * xg + 0.5 * period
    wq = 0.5 * period * wg
    Vr = np.zeros((N, N))
    for (x, y, z), v, s in zip(wells, v0, sig):
        zz = sum(np.exp(-(zq - z - j * period) ** 2 / (2 * s * s)) for j in range(-8, 9))
        zavg = (wq * zz).sum() / period
        Vr += -v * zavg * _transverse_sum(r, a1, a2, np.array([x, y]), s)
    b1, b2 = O.reciprocal(a1, a2)
    for m in range(-2, 3):
        for n in range(-1, 2):
            G = m * b1 + n * b2
            num = (Vr * np.exp(-1j * (r @ G))).mean()
            assert abs(num - V[m + 2, n + 1]) < 1e-12


def test_hamiltonian_is_the_convolution_of_real_space_V():
    """(H c)(G_i) - |k+G_i|^2 c_i equals the plane-wave projection of V(r) psi(r)
    with psi = sum c_G e^{i(k+G).r}: pins the orientation V(G_i - G_j)."""
    a1, a2, wells, v0, sig = _oblique_setup()
    mn, G = O.gvectors(a1, a2, 9.0, 0)
    half = O.table_half(mn)
    z_lo, z_hi = 0.2, 0.6
    tab = O.slice_vg_wells(a1, a2, half, wells, v0, sig, z_lo, z_hi)
    k = np.array([0.31, -0.17])
    H = O.hamiltonian(mn, G, k, tab, half)
    rng = np.random.default_rng(3)
    c = rng.normal(size=len(mn)) + 1j * rng.normal(size=len(mn))
    N = 160
    r = _grid(a1, a2, N)
    xg, wg = roots_legendre(60)
    zq = 0.5 * (z_hi - z_lo) * xg + 0.5 * (z_hi + z_lo)
    wq = 0.5 * (z_hi - z_lo) * wg
    Vr = np.zeros((N, N))
    for (x, y, z), v, s in zip(wells, v0, sig):
        zavg = (wq * np.exp(-(zq - z) ** 2 / (2 * s * s))).sum() / (z_hi - z_lo)
        Vr += -v * zavg * _transverse_sum(r, a1, a2, np.array([x, y]), s)
    psi = (np.exp(1j * (r @ (G + k).T)) * c).sum(-1)
    proj = np.array([(Vr * psi * np.exp(-1j * (r @ (g + k)))).mean() for g in G])
    kin = ((G + k) ** 2).sum(1)
    assert np.abs(H @ c - kin * c - proj).max() < 1e-11
    assert np.abs(H - H.conj().T).max() < 1e-14


# ---------------------------------------------------------------------------
# closed forms and invariants of the whole path
# ---------------------------------------------------------------------------
def _barrier_T(E, V, d, k2):
    eps = E - k2
    if eps > V:
        q = math.sqrt(eps - V)
        return 1.0 / (1.0 + V * V * math.sin(q * d) ** 2 / (4 * eps * (eps - V)))
    kap = math.sqrt(V - eps)
    return 1.0 / (1.0 + V * V * math.sinh(kap * d) ** 2 / (4 * eps * (V - eps)))


@pytest.mark.parametrize("E,V,d,k,nsl", [
    (0.5, 0.3, 1.3, (0.0, 0.0), 3),     # above the barrier
    (0.5, 0.8, 1.3, (0.0, 0.0), 4),     # tunnelling
    (0.5, -0.4, 2.1, (0.0, 0.0), 5),    # well
    (0.9, 0.5, 0.7, (0.3, -0.2), 2),    # oblique incidence: eps = E - |k|^2
    (0.4, 1.5, 3.0, (0.1, 0.1), 7),     # deep tunnelling
])
def test_rectangular_barrier_closed_form(E, V, d, k, nsl):
    """N_G = 1: a constant barrier V of thickness d between V = 0 electrodes has
    T = [1 + V^2 sin^2(qd) / (4 eps (eps - V))]^-1, q = sqrt(eps - V) (sinh form
    under the barrier), eps = E - |k|^2; the barrier may be cut into any
    number of slices."""
    inst = explicit_barrier([V] * nsl, [d / nsl] * nsl, energies=(E,), kpar=(k,))
    T = O.transmission(inst)[0]
    Tc = _barrier_T(E, V, d, k[0] ** 2 + k[1] ** 2)
    assert abs(T - Tc) < 1e-13 * max(1.0, Tc) + 1e-15


def test_free_device_counts_open_channels():
    """V = 0 everywhere: T equals the number of G with |k+G|^2 < E exactly."""
    for E, k in [(0.5, (0.0, 0.0)), (3.0, (0.0, 0.0)), (2.2, (0.21, -0.4)), (6.0, (0.5, 0.5))]:
        inst = minimal_cell(energies=(E,), kpar=(k,))
        inst.v0[:] = 0.0
        T = O.transmission(inst)[0]
        mn, G = O.gvectors(inst.a1, inst.a2, inst.ecut, 0)
        nopen = int((((G + np.array(k)) ** 2).sum(1) < E).sum())
        assert abs(T - nopen) < 1e-12


def test_flux_unitarity_and_conservation():
    """The flux-normalised open-channel S(0,N+1) is unitary (Hermitian slice
    model, flux conserved across every interface): S^H S = I and T + R = n_open."""
    for E, k in [(0.5, (0.0, 0.0)), (2.7, (0.1, 0.3)), (4.4, (-0.2, 0.05))]:
        inst = minimal_cell(energies=(E,), kpar=(k,))
        m = O.Model(inst)
        md = m.modes(np.array(k))
        S = m.total_s(md, E)
        Sf = O.flux_smatrix(S, E, md[0][0], md[-1][0])
        assert np.abs(Sf.conj().T @ Sf - np.eye(len(Sf))).max() < 1e-12
        t, T = O.transmission_from_s(S, E, md[0][0], md[-1][0])
        nL = len(O.open_channels(E, md[0][0]))
        R = float(np.sum(np.abs(Sf[t.shape[0]:, :nL]) ** 2))
        assert abs(T + R - nL) < 1e-12


def test_reciprocity():
    """Real potential, inversion-symmetric basis: T(E, k) = T(E, -k)."""
    for E, k in [(1.7, (0.2, 0.35)), (3.3, (-0.4, 0.1))]:
        a = minimal_cell(energies=(E,), kpar=(k,))
        b = minimal_cell(energies=(E,), kpar=((-k[0], -k[1]),))
        Ta, Tb = O.transmission(a)[0], O.transmission(b)[0]
        assert abs(Ta - Tb) < 1e-12 * max(1.0, Ta)


def _tiny_random_instance(seed, E, k, nsl=4, ecut_shells=1.0):
    rng = np.random.default_rng(seed)
    a = 4.0
    b = 2 * math.pi / a
    half = (2, 2)
    tabs = random_tables(rng, nsl, half, 0.45)
    dz = rng.uniform(0.2, 0.7, nsl)
    z = np.concatenate([[0.0], np.cumsum(dz)])
    inst = explicit_tables([a, 0.0], [0.0, a], ecut_shells * b * b * (1 + 1e-9), z, tabs,
                           None, None, half, [E], [k])
    return inst, tabs, dz


@pytest.mark.parametrize("seed,E,k", [(5, 3.1, (0.21, -0.13)), (6, 1.2, (0.05, 0.4)),
                                      (7, 4.0, (-0.3, 0.0))])
def test_against_expm_brute_force(seed, E, k):
    """An independent 40-digit solve (exact matrix exponential of each slice's
    second-order ODE, plane-wave electrodes, no eigenmodes or S-matrices)
    gives the same T and t (channels matched by their |k+G|^2)."""
    inst, tabs, dz = _tiny_random_instance(seed, E, k)
    m = O.Model(inst)
    T, ts = O.transmission(inst, return_t=True)
    Hs = [O.hamiltonian(m.mn, m.G, np.array(k), t, m.half) for t in m.tables]
    kg2 = ((m.G + np.array(k)) ** 2).sum(1)
    Tb, tb = brute_transmission(Hs, dz, kg2, kg2, E, dps=40)
    assert abs(T[0] - Tb) < 1e-12
    opn = [i for i in range(len(kg2)) if kg2[i] < E]
    order = [i for i in np.argsort(kg2, kind="stable") if kg2[i] < E]
    perm = [opn.index(i) for i in order]
    assert np.abs(ts[0] - tb[np.ix_(perm, perm)]).max() < 1e-12


def test_dense_formulation_matches_star_products():
    """S11 and S21 of the composed S(0,N+1) equal the transmitted and reflected
    amplitudes of one dense solve of all matching conditions."""
    for inst in (minimal_cell(energies=(2.4,), kpar=((0.1, -0.2),)),
                 _tiny_random_instance(9, 2.0, (0.1, 0.1), nsl=6)[0]):
        m = O.Model(inst)
        E = float(inst.energies[0])
        md = m.modes(inst.kpar[0])
        S = m.total_s(md, E)
        a, b = O.transmission_dense(m, md, E)
        assert np.abs(a - S[0]).max() < 1e-11
        assert np.abs(b - S[2]).max() < 1e-11


def test_star_product_is_associative():
    """Composing the interfaces as a balanced tree (layer doubling) equals the
    left-to-right sweep."""
    inst = minimal_cell(energies=(2.9,), kpar=((0.15, 0.05),))
    m = O.Model(inst)
    E = float(inst.energies[0])
    md = m.modes(inst.kpar[0])
    parts = [m.interface_s(md, E, p) for p in range(m.N + 1)]
    while len(parts) > 1:
        nxt = [O.star(parts[i], parts[i + 1]) for i in range(0, len(parts) - 1, 2)]
        if len(parts) % 2:
            nxt.append(parts[-1])
        parts = nxt
    S = m.total_s(md, E)
    for x, y in zip(parts[0], S):
        assert np.abs(x - y).max() < 1e-11


def test_star_identity_and_identical_neighbours():
    """S(p,p) = I is the identity of the star product; two slices with the same
    potential give O = I, so P = I, Q = 0 and S = (E+, 0, 0, E+)."""
    inst = minimal_cell(energies=(2.0,), kpar=((0.1, 0.2),))
    m = O.Model(inst)
    md = m.modes(inst.kpar[0])
    S = m.interface_s(md, 2.0, 3)
    Id = O.identity_s(m.n)
    for x, y in zip(O.star(Id, S), S):
        assert np.abs(x - y).max() < 1e-14
    for x, y in zip(O.star(S, Id), S):
        assert np.abs(x - y).max() < 1e-14
    E, U = md[3]
    k = O.kz(2.0, E)
    ep = np.exp(1j * k * 0.37)
    S2 = O.smatrix_from_transfer(*O.transfer_matrix(U.conj().T @ U, k, k, 0.37))
    assert np.abs(S2[0] - np.diag(ep)).max() < 1e-12
    assert np.abs(S2[1]).max() < 1e-12 and np.abs(S2[2]).max() < 1e-12
    assert np.abs(S2[3] - np.diag(ep)).max() < 1e-12


def test_splitting_a_uniform_slice():
    """A slice of thickness d and the same slice cut in two (d1 + d2 = d)
    give the same S(0, N+1)."""
    rng = np.random.default_rng(11)
    a = 4.0
    b = 2 * math.pi / a
    half = (2, 2)
    tabs = random_tables(rng, 3, half, 0.4)
    z1 = np.array([0.0, 0.4, 1.1, 1.5])
    tabs2 = np.stack([tabs[0], tabs[1], tabs[1], tabs[2]])
    z2 = np.array([0.0, 0.4, 0.63, 1.1, 1.5])
    kw = dict(a1=[a, 0.0], a2=[0.0, a], ecut=b * b * (1 + 1e-9), lead_l_vg=None,
              lead_r_vg=None, vg_half=half, energies=[2.2], kpar=[(0.1, -0.3)])
    i1 = explicit_tables(z_edges=z1, slice_vg=tabs, **kw)
    i2 = explicit_tables(z_edges=z2, slice_vg=tabs2, **kw)
    m1, m2 = O.Model(i1), O.Model(i2)
    S1 = m1.total_s(m1.modes(i1.kpar[0]), 2.2)
    S2 = m2.total_s(m2.modes(i2.kpar[0]), 2.2)
    for x, y in zip(S1, S2):
        assert np.abs(x - y).max() < 1e-11
