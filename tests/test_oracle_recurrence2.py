"""Pins of the oracle's layer doubling with Eq. recurrence2 (transfer blocks
I11, I12 with scattering blocks S21, S22, switched to Eq. recurrence once
the norm of I11 grows).  Each test checks it against something other than itself:
the plain product of the transfer matrices of Eq. transfer (the chain of
Eq. smm1), the star product of Eq. recurrence, the dense solve of all matching
conditions and the 40-digit matrix-exponential solve; and the instability the
switch exists for is shown to be real."""
import numpy as np
import pytest

from oracle import pw_oracle as O
from oracle.brute import brute_transmission
from synthetic import junction, minimal_cell
from tests.test_oracle_pins import _tiny_random_instance


def _setup(inst, i=0):
    m = O.Model(inst)
    E = float(inst.energies[i])
    md = m.modes(np.asarray(inst.kpar[i]))
    return m, E, md


def _rel(x, y):
    return np.abs(x - y).max() / max(np.abs(y).max(), 1e-300)


def test_mixed_blocks_are_the_transfer_matrix_product():
    """I11(m,k) and I12(m,k) of Eq. recurrence2 are the upper blocks of the
    product I(m,n) I(n,k) of the full 2n x 2n transfer matrices (Eq. smm1
    chained), over three thin interfaces of a random cell."""
    inst, _, _ = _tiny_random_instance(21, 2.7, (0.12, -0.07), nsl=2)
    m, E, md = _setup(inst)
    full = None
    elems = []
    for p in range(m.N + 1):
        (Ep, Up), (Eq, Uq) = md[p], md[p + 1]
        blocks = O.transfer_matrix(Up.conj().T @ Uq, O.kz(E, Ep), O.kz(E, Eq), m.thickness(p + 1))
        Ifull = np.block([[blocks[0], blocks[1]], [blocks[2], blocks[3]]])
        full = Ifull if full is None else full @ Ifull
        elems.append(m.interface_mixed(md, E, p))
    T = elems[0]
    for e in elems[1:]:
        T = O.star_mixed(T, e)
    n = m.n
    assert _rel(T[0], full[:n, :n]) < 1e-11
    assert _rel(T[1], full[:n, n:]) < 1e-11


@pytest.mark.parametrize("seed", [3, 4])
def test_mixed_step_equals_star_product(seed):
    """One step of Eq. recurrence2, turned into S by Eq. scatter, equals the
    star product (Eq. recurrence) of the two interfaces' scattering matrices,
    for neighbouring and for already-combined blocks."""
    inst, _, _ = _tiny_random_instance(seed, 3.3, (0.2, 0.1), nsl=4)
    m, E, md = _setup(inst)
    T = [m.interface_mixed(md, E, p) for p in range(m.N + 1)]
    S = [m.interface_s(md, E, p) for p in range(m.N + 1)]
    for a, b in ((0, 1), (2, 3)):
        got = O.s_from_mixed(O.star_mixed(T[a], T[b]))
        ref = O.star(S[a], S[b])
        for x, y in zip(got, ref):
            assert _rel(x, y) < 1e-11
    got = O.s_from_mixed(O.star_mixed(O.star_mixed(T[0], T[1]), O.star_mixed(T[2], T[3])))
    ref = O.star(O.star(S[0], S[1]), O.star(S[2], S[3]))
    for x, y in zip(got, ref):
        assert _rel(x, y) < 1e-10


def test_doubling_matches_dense_solve_and_brute_force():
    """The whole stack by doubling (mixed levels, then Eq. recurrence) gives
    the transmitted and reflected amplitudes of the dense solve and the T of
    the independent 40-digit solve; five interfaces leave an odd block."""
    inst, tabs, dz = _tiny_random_instance(5, 3.1, (0.21, -0.13), nsl=4)
    m, E, md = _setup(inst)
    S, level = m.total_s_doubling(md, E)
    assert level >= 1
    a, b = O.transmission_dense(m, md, E)
    assert np.abs(a - S[0]).max() < 1e-11
    assert np.abs(b - S[2]).max() < 1e-11
    _, T = O.transmission_from_s(S, E, md[0][0], md[-1][0])
    Hs = [O.hamiltonian(m.mn, m.G, np.array((0.21, -0.13)), t, m.half) for t in m.tables]
    kg2 = ((m.G + np.array((0.21, -0.13))) ** 2).sum(1)
    Tb, _ = brute_transmission(Hs, dz, kg2, kg2, E, dps=40)
    assert abs(T - Tb) < 1e-12


@pytest.mark.parametrize("which", ["minimal", "junction"])
def test_doubling_matches_left_to_right_sweep(which):
    """T from the doubling equals T from the left-to-right star products on
    the minimal cell (thin slices: several mixed levels) and on a junction
    (41 interfaces: the switch to Eq. recurrence happens part way)."""
    if which == "minimal":
        inst = minimal_cell(energies=(2.3, 4.1), kpar=((0.1, -0.2), (0.0, 0.0)))
    else:
        inst = junction(ng=48, n_slices=40, n_e=2, n_k=1)
    m = O.Model(inst)
    ref = O.transmission(inst)
    levels = int(np.ceil(np.log2(m.N + 1)))
    for i in range(len(inst.energies)):
        _, E, md = _setup(inst, i)
        S, level = m.total_s_doubling(md, E)
        _, T = O.transmission_from_s(S, E, md[0][0], md[-1][0])
        assert abs(T - ref[i]) < 1e-10 * max(1.0, ref[i])
        assert 1 <= level
        if which == "junction":
            assert level < levels   # I11 grew past the criterion before the last level


def test_switch_is_needed():
    """Without the switch the transfer blocks carry the growing exponentials
    of the evanescent modes and T is lost (the instability that Sec. II A
    gives as the reason for the scattering form); a loose criterion already
    costs accuracy; the default keeps 1e-13."""
    inst = junction(ng=48, n_slices=40, n_e=1, n_k=1)
    m, E, md = _setup(inst)
    ref = O.transmission(inst)[0]

    def T_of(cond_max):
        S, level = m.total_s_doubling(md, E, cond_max)
        return O.transmission_from_s(S, E, md[0][0], md[-1][0])[1], level

    T_def, lv_def = T_of(O.COND_SWITCH)
    T_never, lv_never = T_of(np.inf)
    T_loose, lv_loose = T_of(1e10)
    assert abs(T_def - ref) < 1e-13 * max(1.0, ref)
    assert lv_never == int(np.ceil(np.log2(m.N + 1)))
    assert not abs(T_never - ref) < 1e-3 * max(1.0, ref)
    assert lv_loose > lv_def
    assert abs(T_loose - ref) > abs(T_def - ref)


def test_single_interface_and_ill_conditioned_start():
    """One interface: the doubling is Eq. scatter itself.  A criterion below
    every interface's I11 norm turns the elements into scattering matrices
    before any mixed level, and the result is the left-to-right sweep's."""
    inst, _, _ = _tiny_random_instance(8, 2.2, (0.0, 0.3), nsl=3)
    m, E, md = _setup(inst)
    S1, lv1 = O.doubling([m.interface_mixed(md, E, 0)])
    for x, y in zip(S1, m.interface_s(md, E, 0)):
        assert np.abs(x - y).max() < 1e-13
    assert lv1 == 0
    S, lv = m.total_s_doubling(md, E, cond_max=0.5)
    assert lv == 0
    for x, y in zip(S, m.total_s(md, E)):
        assert _rel(x, y) < 1e-11


def test_switching_measure_tracks_the_condition_number():
    """The switching measure is the matrix 1-norm of I11 (largest column sum,
    not the row sum), and on a junction it switches at the same level as the
    2-norm condition number would."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    A[:, 2] *= 50.0
    assert abs(O.i11_growth(A) - np.linalg.norm(A, 1)) < 1e-12 * np.linalg.norm(A, 1)
    assert O.i11_growth(A) != pytest.approx(np.linalg.norm(A, np.inf))
    inst = junction(ng=48, n_slices=40, n_e=1, n_k=1)
    m, E, md = _setup(inst)
    els = [m.interface_mixed(md, E, p) for p in range(m.N + 1)]
    _, lv = O.doubling(els)
    orig = O.i11_growth
    try:
        O.i11_growth = lambda I11: float(np.linalg.cond(I11))
        _, lv2 = O.doubling(els)
    finally:
        O.i11_growth = orig
    assert lv == lv2
