"""The pins bite: plausible mistakes planted in the oracle (on the CPU, by
monkeypatching) make at least one pin of test_oracle_pins fail."""
import math

import numpy as np
import pytest

from oracle import pw_oracle as O
import tests.test_oracle_pins as pins


def _expect_failure(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_transposed_overlap_is_caught(monkeypatch):
    monkeypatch.setattr(O, "overlap", lambda Up, Uq: Uq.conj().T @ Up)
    _expect_failure(pins.test_against_expm_brute_force, 5, 3.1, (0.21, -0.13))


def test_wrong_fourier_sign_is_caught(monkeypatch):
    orig = O.slice_vg_wells

    def flipped(a1, a2, half, wells, v0, sigma, z_lo, z_hi):
        return np.conj(orig(a1, a2, half, wells, v0, sigma, z_lo, z_hi))
    monkeypatch.setattr(O, "slice_vg_wells", flipped)
    _expect_failure(pins.test_slice_potential_against_quadrature)


def test_swapped_convolution_index_is_caught(monkeypatch):
    orig = O.hamiltonian

    def swapped(mn, G, kpar, table, half):
        H = orig(mn, G, kpar, table, half)
        d = np.diag(np.diag(H))
        return (H - d).T + d
    monkeypatch.setattr(O, "hamiltonian", swapped)
    _expect_failure(pins.test_hamiltonian_is_the_convolution_of_real_space_V)


def test_inverted_flux_factor_is_caught(monkeypatch):
    orig = O.flux_smatrix

    def inverted(S, E, EL, ER):
        oL = O.open_channels(E, EL)
        oR = O.open_channels(E, ER)
        kL = np.sqrt(E - np.asarray(EL)[oL])
        kR = np.sqrt(E - np.asarray(ER)[oR])
        kout = np.concatenate([kR, kL])
        kin = np.concatenate([kL, kR])
        raw = orig(S, E, EL, ER) / np.sqrt(kout[:, None] / kin[None, :])
        return raw * np.sqrt(kin[None, :] / kout[:, None])
    monkeypatch.setattr(O, "flux_smatrix", inverted)
    _expect_failure(pins.test_flux_unitarity_and_conservation)


def test_phase_of_wrong_slice_is_caught(monkeypatch):
    def left_thickness(self, q):
        p = q - 1
        return self.dz[p - 1] if 1 <= p <= self.N else 0.0
    monkeypatch.setattr(O.Model, "thickness", left_thickness)
    _expect_failure(pins.test_against_expm_brute_force, 5, 3.1, (0.21, -0.13))


def test_growing_evanescent_branch_is_caught(monkeypatch):
    def bad_kz(E, En):
        En = np.asarray(En, dtype=np.float64)
        d = E - En
        return np.where(d > 0, np.sqrt(np.abs(d)) + 0j, -1j * np.sqrt(np.abs(d)))
    monkeypatch.setattr(O, "kz", bad_kz)
    _expect_failure(pins.test_against_expm_brute_force, 5, 3.1, (0.21, -0.13))


def test_dropped_multiple_scattering_is_caught(monkeypatch):
    def star_no_x(Sa, Sb):
        a11, a12, a21, a22 = Sa
        b11, b12, b21, b22 = Sb
        return (b11 @ a11, b12 + b11 @ a12 @ b22, a21 + a22 @ b21 @ a11,
                a22 @ b22 + a22 @ b21 @ a12 @ b22)
    monkeypatch.setattr(O, "star", star_no_x)
    _expect_failure(pins.test_against_expm_brute_force, 5, 3.1, (0.21, -0.13))


def test_wrong_transfer_sign_is_caught(monkeypatch):
    orig = O.transfer_matrix

    def bad(Oo, kp, kq, dzq):
        I11, I12, I21, I22 = orig(Oo, kp, kq, dzq)
        return I11, I21, I12, I22
    monkeypatch.setattr(O, "transfer_matrix", bad)
    _expect_failure(pins.test_rectangular_barrier_closed_form, 0.5, 0.3, 1.3, (0.0, 0.0), 3)


# ---------------------------------------------------------------------------
# Eq. recurrence2 (layer doubling with transfer and scattering blocks)
# ---------------------------------------------------------------------------
def _star_mixed_variant(kind):
    def f(Ta, Tb):
        a11, a12, a21, a22 = Ta
        b11, b12, b21, b22 = Tb
        X = (a11 + b21 @ a12) if kind == "transposed_x" else (a11 + a12 @ b21)
        Xinv = np.linalg.inv(X)
        I11 = X @ b11
        I12 = X @ b12 if kind == "dropped_term" else X @ b12 + a12 @ b22
        S21 = (a21 + Xinv @ a22 @ b21) if kind == "inverse_side" else (a21 + a22 @ b21 @ Xinv)
        sign = 1.0 if kind == "sign" else -1.0
        S22 = a22 @ b22 + sign * a22 @ b21 @ Xinv @ a12 @ b22
        return I11, I12, S21, S22
    return f


@pytest.mark.parametrize("kind", ["transposed_x", "dropped_term", "inverse_side", "sign"])
def test_mixed_recurrence_mistakes_are_caught(monkeypatch, kind):
    import tests.test_oracle_recurrence2 as r2
    monkeypatch.setattr(O, "star_mixed", _star_mixed_variant(kind))
    with pytest.raises(AssertionError):
        r2.test_mixed_blocks_are_the_transfer_matrix_product()
        r2.test_mixed_step_equals_star_product(3)


def test_missing_switch_is_caught(monkeypatch):
    import tests.test_oracle_recurrence2 as r2
    orig = O.doubling
    monkeypatch.setattr(O, "doubling", lambda elements, cond_max=O.COND_SWITCH: orig(elements, np.inf))
    _expect_failure(r2.test_doubling_matches_left_to_right_sweep, "junction")


# ---------------------------------------------------------------------------
# periodic electrodes (App. B complex bands, App. C)
# ---------------------------------------------------------------------------
def test_conjugated_tilt_phases_are_caught(monkeypatch):
    from oracle import complex_bands as CB
    import tests.test_oracle_periodic as per
    orig = CB.tilt_phases
    monkeypatch.setattr(CB, "tilt_phases", lambda G, a3: np.conj(orig(G, a3)))
    _expect_failure(per.test_tilted_cell_perfect_crystal)


def test_bloch_problem_sign_mistake_is_caught(monkeypatch):
    from oracle import complex_bands as CB
    import scipy.linalg
    import tests.test_oracle_periodic as per

    def bad(S):
        S11, S12, S21, S22 = S
        n = S11.shape[0]
        Id, Z = np.eye(n, dtype=np.complex128), np.zeros((n, n), dtype=np.complex128)
        return scipy.linalg.eig(np.block([[S11, Z], [S21, Id]]), np.block([[Id, -S12], [Z, -S22]]))
    monkeypatch.setattr(CB, "complex_bands", bad)
    # invisible for uniform cells (S12 = S21 = 0 there); random cells catch it
    with pytest.raises((AssertionError, ValueError, np.linalg.LinAlgError)):
        per.test_periodic_electrodes_conserve_flux_and_pair_bloch_factors(4, 3.7, (0.13, -0.21))


def test_missing_flux_normalisation_is_caught(monkeypatch):
    from oracle import complex_bands as CB
    import tests.test_oracle_periodic as per
    orig = CB.bloch_states

    def unnormalised(lam, X, ref_mode, E, tol=1e-7):
        st = orig(lam, X, ref_mode, E, tol)
        for side in ("R", "L"):
            p = st["prop" + side]
            nrm = np.sqrt(np.sum(np.abs(st["a" + side][:, p]) ** 2 + np.abs(st["b" + side][:, p]) ** 2, axis=0))
            st["a" + side][:, p] /= nrm
            st["b" + side][:, p] /= nrm
        return st
    monkeypatch.setattr(CB, "bloch_states", unnormalised)
    _expect_failure(per.test_periodic_electrodes_conserve_flux_and_pair_bloch_factors, 4, 3.7, (0.13, -0.21))


def test_wrong_next_cell_in_the_right_electrode_is_caught(monkeypatch):
    from oracle import complex_bands as CB
    import tests.test_oracle_periodic as per
    orig = CB.cell_smatrix
    # every slice after the reference moved, as if the whole chain were the next cell
    monkeypatch.setattr(CB, "cell_smatrix",
                        lambda modes, dz, E, D=None, ref="last": orig(modes, dz, E, D, "last") if D is None
                        else CB.chain_s(list(modes) + [(modes[0][0], D[:, None] * modes[0][1])],
                                        [0.0] + list(dz[1:]) + [dz[0]], E) if ref == "last"
                        else CB.chain_s([modes[0]] + [(m[0], D[:, None] * m[1]) for m in modes[1:]]
                                        + [(modes[0][0], D[:, None] * modes[0][1])],
                                        [0.0] + list(dz[1:]) + [dz[0]], E))
    _expect_failure(per.test_tilted_cell_perfect_crystal)


# ---------------------------------------------------------------------------
# separable projector terms (Eqs. nloc, gsol_p0, calm_0)
# ---------------------------------------------------------------------------
def test_missing_cell_area_in_calm_is_caught(monkeypatch):
    from oracle import separable as NL
    import tests.test_oracle_separable as sep
    orig = NL.transmission_nonlocal
    monkeypatch.setattr(NL, "transmission_nonlocal",
                        lambda modes, dz, E, projs, D, area, q=16: orig(modes, dz, E, projs, D, 1.0, q))
    _expect_failure(sep.test_one_dimensional_separable_potential_closed_form, 0.9, (1, 4))


def test_incoming_green_function_is_caught(monkeypatch):
    from oracle import separable as NL
    import tests.test_oracle_separable as sep
    orig = NL._slice_terms

    def incoming(U, k, za, zb, projs, q):   # e^{-ik|u|}: the other branch, no longer outgoing
        return orig(U, -k, za, zb, projs, q)
    monkeypatch.setattr(NL, "_slice_terms", incoming)
    _expect_failure(sep.test_one_dimensional_separable_potential_closed_form, 0.9, (1, 4))


def test_particular_derivatives_dropped_are_caught(monkeypatch):
    from oracle import separable as NL
    import tests.test_oracle_separable as sep
    orig = NL._slice_terms

    def no_deriv(U, k, za, zb, projs, q):
        fa, dfa, fb, dfb, Ha, Hb, P = orig(U, k, za, zb, projs, q)
        return fa, 0 * dfa, fb, 0 * dfb, Ha, Hb, P
    monkeypatch.setattr(NL, "_slice_terms", no_deriv)
    _expect_failure(sep.test_hermitian_projector_terms_conserve_flux, np.diag([0.8, -1.3]))


def test_continuum_pin_catches_a_misweighted_slice_average(monkeypatch):
    """The slice average with sqrt(pi) in place of sqrt(pi/2) (each well's
    z-weight off by sqrt 2) is caught by the continuum pin.  (Shifting every
    well in z, or conjugating the tables - the transverse mirror image, with
    T(-k) = T(k) for a real potential - leaves T unchanged: no T-based pin
    sees those; the quadrature pin of the tables does.)"""
    import tests.test_oracle_continuum as cont
    orig = O.slice_vg_wells

    def misweighted(a1, a2, half, wells, v0, sigma, z_lo, z_hi):
        return math.sqrt(2.0) * orig(a1, a2, half, wells, v0, sigma, z_lo, z_hi)
    monkeypatch.setattr(O, "slice_vg_wells", misweighted)
    _expect_failure(cont.test_slice_model_converges_to_the_continuum, 3.4, (0.3, 0.2))
