"""The pins bite: plausible mistakes planted in the oracle (on the CPU, by
monkeypatching) make at least one pin of test_oracle_pins fail."""
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
