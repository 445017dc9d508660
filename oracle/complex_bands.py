"""Periodic electrodes for the CPU oracle: the complex band structure of a
z-periodic electrode (App. B, the generalised Bloch eigenproblem Eq. cmp) and
the transmission between two such electrodes (App. C), without nonlocal terms.

TEST INFRASTRUCTURE ONLY, like ``pw_oracle``: nothing in the product path may
import it; it shares no code with the CUDA path.

Amplitude convention (that of the star products in ``pw_oracle``): in a slice
q with modes U_q and wavenumbers k_q the field near the slice's right edge z_q
is psi(G, z) = U_q (e^{ik(z - z_q)} a_q + e^{-ik(z - z_q)} b_q), so both
amplitudes are referenced at the right edge.  S(p, m) of a chain of slices
maps (a_p, b_m) to (a_m, b_p).

Electrode cell: slices c_1 .. c_M over one period d along z (the cell's
third lattice vector a3 = (a3_perp, d)).  Its reference slice is c_M, whose
right edge is the cell boundary (for the right electrode, c_1, whose left edge
meets the device).  The chain c_M -> c_1' -> ... -> c_M' of the next cell
gives S(c_M, c_M'), and the generalised Bloch conditions (Eqs. bc1,
bc2: psi(r_perp + a3_perp, z + d) = lambda psi(r_perp, z), lambda =
e^{i k_perp . a3_perp + i k d}) make the amplitudes of c_M' lambda times those
of c_M.  With S = S(c_M, c_M') that is Eq. cmp with X = [a; b]:
    [[S11, 0], [S21, -1]] X = lambda [[1, -S12], [0, -S22]] X.
A tilted cell (a3_perp != 0): the next cell is the present one moved by a3;
its slice potentials are translated transversally, so its slice modes are
D U with D = diag(e^{-i G . a3_perp}) (the translation of a plane-wave
expansion), while the Bloch factor carries e^{i k_perp . a3_perp}.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from oracle.pw_oracle import (hamiltonian, identity_s, kz, overlap, slice_modes, smatrix_from_transfer,
                              star, transfer_matrix)


def chain_s(modes, thick, E):
    """S(0, m) of the chain of slices modes[0..m] (pairs (E_q, U_q)) by
    Eqs. transfer, scatter and recurrence; interface q joins slices q and q+1
    with the phase of slice q+1 over thick[q+1]."""
    n = len(modes[0][0])
    S = identity_s(n)
    for q in range(len(modes) - 1):
        (Ep, Up), (Eq, Uq) = modes[q], modes[q + 1]
        S = star(S, smatrix_from_transfer(*transfer_matrix(overlap(Up, Uq), kz(E, Ep), kz(E, Eq),
                                                           thick[q + 1])))
    return S


def cell_smatrix(cell_modes, cell_dz, E, D=None, ref="last"):
    """S over one period of an electrode cell (modes of c_1 .. c_M and their
    thicknesses) from its reference slice to the same slice of the next cell:
    ref = "last": c_M -> c_1' -> ... -> c_M'; ref = "first": c_1 -> c_2 ->
    ... -> c_M -> c_1'.  D (vector) is the tilt's diag(e^{-i G . a3_perp})
    applied to the modes of the slices of the next cell (None: a3 along z)."""
    def moved(m):
        return m if D is None else (m[0], D[:, None] * m[1])
    if ref == "last":
        chain = [cell_modes[-1]] + [moved(m) for m in cell_modes]
        thick = [0.0] + list(cell_dz)
    else:
        chain = list(cell_modes) + [moved(cell_modes[0])]
        thick = [0.0] + list(cell_dz[1:]) + [cell_dz[0]]
    return chain_s(chain, thick, E)


def complex_bands(S):
    """Eq. cmp without nonlocal terms: the 2n generalised eigenvalues lambda
    and eigenvectors X = [a; b] (amplitudes of the reference slice) of
    [[S11, 0], [S21, -1]] X = lambda [[1, -S12], [0, -S22]] X."""
    S11, S12, S21, S22 = S
    n = S11.shape[0]
    Id = np.eye(n, dtype=np.complex128)
    Z = np.zeros((n, n), dtype=np.complex128)
    P = np.block([[S11, Z], [S21, -Id]])
    Q = np.block([[Id, -S12], [Z, -S22]])
    lam, X = scipy.linalg.eig(P, Q)
    return lam, X


def edge_fields(ref_mode, E, a, b):
    """psi and d psi / dz at the reference slice's right edge for amplitude
    columns a, b (the i of the derivative included)."""
    En, U = ref_mode
    k = kz(E, En)
    return U @ (a + b), 1j * (U * k[None, :]) @ (a - b)


def flux_matrix(ref_mode, E, a, b):
    """F_ij = (psi_i^H psi'_j - psi'_i^H psi_j) / 2i, the z-flux form of the
    states (columns) at one plane (per unit cell area, in units where a
    plane wave e^{ikz} carries flux k)."""
    psi, dpsi = edge_fields(ref_mode, E, a, b)
    return (psi.conj().T @ dpsi - dpsi.conj().T @ psi) / 2j


def bloch_states(lam, X, ref_mode, E, tol=1e-7):
    """The electrode's generalised Bloch states split by direction:
    right-going = decaying to +z (|lambda| < 1) or propagating (|lambda| = 1)
    with positive flux; left-going the rest.  Propagating states with equal
    lambda are made flux-orthogonal (eigenvectors of their flux form) and
    scaled to unit flux.  Returns a dict of amplitude matrices aR, bR, aL, bL
    (n x n each), the boolean masks propR, propL and the lambdas."""
    n = X.shape[0] // 2
    a, b = X[:n], X[n:]
    mag = np.abs(lam)
    prop = np.isfinite(lam) & (np.abs(mag - 1.0) < tol)
    cols_a, cols_b, right, is_prop, lams = [], [], [], [], []
    done = np.zeros(len(lam), dtype=bool)
    for i in range(len(lam)):
        if done[i]:
            continue
        if not prop[i]:
            done[i] = True
            s = np.linalg.norm(X[:, i])
            cols_a.append(a[:, i] / s)
            cols_b.append(b[:, i] / s)
            right.append(bool(np.isfinite(lam[i]) and mag[i] < 1.0))
            is_prop.append(False)
            lams.append(lam[i])
            continue
        grp = [j for j in range(len(lam)) if prop[j] and not done[j] and abs(lam[j] - lam[i]) < 1e-6]
        for j in grp:
            done[j] = True
        ag, bg = a[:, grp], b[:, grp]
        # orthonormal basis of the group's span, then the flux form on it
        Qb, _ = np.linalg.qr(np.vstack([ag, bg]))
        ag, bg = Qb[:n], Qb[n:]
        F = flux_matrix(ref_mode, E, ag, bg)
        w, V = np.linalg.eigh(0.5 * (F + F.conj().T))
        for c in range(len(grp)):
            if abs(w[c]) < 1e-12:
                raise ValueError("a propagating Bloch state without flux (band edge)")
            s = 1.0 / np.sqrt(abs(w[c]))
            cols_a.append(ag @ V[:, c] * s)
            cols_b.append(bg @ V[:, c] * s)
            right.append(bool(w[c] > 0))
            is_prop.append(True)
            lams.append(lam[i])
    right = np.array(right)
    is_prop = np.array(is_prop)
    A = np.array(cols_a).T
    B = np.array(cols_b).T
    lams = np.array(lams)
    if right.sum() != n:
        raise ValueError(f"{right.sum()} right-going states of {2 * n}")
    return {"aR": A[:, right], "bR": B[:, right], "aL": A[:, ~right], "bL": B[:, ~right],
            "propR": is_prop[right], "propL": is_prop[~right], "lamR": lams[right], "lamL": lams[~right]}


def lead_modes(mn, G, kpar, half, tables):
    """Slice modes of a list of Fourier tables."""
    return [slice_modes(hamiltonian(mn, G, kpar, t, half)) for t in tables]


def tilt_phases(G, a3_perp):
    """D = e^{-i G . a3_perp} for the basis G (n x 2): the plane-wave
    coefficients of a field translated by a3_perp, up to the Bloch factor
    e^{-i k_perp . a3_perp} that Eq. cmp's eigenvalue carries."""
    return np.exp(-1j * (G @ np.asarray(a3_perp, dtype=np.float64)))


def translate_table(table, b1, b2, shift):
    """Fourier table of the potential moved by shift: V(r - s) has
    coefficients V(dG) e^{-i dG . s}, dG = dm b1 + dn b2 (table indexed by
    dm in [-Dm, Dm], dn in [-Dn, Dn])."""
    dm = (table.shape[0] - 1) // 2
    dn = (table.shape[1] - 1) // 2
    im = np.arange(-dm, dm + 1)[:, None]
    inn = np.arange(-dn, dn + 1)[None, :]
    dgx = im * b1[0] + inn * b2[0]
    dgy = im * b1[1] + inn * b2[1]
    return table * np.exp(-1j * (dgx * shift[0] + dgy * shift[1]))


def amplitudes_from_fields(ref_mode, E, psi, dpsi):
    """(a, b) in a slice's mode basis from psi and d psi / dz at its right
    edge: a + b = U^H psi, a - b = (i K)^-1 U^H psi'."""
    En, U = ref_mode
    k = kz(E, En)
    s = U.conj().T @ psi
    d = (U.conj().T @ dpsi) / (1j * k)[:, None]
    return 0.5 * (s + d), 0.5 * (s - d)


def electrode_states(mn, G, half, kpar, E, cell, ref, D=None):
    """The generalised Bloch states of a periodic electrode at its reference
    slice: ref = "last" (the left electrode: the cell's last slice, whose
    right edge meets the device) or "first" (the right electrode: its first
    slice).  cell = (tables, thicknesses) in order along +z.  Returns the
    reference slice's modes and the bloch_states dict."""
    tables, dz = cell
    modes = lead_modes(mn, G, kpar, half, tables)
    refm = modes[-1] if ref == "last" else modes[0]
    lam, X = complex_bands(cell_smatrix(modes, dz, E, D, ref))
    return refm, bloch_states(lam, X, refm, E)


def coset_labels(mn, c):
    """Band folding (App. B): the supercell reciprocal vectors G = m B1 + n B2
    fall into det(c) classes modulo the primitive reciprocal lattice, spanned
    by b1 = c11 B1 + c12 B2 and b2 = c21 B1 + c22 B2 (c integer); the label of
    (m, n) is its fractional coordinate in that lattice."""
    C = np.asarray(c, dtype=np.float64).T        # columns: b1, b2 in (B1, B2) coordinates
    x = np.linalg.solve(C, np.asarray(mn, dtype=np.float64).T).T
    frac = np.round(x - np.floor(x + 1e-9), 9) % 1.0
    return [tuple(f) for f in frac]


def electrode_states_folded(mn, G, half, kpar, E, cell, ref, c):
    """The same states from the primitive cell's complex bands folded into the
    supercell (App. B): for a potential with the primitive transverse period
    the Hamiltonian couples only reciprocal vectors of one class (coset) of
    coset_labels, so each class is the primitive problem at k_perp + g_c with
    its own plane waves; its Bloch states, expanded in the supercell waves
    K_perp + M B1 + N B2 of that class, are the supercell's.  Each class is
    solved alone and its states are turned into amplitudes of the full
    reference slice through their fields.  Returns (reference modes, states)
    like electrode_states."""
    tables, dz = cell
    n = len(mn)
    labels = coset_labels(mn, c)
    full_modes = lead_modes(mn, G, kpar, half, tables)
    ref_full = full_modes[-1] if ref == "last" else full_modes[0]
    cols = {"aR": [], "bR": [], "aL": [], "bL": [], "propR": [], "propL": [], "lamR": [], "lamL": []}
    for lab in sorted(set(labels)):
        idx = np.array([i for i in range(n) if labels[i] == lab])
        ref_c, st = electrode_states(mn[idx], G[idx], half, kpar, E, cell, ref)
        for side in ("R", "L"):
            psi_c, dpsi_c = edge_fields(ref_c, E, st["a" + side], st["b" + side])
            psi = np.zeros((n, psi_c.shape[1]), dtype=np.complex128)
            dpsi = np.zeros_like(psi)
            psi[idx] = psi_c
            dpsi[idx] = dpsi_c
            a, b = amplitudes_from_fields(ref_full, E, psi, dpsi)
            cols["a" + side].append(a)
            cols["b" + side].append(b)
            cols["prop" + side].append(st["prop" + side])
            cols["lam" + side].append(st["lam" + side])
    return ref_full, {k: np.concatenate(v, axis=1 if k[0] in "ab" else 0) for k, v in cols.items()}


def transmission_from_states(mn, G, half, kpar, E, dev_tables, dev_dz, left, right, right_dz0):
    """t, r, T from the electrodes' states at their reference slices (left:
    the last slice of the left electrode, right: the first slice r_1 of the
    right electrode, thickness right_dz0), as in transmission_periodic."""
    ref_l, bl = left
    ref_r, br = right
    Dm = lead_modes(mn, G, kpar, half, dev_tables)
    S11, S12, S21, S22 = chain_s([ref_l] + Dm + [ref_r], [0.0] + list(dev_dz) + [right_dz0], E)
    alpha_cols = np.nonzero(bl["propR"])[0]
    aR, bR, aL, bL = bl["aR"], bl["bR"], bl["aL"], bl["bL"]
    cR, dR = br["aR"], br["bR"]
    M = np.block([[-S11 @ aL, cR - S12 @ dR], [bL - S21 @ aL, -S22 @ dR]])
    rhs = np.vstack([S11 @ aR[:, alpha_cols], S21 @ aR[:, alpha_cols] - bR[:, alpha_cols]])
    sol = np.linalg.solve(M, rhs)
    n = len(mn)
    beta, gamma = sol[:n], sol[n:]
    t = gamma[br["propR"]]
    r = beta[bl["propL"]]
    return t, r, float(np.sum(np.abs(t) ** 2))


def transmission_periodic(mn, G, half, kpar, E, dev_tables, dev_dz, left_cell, right_cell,
                          tilt_left=None, tilt_right=None):
    """t, r and T between periodic electrodes (App. C without nonlocal terms).

    left_cell / right_cell: (tables, thicknesses) of one period, in order along
    +z; the left electrode's last period ends at the device (z = 0), the right
    electrode's first period starts at its far edge.  tilt_*: None or
    D = e^{-i G . a3_perp} of that electrode's cell.  Incident: the left
    electrode's right-going propagating states (unit flux).  Unknowns: the
    reflected left-going amplitudes beta of the left electrode and the
    transmitted right-going amplitudes gamma of the right one, from
    S(c_M, r_1) of the chain [left reference slice, device slices, r_1]:
        a_r1 = S11 a_cM + S12 b_r1,  b_cM = S21 a_cM + S22 b_r1,
        (a_cM, b_cM) = (aR, bR) alpha + (aL, bL) beta,  (a_r1, b_r1) = (aR', bR') gamma.
    Returns (t, r, T, info): t = gamma and r = beta on propagating states."""
    left = electrode_states(mn, G, half, kpar, E, left_cell, "last", tilt_left)
    right = electrode_states(mn, G, half, kpar, E, right_cell, "first", tilt_right)
    t, r, T = transmission_from_states(mn, G, half, kpar, E, dev_tables, dev_dz, left, right, right_cell[1][0])
    return t, r, T, {"left": left[1], "right": right[1]}
