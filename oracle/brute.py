"""High-precision brute-force transmission of a slice model, for pinning the
oracle.  TEST INFRASTRUCTURE ONLY (tests may import it; the product path never).

It uses none of the eigen-mode, transfer-matrix or scattering-matrix machinery
of the method.  Inside slice p the transverse-Fourier coefficients c(z) obey
c'' = (H_p - E) c (Eq. loc with the z-dependence kept), so the exact state
propagator over the slice is the matrix exponential
    [c; c'](z_p) = expm(dz_p [[0, 1], [H_p - E, 0]]) [c; c'](z_{p-1}),
evaluated with mpmath at ``dps`` significant digits.  The electrodes are
V = 0 half-spaces (plane-wave modes, no eigensolver needed), and the
incoming/outgoing/decaying conditions fix the reflected and transmitted
amplitudes through one small linear solve.  T follows with the flux factor
sqrt(k_out / k_in)."""
from __future__ import annotations

import mpmath as mp
import numpy as np


def brute_transmission(H_slices, dz, kg2_left, kg2_right, E, dps=40):
    """T and the flux-normalised t for V = 0 electrodes.

    H_slices: list of (n, n) complex Hermitian matrices H_p (numpy)
    dz: thicknesses of the slices
    kg2_left / kg2_right: |k+G|^2 of each basis vector (the free electrodes'
    transverse energies)
    Returns (T, t) with t of shape (open right, open left)."""
    mp.mp.dps = dps
    n = H_slices[0].shape[0]
    E = mp.mpf(E)
    M = mp.eye(2 * n)
    for H, d in zip(H_slices, dz):
        gen = mp.zeros(2 * n, 2 * n)
        for i in range(n):
            gen[i, n + i] = 1
            for j in range(n):
                gen[n + i, j] = mp.mpc(complex(H[i, j]))
            gen[n + i, i] -= E
        M = mp.expm(gen * mp.mpf(d)) * M

    def kvec(kg2):
        out = []
        for v in kg2:
            d = E - mp.mpf(v)
            out.append(mp.sqrt(d) if d > 0 else 1j * mp.sqrt(-d))
        return out

    kL = kvec(kg2_left)
    kR = kvec(kg2_right)
    openL = [i for i in range(n) if E > kg2_left[i]]
    openR = [i for i in range(n) if E > kg2_right[i]]
    # unknowns x = [r (n); t (n)] per incident channel j:
    #   psi(0) = e_j + r, psi'(0) = i kL (e_j - r)
    #   psi(d) = t,       psi'(d) = i kR t
    #   M [psi(0); psi'(0)] = [psi(d); psi'(d)]
    A = mp.zeros(2 * n, 2 * n)
    for row in range(2 * n):
        for c in range(n):
            A[row, c] = M[row, c] - M[row, n + c] * 1j * kL[c]
    for c in range(n):
        A[c, n + c] -= 1
        A[n + c, n + c] -= 1j * kR[c]
    t = np.zeros((len(openR), len(openL)), dtype=np.complex128)
    T = mp.mpf(0)
    for jj, j in enumerate(openL):
        b = mp.zeros(2 * n, 1)
        for row in range(2 * n):
            b[row] = -(M[row, j] + M[row, n + j] * 1j * kL[j])
        x = mp.lu_solve(A, b)
        for ii, i in enumerate(openR):
            ti = x[n + i] * mp.sqrt(kR[i] / kL[j])
            t[ii, jj] = complex(ti)
            T += abs(ti) ** 2
    return float(T), t
