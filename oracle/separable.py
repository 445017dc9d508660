"""Nonlocal (separable) pseudopotential terms for the CPU oracle: the
particular solutions of Eq. nloc, the general slice solution Eq. gsol_p0 and
the coefficients C of Eq. calm_0, solved with the interface matching as one
linear system (the M X = D of Eq. trans), without electrode-crossing
projectors.

TEST INFRASTRUCTURE ONLY, like ``pw_oracle``: nothing in the product path may
import it; it shares no code with the CUDA path.

Units and conventions (Ry, hbar^2/2m = 1).  Eq. ksep in the plane-wave basis
G of the transverse cell (area A) at k_perp:
    E psi(G, z) = -d^2/dz^2 psi + sum_G' H_p(G, G') psi(G', z) + sum_alpha C_alpha W_alpha(G, z),
    C_alpha = sum_beta D_alpha,beta <W_beta | psi>,  <W | psi> = A sum_G int dz W(G, z)^* psi(G, z),
where W_alpha(G, z) are the plane-wave coefficients of the Bloch sum of the
projector of Eq. kse0 (W(r) = sum_G W(G, z) e^{i(k+G).r}).  In slice p (modes
U, wavenumbers k) the general solution is
    psi = U (e^{ik(z - z_{p-1})} a_p + e^{-ik(z - z_p)} b_p + sum_alpha C_alpha f_alpha(z)),
with the particular solution of each mode f'' + k^2 f = w (w = U^H W_alpha):
    f(z) = int_slice g(z - z') w(z') dz',  g(u) = e^{ik|u|} / (2ik)
(the outgoing Green's function of d^2 + k^2), so f(z_a) = -f'(z_a) / ik and
f(z_b) = f'(z_b) / ik at the slice edges.  Integrals over z use Gauss-Legendre
rules per slice; the kink of g is handled by splitting the inner integral at
the outer node.  Projectors vanish in the electrodes (slices 0 and N+1).
"""
from __future__ import annotations

import numpy as np

from oracle.pw_oracle import kz, transmission_from_s


def gaussian_projector(G, kpar, area, tau, s, z_lo, z_hi):
    """W(G, z) of the Bloch sum of exp(-|r - tau|^2 / 2 s^2), restricted to
    z_lo <= z <= z_hi: (2 pi s^2 / A) e^{-|k+G|^2 s^2 / 2} e^{-i (k+G).tau_perp}
    e^{-(z - tau_z)^2 / 2 s^2}.  Returns a function of a z array (n x len(z))."""
    q = np.asarray(G) + np.asarray(kpar)[None, :]
    amp = (2.0 * np.pi * s * s / area) * np.exp(-0.5 * (q ** 2).sum(1) * s * s) * \
        np.exp(-1j * (q @ np.asarray(tau[:2], dtype=np.float64)))

    def W(z):
        z = np.asarray(z, dtype=np.float64)
        prof = np.exp(-0.5 * ((z - tau[2]) / s) ** 2) * ((z >= z_lo) & (z <= z_hi))
        return amp[:, None] * prof[None, :]
    return W


def _gl(a, b, q):
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def _slice_terms(U, k, za, zb, projs, q):
    """For one slice: the particular solutions' edge values and derivatives,
    and the overlaps that Eq. calm_0 needs (all in mode space).
    Returns fa, dfa, fb, dfb (n x nproj), Ha, Hb (nproj x n: <W_beta| e^{ik(z-za)}>,
    <W_beta| e^{-ik(z-zb)}> per mode, without the factor A) and P (nproj x nproj:
    <W_beta | U f_alpha>, without A)."""
    n = U.shape[1]
    m = len(projs)
    z, wz = _gl(za, zb, q)
    wmode = [U.conj().T @ W(z) for W in projs]             # w_alpha(z) per node: n x q
    ik = 1j * k
    fa = np.zeros((n, m), dtype=np.complex128)
    fb = np.zeros((n, m), dtype=np.complex128)
    for a in range(m):
        fa[:, a] = (wmode[a] * np.exp(ik[:, None] * (z[None, :] - za)) * wz[None, :]).sum(1) / (2 * ik)
        fb[:, a] = (wmode[a] * np.exp(ik[:, None] * (zb - z[None, :])) * wz[None, :]).sum(1) / (2 * ik)
    dfa, dfb = -ik[:, None] * fa, ik[:, None] * fb
    Ha = np.array([(np.conj(wmode[b]) * np.exp(ik[:, None] * (z[None, :] - za)) * wz[None, :]).sum(1)
                   for b in range(m)]).reshape(m, n)
    Hb = np.array([(np.conj(wmode[b]) * np.exp(-ik[:, None] * (z[None, :] - zb)) * wz[None, :]).sum(1)
                   for b in range(m)]).reshape(m, n)
    # f_alpha at the outer nodes: inner integrals split at the node
    P = np.zeros((m, m), dtype=np.complex128)
    f_nodes = np.zeros((m, n, q), dtype=np.complex128)
    for i, zi in enumerate(z):
        zl, wl = _gl(za, zi, q)
        zr, wr = _gl(zi, zb, q)
        for a in range(m):
            left = (U.conj().T @ projs[a](zl)) * np.exp(ik[:, None] * (zi - zl[None, :])) * wl[None, :]
            right = (U.conj().T @ projs[a](zr)) * np.exp(ik[:, None] * (zr[None, :] - zi)) * wr[None, :]
            f_nodes[a, :, i] = (left.sum(1) + right.sum(1)) / (2 * ik)
    for b in range(m):
        for a in range(m):
            P[b, a] = (np.conj(wmode[b]) * f_nodes[a] * wz[None, :]).sum()
    return fa, dfa, fb, dfb, Ha, Hb, P


def transmission_nonlocal(modes, dz, E, projs, D, area, q=16):
    """t, r, T and C for incidence from the left electrode, from one linear
    system of the interface matching (psi and dpsi/dz continuous at every
    z_p) and Eq. calm_0.  modes: (E_q, U_q) of slices 0..N+1 (electrodes
    first and last), dz: thicknesses of slices 1..N (the device starts at
    z = 0), projs: list of W_alpha(z) functions, D: their coefficient matrix.
    Unknowns: b_0, (a_p, b_p) for p = 1..N, a_{N+1}, C; a_0 = 1 on every
    left channel, b_{N+1} = 0.  Returns (t, r, T, a_{N+1}, C) with t and r
    flux-normalised on open channels."""
    N = len(dz)
    n = modes[0][1].shape[0]
    m = len(projs)
    D = np.atleast_2d(np.asarray(D, dtype=np.complex128)).reshape(m, m)
    ks = [kz(E, En) for En, _ in modes]
    Us = [U for _, U in modes]
    thick = [0.0] + list(dz) + [0.0]
    zs = np.concatenate([[0.0], np.cumsum(dz)])             # z_0 .. z_N
    es = [np.exp(1j * ks[p] * thick[p]) for p in range(N + 2)]
    terms = [None] + [_slice_terms(Us[p], ks[p], zs[p - 1], zs[p], projs, q) for p in range(1, N + 1)] + [None]
    nunk = 2 * n * (N + 1) + m

    def ca(p):
        return n + 2 * n * (p - 1) if p <= N else n + 2 * n * N

    def cb(p):
        return 0 if p == 0 else n + 2 * n * (p - 1) + n
    c0 = 2 * n * (N + 1)
    M = np.zeros((nunk, nunk), dtype=np.complex128)
    rhs = np.zeros((nunk, n), dtype=np.complex128)
    for p in range(N + 1):
        r0 = 2 * n * p
        Up, Uq = Us[p], Us[p + 1]
        ikp, ikq = 1j * ks[p], 1j * ks[p + 1]
        ep, eq = es[p], es[p + 1]
        q_ = p + 1
        # slice p at its right edge z_p
        if p == 0:
            rhs[r0:r0 + n] -= Up
            rhs[r0 + n:r0 + 2 * n] -= Up * ikp[None, :]
            M[r0:r0 + n, cb(0):cb(0) + n] += Up
            M[r0 + n:r0 + 2 * n, cb(0):cb(0) + n] += -Up * ikp[None, :]
        else:
            M[r0:r0 + n, ca(p):ca(p) + n] += Up * ep[None, :]
            M[r0:r0 + n, cb(p):cb(p) + n] += Up
            M[r0 + n:r0 + 2 * n, ca(p):ca(p) + n] += Up * (ikp * ep)[None, :]
            M[r0 + n:r0 + 2 * n, cb(p):cb(p) + n] += -Up * ikp[None, :]
            _, _, fb, dfb, _, _, _ = terms[p]
            M[r0:r0 + n, c0:c0 + m] += Up @ fb
            M[r0 + n:r0 + 2 * n, c0:c0 + m] += Up @ dfb
        # slice p+1 at its left edge z_p
        M[r0:r0 + n, ca(q_):ca(q_) + n] -= Uq
        M[r0 + n:r0 + 2 * n, ca(q_):ca(q_) + n] -= Uq * ikq[None, :]
        if q_ <= N:
            M[r0:r0 + n, cb(q_):cb(q_) + n] -= Uq * eq[None, :]
            M[r0 + n:r0 + 2 * n, cb(q_):cb(q_) + n] -= -Uq * (ikq * eq)[None, :]
            fa, dfa, _, _, _, _, _ = terms[q_]
            M[r0:r0 + n, c0:c0 + m] -= Uq @ fa
            M[r0 + n:r0 + 2 * n, c0:c0 + m] -= Uq @ dfa
    # Eq. calm_0: C - D A sum_p <W | psi>_p = 0
    rows = slice(c0, c0 + m)
    M[rows, c0:c0 + m] += np.eye(m)
    for p in range(1, N + 1):
        _, _, _, _, Ha, Hb, P = terms[p]
        M[rows, ca(p):ca(p) + n] -= area * D @ Ha
        M[rows, cb(p):cb(p) + n] -= area * D @ Hb
        M[rows, c0:c0 + m] -= area * D @ P
    x = np.linalg.solve(M, rhs)
    aN1 = x[ca(N + 1):ca(N + 1) + n]
    b0 = x[0:n]
    C = x[c0:c0 + m]
    EL, ER = modes[0][0], modes[-1][0]
    t, T = transmission_from_s((aN1, None, None, None), E, EL, ER)
    oL = np.nonzero(np.asarray(EL) < E)[0]
    kL = np.sqrt(E - np.asarray(EL)[oL])
    r = b0[np.ix_(oL, oL)] * np.sqrt(kL[:, None] / kL[None, :])
    return t, r, T, aN1, C
