"""A finite-difference solve of the continuous-z problem, for a convergence
pin of the slice model.

TEST INFRASTRUCTURE ONLY, like ``pw_oracle``: nothing in the product path may
import it; it shares no code with the CUDA path, nor with the slice model of
``pw_oracle`` (it evaluates the wells' potential at each height itself and
never forms slices, modes, overlaps or S-matrices).

The problem: E psi = -laplacian psi + V(r) psi in the transverse plane-wave
basis G (coefficients psi_G(z)), V the Gaussian wells -v0 exp(-|r - R|^2 /
2 sigma^2) (with their transverse periodic images) for 0 <= z <= L and 0
outside (free electrodes).  Three-point differences on z_j = j h turn it into
    psi_{j-1} - (2 + h^2 (H(z_j) - E)) psi_j + psi_{j+1} = 0,
H(z)_{GG'} = |k+G|^2 delta + V_{G-G'}(z).  In the free electrodes the discrete
plane waves e^{+-i kappa z} with 2 - 2 cos(kappa h) = h^2 (E - |k+G|^2) solve
the scheme exactly, which gives exact discrete transparent conditions; the
transmitted flux of a discrete wave is proportional to sin(kappa h).  T is
second order in h; Richardson extrapolation over h, h/2, h/4 gives the
continuum value to about 1e-6 and better.
"""
from __future__ import annotations

import numpy as np


def wells_vg(G, area, wells_xyz, v0, sigma, z):
    """V_{dG}(z) for every pair of basis vectors: -(2 pi sigma^2 / A) sum_i v0_i
    e^{-sigma^2 |dG|^2 / 2} e^{-i dG . R_i} e^{-(z - Z_i)^2 / 2 sigma^2}
    (the transverse Fourier integral over the plane includes the images)."""
    dG = G[:, None, :] - G[None, :, :]
    out = np.zeros((len(G), len(G)), dtype=np.complex128)
    for (x, y, zz), v, s in zip(wells_xyz, v0, sigma):
        ph = np.exp(-1j * (dG[..., 0] * x + dG[..., 1] * y))
        out += -(2 * np.pi * s * s / area) * v * np.exp(-0.5 * s * s * (dG ** 2).sum(-1)) * ph * \
            np.exp(-0.5 * ((z - zz) / s) ** 2)
    return out


def _kappa(eps, h):
    """Discrete wavenumber of the three-point scheme, Re >= 0 and Im >= 0."""
    c = 1.0 - 0.5 * h * h * eps.astype(np.complex128)
    kap = np.arccos(c) / h
    kap = np.where(kap.imag < 0, -kap, kap)
    return kap


def transmission_fd(G, kpar, E, area, wells_xyz, v0, sigma, L, h):
    """T from the left electrode by the three-point scheme with step h = L / J:
    unknowns psi_0 .. psi_J (blocks of n), block-tridiagonal elimination."""
    n = len(G)
    J = int(round(L / h))
    h = L / J
    eps = E - ((G + np.asarray(kpar)[None, :]) ** 2).sum(1)
    kap = _kappa(eps, h)
    e1 = np.exp(1j * kap * h)
    opn = np.nonzero(eps > 0)[0]
    Id = np.eye(n, dtype=np.complex128)
    T = 0.0
    # diagonal blocks; the boundary rows fold in psi_{-1} and psi_{J+1}
    diag = [-(2.0 * Id + h * h * (np.diag(((G + kpar) ** 2).sum(1)) + wells_vg(G, area, wells_xyz, v0, sigma, j * h)
                                   - E * Id)) for j in range(J + 1)]
    # left: psi_{-1} = d e^{-i kap h} + (psi_0 - d) e^{i kap h}  (d: incident amplitudes)
    diag[0] = diag[0] + np.diag(e1)
    # right: psi_{J+1} = psi_J e^{i kap h}
    diag[J] = diag[J] + np.diag(e1)
    for g_in in opn:
        d = np.zeros(n, dtype=np.complex128)
        d[g_in] = 1.0
        rhs = [np.zeros(n, dtype=np.complex128) for _ in range(J + 1)]
        rhs[0] = -(d * (np.exp(-1j * kap * h) - e1))
        # block Thomas: off-diagonal blocks are the identity
        Dp = [None] * (J + 1)
        yp = [None] * (J + 1)
        Dp[0] = diag[0]
        yp[0] = rhs[0]
        for j in range(1, J + 1):
            inv_prev = np.linalg.solve(Dp[j - 1], np.column_stack([Id, yp[j - 1]]))
            Dp[j] = diag[j] - inv_prev[:, :n]
            yp[j] = rhs[j] - inv_prev[:, n]
        # the right electrode holds t_G e^{i kap j h} for j >= J
        t = np.linalg.solve(Dp[J], yp[J]) * np.exp(-1j * kap * J * h)
        flux = np.sin(kap[opn].real * h)
        T += float(np.sum(np.abs(t[opn]) ** 2 * flux) / np.sin(kap[g_in].real * h))
    return T


def richardson(values, order=2):
    """Extrapolate T(h) = T0 + c2 h^2 + c4 h^4 + ... from values at h, h/2,
    h/4, ... (two levels of Richardson for three values)."""
    v = list(values)
    p = order
    while len(v) > 1:
        r = 2.0 ** p
        v = [(r * v[i + 1] - v[i]) / (r - 1.0) for i in range(len(v) - 1)]
        p += 2
    return v[0]
