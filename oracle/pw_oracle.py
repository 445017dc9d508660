"""Plain FP64 CPU oracle of the plane-wave multiple-scattering transport path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module; only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline do.  It shares no code with the CUDA path.

It computes, in the order and notation of Li, Chu, Zhang & Cheng (PRB 2015,
"plane-wave multiple scattering"), the transmission of a slice model of a
junction between two z-invariant electrodes:

* Sec. II A: the transverse basis {G_perp} (2D reciprocal vectors below a
  cutoff) and, for every slice p, the slice potential's Fourier coefficients
  V^p(G) (Eq. loc), here in closed form for Gaussian wells averaged over the
  slice thickness (the paper requires the potential to be z-independent inside
  a slice; the slice average is the reading taken).
* Eq. loc (= App. A Eq. A8): H_p(G,G') = |k+G|^2 delta + V^p(G-G'); its
  eigenpairs E_n^p, phi_n^p.  k_n^p = sqrt(E - E_n^p) in Ry units (the printed
  sqrt(2m(E-E_n)/hbar) lacks a square on hbar); propagating modes take the
  positive root, evanescent modes the root with positive imaginary part.
* App. A Eq. transfer: transfer matrix I(p,p+1) built from the overlaps
  sum_s (M^{p+1}_{js})^* M^p_{ns} = (U_p^H U_{p+1})_{nj}.
* App. A Eq. scatter: the interface scattering matrix S(p,p+1) from I.
* Eq. recurrence (= App. A Eq. recurrence): the star product S(m,k) of
  S(m,n) and S(n,k), applied left to right over all interfaces.
* Eq. recurrence2 (App. A, Sec. II A): layer doubling over the interfaces
  with the transfer blocks I11, I12 and the scattering blocks S21, S22 while
  cond(I11) stays below a criterion, then Eq. recurrence (``doubling``).
* App. C: with z-invariant electrodes and no nonlocal terms the electrodes
  are slices 0 and N+1, so the junction's S(0,N+1) follows from two more
  interfaces; with A^0 = I and B^{N+1} = 0 the transmission amplitudes are
  A^{N+1} = S11(0,N+1).  The flux-normalised t_ij = sqrt(k_i^R/k_j^L) S11_ij on
  open channels and T = Tr(t^H t) (Sec. II B, Eq. T1_d sums T over k_par).

Every function is pinned by the tests in ``tests/test_oracle_*.py`` against
closed forms, invariants, quadrature and an independent high-precision
brute-force solve (``oracle/brute.py``).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SHELL_QUANTUM = 1e-8   # Ry: |G|^2 values closer than this belong to the same shell


# ---------------------------------------------------------------------------
# a1: transverse basis and slice potentials (Sec. II A, Eq. loc)
# ---------------------------------------------------------------------------
def reciprocal(a1, a2):
    """2D reciprocal vectors b1, b2 with a_i . b_j = 2 pi delta_ij."""
    A = np.array([a1, a2], dtype=np.float64).T           # columns a1, a2
    B = 2.0 * math.pi * np.linalg.inv(A).T               # columns b1, b2
    return B[:, 0].copy(), B[:, 1].copy()


def gvectors(a1, a2, ecut=0.0, ng_exact=0):
    """The basis {G_perp}: integer pairs (m, n) with G = m b1 + n b2.

    ``ng_exact == 0``: every G with |G|^2 <= ecut (whole shells).
    ``ng_exact > 0``: the first ng_exact G ordered by (|G|^2, m, n).
    The order is always (shell, m, n); shells are |G|^2 quantised to
    SHELL_QUANTUM so that round-off never reorders a shell."""
    b1, b2 = reciprocal(a1, a2)
    if ng_exact > 0:
        ec = (2.0 * math.pi) ** 2 / max(np.linalg.norm(a1), np.linalg.norm(a2)) ** 2
        while True:
            mn, g2 = _enumerate(a1, a2, b1, b2, ec)
            if len(mn) >= ng_exact + 64:
                break
            ec *= 1.5
        return mn[:ng_exact], (mn[:ng_exact] @ np.array([b1, b2]))
    mn, g2 = _enumerate(a1, a2, b1, b2, ecut)
    return mn, mn @ np.array([b1, b2])


def _enumerate(a1, a2, b1, b2, ecut):
    gmax = math.sqrt(max(ecut, 0.0))
    mmax = int(math.floor(gmax * np.linalg.norm(a1) / (2 * math.pi))) + 1
    nmax = int(math.floor(gmax * np.linalg.norm(a2) / (2 * math.pi))) + 1
    rows = []
    for m in range(-mmax, mmax + 1):
        for n in range(-nmax, nmax + 1):
            g = m * b1 + n * b2
            g2 = float(g @ g)
            if g2 <= ecut:
                rows.append((round(g2 / SHELL_QUANTUM), m, n, g2))
    rows.sort(key=lambda r: (r[0], r[1], r[2]))
    mn = np.array([[r[1], r[2]] for r in rows], dtype=np.int64).reshape(-1, 2)
    g2 = np.array([r[3] for r in rows])
    return mn, g2


def table_half(mn):
    """Index ranges (Dm, Dn) of the difference vectors G - G' of a basis."""
    return int(2 * np.abs(mn[:, 0]).max()), int(2 * np.abs(mn[:, 1]).max())


def _dg_grid(a1, a2, half):
    b1, b2 = reciprocal(a1, a2)
    dm, dn = half
    im = np.arange(-dm, dm + 1)[:, None, None]
    inn = np.arange(-dn, dn + 1)[None, :, None]
    return im * b1[None, None, :] + inn * b2[None, None, :]      # (2Dm+1, 2Dn+1, 2)


def cell_area(a1, a2):
    return abs(a1[0] * a2[1] - a1[1] * a2[0])


def slice_vg_wells(a1, a2, half, wells_xyz, v0, sigma, z_lo, z_hi):
    """V^p(dG) of the wells -v0 exp(-|r-R|^2/2 sigma^2) averaged over the slice
    z in [z_lo, z_hi]:  (1/A) int_cell d^2r V e^{-i dG.r} summed over transverse
    images = -(2 pi sigma^2 / A) v0 e^{-sigma^2 |dG|^2 / 2} e^{-i dG.R_perp} w,
    w = (sigma sqrt(pi/2) / dz) [erf((z_hi-Z)/(sqrt2 sigma)) - erf((z_lo-Z)/(sqrt2 sigma))]."""
    dG = _dg_grid(a1, a2, half)
    g2 = (dG ** 2).sum(-1)
    area = cell_area(a1, a2)
    dz = z_hi - z_lo
    out = np.zeros(g2.shape, dtype=np.complex128)
    for (x, y, z), v, s in zip(wells_xyz, v0, sigma):
        w = (s * math.sqrt(math.pi / 2.0) / dz) * (
            erf((z_hi - z) / (math.sqrt(2.0) * s)) - erf((z_lo - z) / (math.sqrt(2.0) * s)))
        phase = np.exp(-1j * (dG[..., 0] * x + dG[..., 1] * y))
        out += -(2.0 * math.pi * s * s / area) * v * np.exp(-0.5 * s * s * g2) * phase * w
    return out


def lead_vg(a1, a2, half, lead):
    """Fourier table of a z-invariant electrode: the z-average over one period
    of a periodic array of wells, i.e. each well's whole z-integral
    sigma sqrt(2 pi) divided by the period."""
    dG = _dg_grid(a1, a2, half)
    g2 = (dG ** 2).sum(-1)
    area = cell_area(a1, a2)
    out = np.zeros(g2.shape, dtype=np.complex128)
    for (x, y), v, s in zip(lead.wells_xy, lead.v0, lead.sigma):
        w = s * math.sqrt(2.0 * math.pi) / lead.period
        phase = np.exp(-1j * (dG[..., 0] * x + dG[..., 1] * y))
        out += -(2.0 * math.pi * s * s / area) * v * np.exp(-0.5 * s * s * g2) * phase * w
    return out


def potential_tables(inst, half):
    """All Fourier tables of an instance: slices 1..N, then the two leads.
    Returns (slices (N, 2Dm+1, 2Dn+1), left (.,.), right (.,.))."""
    if inst.slice_vg is not None:
        return _embed_tables(inst, half)
    z = inst.z_edges
    sl = np.stack([slice_vg_wells(inst.a1, inst.a2, half, inst.wells_xyz, inst.v0,
                                  inst.sigma, z[p], z[p + 1]) for p in range(len(z) - 1)])
    return sl, lead_vg(inst.a1, inst.a2, half, inst.lead_left), \
        lead_vg(inst.a1, inst.a2, half, inst.lead_right)


def _embed_tables(inst, half):
    """Explicit tables given with their own half ranges, re-indexed to ``half``."""
    dm, dn = half
    sm, sn = inst.vg_half

    def emb(t):
        out = np.zeros((2 * dm + 1, 2 * dn + 1), dtype=np.complex128)
        for i in range(-min(dm, sm), min(dm, sm) + 1):
            for j in range(-min(dn, sn), min(dn, sn) + 1):
                out[i + dm, j + dn] = t[i + sm, j + sn]
        return out

    sl = np.stack([emb(t) for t in inst.slice_vg])
    return sl, emb(inst.lead_vg[0]), emb(inst.lead_vg[1])


# ---------------------------------------------------------------------------
# a2: slice eigenproblem (Eq. loc)
# ---------------------------------------------------------------------------
def hamiltonian(mn, G, kpar, table, half):
    """H(G_i, G_j) = |k + G_i|^2 delta_ij + V(G_i - G_j)."""
    dm, dn = half
    kg = G + np.asarray(kpar)[None, :]
    H = table[(mn[:, 0][:, None] - mn[:, 0][None, :]) + dm,
              (mn[:, 1][:, None] - mn[:, 1][None, :]) + dn].astype(np.complex128)
    H[np.diag_indices(len(mn))] += (kg ** 2).sum(-1)
    return H


def slice_modes(H):
    """Eigenvalues (ascending) and orthonormal eigenvectors (columns) of H."""
    return np.linalg.eigh(H)


def kz(E, En):
    """k_n = sqrt(E - E_n): positive real for E > E_n (propagating to +z),
    i sqrt(E_n - E) for E < E_n (decaying to +z)."""
    En = np.asarray(En, dtype=np.float64)
    d = E - En
    return np.where(d > 0, np.sqrt(np.abs(d)) + 0j, 1j * np.sqrt(np.abs(d)))


# ---------------------------------------------------------------------------
# a3-a4: overlaps, transfer matrix (Eq. transfer), interface S (Eq. scatter)
# ---------------------------------------------------------------------------
def overlap(Up, Uq):
    """sum_s (M^{q}_{js})^* M^p_{ns} with M^p_{ns} = phi_n^p(G_s)^*: (U_p^H U_q)_{nj}."""
    return Up.conj().T @ Uq


def transfer_matrix(O, kp, kq, dzq):
    """I(p,p+1) of Eq. transfer: I_nj = O_nj / (2 k_n^p) x
    [[e^{-ik_j dz}(k_n+k_j), e^{ik_j dz}(k_n-k_j)], [e^{-ik_j dz}(k_n-k_j), e^{ik_j dz}(k_n+k_j)]],
    with k_j and dz of slice p+1."""
    kn = kp[:, None]
    kj = kq[None, :]
    em = np.exp(-1j * kq * dzq)[None, :]
    ep = np.exp(1j * kq * dzq)[None, :]
    f = O / (2.0 * kn)
    I11 = f * em * (kn + kj)
    I12 = f * ep * (kn - kj)
    I21 = f * em * (kn - kj)
    I22 = f * ep * (kn + kj)
    return I11, I12, I21, I22


def smatrix_from_transfer(I11, I12, I21, I22):
    """Eq. scatter: S11 = I11^-1, S12 = -I11^-1 I12, S21 = I21 S11, S22 = I22 + I21 S12."""
    S11 = np.linalg.inv(I11)
    S12 = -S11 @ I12
    S21 = I21 @ S11
    S22 = I22 + I21 @ S12
    return S11, S12, S21, S22


def identity_s(n):
    """S(p,p) = I: S11 = S22 = 1, S12 = S21 = 0 (the identity of the star product)."""
    e = np.eye(n, dtype=np.complex128)
    z = np.zeros((n, n), dtype=np.complex128)
    return e.copy(), z, z.copy(), e.copy()


# ---------------------------------------------------------------------------
# a5: star product (Eq. recurrence)
# ---------------------------------------------------------------------------
def star(Sa, Sb):
    """S(m,k) from S(m,n) = Sa and S(n,k) = Sb (Eq. recurrence), with
    X = I - S12(m,n) S21(n,k)."""
    a11, a12, a21, a22 = Sa
    b11, b12, b21, b22 = Sb
    n = a11.shape[0]
    Xinv = np.linalg.inv(np.eye(n) - a12 @ b21)
    S11 = b11 @ Xinv @ a11
    S12 = b12 + b11 @ Xinv @ a12 @ b22
    S21 = a21 + a22 @ b21 @ Xinv @ a11
    S22 = a22 @ b22 + a22 @ b21 @ Xinv @ a12 @ b22
    return S11, S12, S21, S22


# ---------------------------------------------------------------------------
# Eq. recurrence2: layer doubling with transfer blocks I11, I12 and scattering
# blocks S21, S22 while cond(I11) stays small (App. A, last part; Sec. II A)
# ---------------------------------------------------------------------------
COND_SWITCH = 1e4   # reading: the paper does not print its switching criterion


def i11_growth(I11):
    """The switching measure of Eq. recurrence2: the 1-norm (largest absolute
    column sum) of I11.  I11 = S11^-1 with S11 bounded by flux conservation
    (its evanescent entries decay), so the norm of I11 tracks its condition
    number: it grows with the exponentials of the evanescent modes that make
    the transfer form unstable."""
    return float(np.abs(I11).sum(axis=0).max())


def mixed_from_transfer(I11, I12, I21, I22):
    """The mixed element (I11, I12, S21, S22) of one interface: the transfer
    blocks of Eq. transfer and S21 = I21 I11^-1, S22 = I22 - I21 I11^-1 I12 of
    Eq. scatter."""
    _, _, S21, S22 = smatrix_from_transfer(I11, I12, I21, I22)
    return I11, I12, S21, S22


def star_mixed(Ta, Tb):
    """Eq. recurrence2 (no nonlocal terms): the mixed element of (m,k) from
    those of (m,n) = Ta and (n,k) = Tb, with X = I11(m,n) + I12(m,n) S21(n,k):
    I11 = X I11(n,k), I12 = X I12(n,k) + I12(m,n) S22(n,k),
    S21 = S21(m,n) + S22(m,n) S21(n,k) X^-1,
    S22 = S22(m,n) S22(n,k) - S22(m,n) S21(n,k) X^-1 I12(m,n) S22(n,k)."""
    a11, a12, a21, a22 = Ta
    b11, b12, b21, b22 = Tb
    X = a11 + a12 @ b21
    Xinv = np.linalg.inv(X)
    I11 = X @ b11
    I12 = X @ b12 + a12 @ b22
    S21 = a21 + a22 @ b21 @ Xinv
    S22 = a22 @ b22 - a22 @ b21 @ Xinv @ a12 @ b22
    return I11, I12, S21, S22


def s_from_mixed(T):
    """S11 = I11^-1 and S12 = -I11^-1 I12 (Eq. scatter); S21, S22 carried over."""
    I11, I12, S21, S22 = T
    S11 = np.linalg.inv(I11)
    return S11, -S11 @ I12, S21, S22


def doubling(elements, cond_max=COND_SWITCH):
    """S of the whole stack from the mixed elements of its interfaces, in
    order, by layer doubling: neighbours are combined pairwise, level by level
    (an odd block moves up unchanged), with Eq. recurrence2 as long as every
    block's I11 has i11_growth at most cond_max; once one exceeds it, every
    block is turned into its scattering matrix (Eq. scatter) and the remaining
    levels use Eq. recurrence.  Returns (S, level), level = the number of
    doubling levels done in the mixed form."""
    blocks = list(elements)
    mixed, level = True, 0

    def too_ill(bs):
        return max(i11_growth(b[0]) for b in bs) > cond_max

    if too_ill(blocks):
        blocks, mixed = [s_from_mixed(b) for b in blocks], False
    while len(blocks) > 1:
        comb = star_mixed if mixed else star
        nxt = [comb(blocks[i], blocks[i + 1]) for i in range(0, len(blocks) - 1, 2)]
        if len(blocks) % 2:
            nxt.append(blocks[-1])
        blocks = nxt
        if mixed:
            level += 1
            if too_ill(blocks):
                blocks, mixed = [s_from_mixed(b) for b in blocks], False
    S = s_from_mixed(blocks[0]) if mixed else blocks[0]
    return S, level


# ---------------------------------------------------------------------------
# whole path for one instance and k_par
# ---------------------------------------------------------------------------
class Model:
    """Basis, tables and slice geometry of one instance (independent of E, k)."""

    def __init__(self, inst):
        self.inst = inst
        self.mn, self.G = gvectors(inst.a1, inst.a2, inst.ecut, inst.ng_exact)
        self.half = table_half(self.mn)
        self.tables, self.vl, self.vr = potential_tables(inst, self.half)
        z = inst.z_edges
        self.dz = np.diff(z)
        self.n = len(self.mn)
        self.N = len(self.dz)

    def all_tables(self):
        """Tables in slice order 0 (left lead), 1..N, N+1 (right lead)."""
        return [self.vl] + list(self.tables) + [self.vr]

    def modes(self, kpar):
        """Eigenpairs of every slice 0..N+1 at this k_par (independent of E)."""
        return [slice_modes(hamiltonian(self.mn, self.G, kpar, t, self.half))
                for t in self.all_tables()]

    def thickness(self, q):
        """dz of slice q; the right electrode (q = N+1) carries no phase."""
        return self.dz[q - 1] if 1 <= q <= self.N else 0.0

    def interface_s(self, modes, E, p):
        """S(p, p+1) of Eqs. transfer and scatter."""
        (Ep, Up), (Eq, Uq) = modes[p], modes[p + 1]
        O = overlap(Up, Uq)
        return smatrix_from_transfer(*transfer_matrix(O, kz(E, Ep), kz(E, Eq),
                                                      self.thickness(p + 1)))

    def interface_mixed(self, modes, E, p):
        """The mixed element (I11, I12, S21, S22) of interface (p, p+1)."""
        (Ep, Up), (Eq, Uq) = modes[p], modes[p + 1]
        O = overlap(Up, Uq)
        return mixed_from_transfer(*transfer_matrix(O, kz(E, Ep), kz(E, Eq), self.thickness(p + 1)))

    def total_s_doubling(self, modes, E, cond_max=COND_SWITCH):
        """S(0, N+1) by layer doubling with Eq. recurrence2 while the growth of
        I11 stays <= cond_max, then Eq. recurrence; returns (S, mixed levels)."""
        return doubling([self.interface_mixed(modes, E, p) for p in range(self.N + 1)], cond_max)

    def total_s(self, modes, E, p0=0, p1=None):
        """S(p0, p1) by applying Eq. recurrence left to right."""
        p1 = self.N + 1 if p1 is None else p1
        S = identity_s(self.n)
        for p in range(p0, p1):
            S = star(S, self.interface_s(modes, E, p))
        return S


def open_channels(E, En):
    return np.nonzero(np.asarray(En) < E)[0]


def transmission_from_s(S, E, EL, ER):
    """Flux-normalised t_ij = sqrt(k_i^R / k_j^L) S11_ij on open channels and
    T = sum |t_ij|^2 (App. C: A^0 = I, B^{N+1} = 0 gives t = A^{N+1})."""
    oL = open_channels(E, EL)
    oR = open_channels(E, ER)
    kL = np.sqrt(E - np.asarray(EL)[oL])
    kR = np.sqrt(E - np.asarray(ER)[oR])
    t = S[0][np.ix_(oR, oL)] * np.sqrt(kR[:, None] / kL[None, :])
    return t, float(np.sum(np.abs(t) ** 2))


def flux_smatrix(S, E, EL, ER):
    """The flux-normalised scattering matrix on open channels,
    [[t, t'], [r, r']] with rows (right out, left out) and columns
    (left in, right in).  Unitary for a Hermitian slice model."""
    oL = open_channels(E, EL)
    oR = open_channels(E, ER)
    kL = np.sqrt(E - np.asarray(EL)[oL])
    kR = np.sqrt(E - np.asarray(ER)[oR])
    kout = np.concatenate([kR, kL])
    kin = np.concatenate([kL, kR])
    blk = np.block([[S[0][np.ix_(oR, oL)], S[1][np.ix_(oR, oR)]],
                    [S[2][np.ix_(oL, oL)], S[3][np.ix_(oL, oR)]]])
    return blk * np.sqrt(kout[:, None] / kin[None, :])


def transmission(inst, points=None, model=None, return_t=False):
    """T(E, k_par) for every point of the instance (or the given index list).
    Returns an array of T (and the list of t matrices when asked)."""
    model = model or Model(inst)
    idx = range(len(inst.energies)) if points is None else points
    Ts, ts = [], []
    cache = {}
    for i in idx:
        E = float(inst.energies[i])
        k = tuple(np.asarray(inst.kpar[i], dtype=np.float64))
        if k not in cache:
            cache.clear()
            cache[k] = model.modes(np.array(k))
        modes = cache[k]
        S = model.total_s(modes, E)
        t, T = transmission_from_s(S, E, modes[0][0], modes[-1][0])
        Ts.append(T)
        ts.append(t)
    Ts = np.array(Ts)
    return (Ts, ts) if return_t else Ts


# ---------------------------------------------------------------------------
# second formulation (for pins): one dense linear system of all interface
# matching conditions, no transfer or scattering matrices
# ---------------------------------------------------------------------------
def transmission_dense(model, modes, E):
    """Continuity of psi and d psi/dz at every interface in the G basis,
    solved as one linear system.  Unknowns: slice amplitudes a_p (forward,
    referenced at the slice's left edge) and b_p (backward, referenced at its
    right edge) for p = 1..N, the reflected b_0 and the transmitted a_{N+1};
    incident a_0 = I on the left electrode's open channels, b_{N+1} = 0.
    Returns S11(0,N+1) restricted to the incident columns (all left channels)."""
    n, N = model.n, model.N
    ks = [kz(E, Ep) for Ep, _ in modes]
    Us = [U for _, U in modes]
    es = [np.exp(1j * ks[q] * model.thickness(q)) for q in range(N + 2)]
    nunk = 2 * n * (N + 1)
    # unknown layout: [b_0, (a_1, b_1), ..., (a_N, b_N), a_{N+1}]
    def col_a(q):
        return n + 2 * n * (q - 1) if q <= N else n + 2 * n * N

    def col_b(q):
        return 0 if q == 0 else n + 2 * n * (q - 1) + n

    M = np.zeros((nunk, nunk), dtype=np.complex128)
    rhs = np.zeros((nunk, n), dtype=np.complex128)
    for p in range(N + 1):
        r0 = 2 * n * p
        Up, Uq = Us[p], Us[p + 1]
        kp, kq = ks[p], ks[p + 1]
        ep, eq = es[p], es[p + 1]
        # left side (slice p) at z_p:  U_p (e_p a_p + b_p);  U_p K_p (e_p a_p - b_p)
        if p == 0:
            rhs[r0:r0 + n] -= Up                      # incident a_0 = I
            rhs[r0 + n:r0 + 2 * n] -= Up * kp[None, :]
            M[r0:r0 + n, col_b(0):col_b(0) + n] += Up
            M[r0 + n:r0 + 2 * n, col_b(0):col_b(0) + n] += -Up * kp[None, :]
        else:
            ca, cb = col_a(p), col_b(p)
            M[r0:r0 + n, ca:ca + n] += Up * ep[None, :]
            M[r0:r0 + n, cb:cb + n] += Up
            M[r0 + n:r0 + 2 * n, ca:ca + n] += Up * (kp * ep)[None, :]
            M[r0 + n:r0 + 2 * n, cb:cb + n] += -Up * kp[None, :]
        # right side (slice p+1) at z_p: U_q (a_q + e_q b_q); U_q K_q (a_q - e_q b_q)
        q = p + 1
        ca = col_a(q)
        M[r0:r0 + n, ca:ca + n] -= Uq
        M[r0 + n:r0 + 2 * n, ca:ca + n] -= Uq * kq[None, :]
        if q <= N:
            cb = col_b(q)
            M[r0:r0 + n, cb:cb + n] -= Uq * eq[None, :]
            M[r0 + n:r0 + 2 * n, cb:cb + n] -= -Uq * (kq * eq)[None, :]
    x = np.linalg.solve(M, rhs)
    return x[col_a(N + 1):col_a(N + 1) + n], x[0:n]


# ---------------------------------------------------------------------------
# adjoint (derivative of T with respect to slice Hamiltonians), for pw_grad
# ---------------------------------------------------------------------------
def dense_amplitudes(model, modes, E, inc_left, inc_right):
    """All slice amplitudes from one dense solve of the interface matching
    conditions (as in transmission_dense), for given incoming amplitudes:
    inc_left = a_0 (n x m, forward waves in the left electrode) and
    inc_right = b_{N+1} (n x m, backward waves in the right electrode,
    referenced at the right edge of the device).  Returns lists a[q], b[q]
    (q = 0..N+1) of n x m arrays; a[0] and b[N+1] are the given ones."""
    n, N = model.n, model.N
    ks = [kz(E, Ep) for Ep, _ in modes]
    Us = [U for _, U in modes]
    es = [np.exp(1j * ks[q] * model.thickness(q)) for q in range(N + 2)]
    m = inc_left.shape[1]
    # unknowns: b_0, (a_q, b_q) q = 1..N, a_{N+1}
    def ca(q):
        return n + 2 * n * (q - 1) if q <= N else n + 2 * n * N

    def cb(q):
        return 0 if q == 0 else n + 2 * n * (q - 1) + n

    nunk = 2 * n * (N + 1)
    M = np.zeros((nunk, nunk), dtype=np.complex128)
    rhs = np.zeros((nunk, m), dtype=np.complex128)
    for p in range(N + 1):
        r0 = 2 * n * p
        Up, Uq, kp, kq, ep, eq = Us[p], Us[p + 1], ks[p], ks[p + 1], es[p], es[p + 1]
        q = p + 1
        # left side (slice p) at z_p
        if p == 0:
            rhs[r0:r0 + n] -= Up @ inc_left
            rhs[r0 + n:r0 + 2 * n] -= (Up * kp[None, :]) @ inc_left
            M[r0:r0 + n, cb(0):cb(0) + n] += Up
            M[r0 + n:r0 + 2 * n, cb(0):cb(0) + n] += -Up * kp[None, :]
        else:
            M[r0:r0 + n, ca(p):ca(p) + n] += Up * ep[None, :]
            M[r0:r0 + n, cb(p):cb(p) + n] += Up
            M[r0 + n:r0 + 2 * n, ca(p):ca(p) + n] += Up * (kp * ep)[None, :]
            M[r0 + n:r0 + 2 * n, cb(p):cb(p) + n] += -Up * kp[None, :]
        # right side (slice q) at z_p
        M[r0:r0 + n, ca(q):ca(q) + n] -= Uq
        M[r0 + n:r0 + 2 * n, ca(q):ca(q) + n] -= Uq * kq[None, :]
        if q <= N:
            M[r0:r0 + n, cb(q):cb(q) + n] -= Uq * eq[None, :]
            M[r0 + n:r0 + 2 * n, cb(q):cb(q) + n] -= -Uq * (kq * eq)[None, :]
        else:
            rhs[r0:r0 + n] += Uq @ inc_right
            rhs[r0 + n:r0 + 2 * n] += -(Uq * kq[None, :]) @ inc_right
    x = np.linalg.solve(M, rhs)
    a = [inc_left] + [x[ca(q):ca(q) + n] for q in range(1, N + 2)]
    b = [x[cb(q):cb(q) + n] for q in range(0, N + 1)] + [inc_right]
    return a, b


def _slice_integrals(k, dz):
    """J1(m,n) = int_0^dz e^{i(k_m+k_n)s} ds and
    J2(m,n) = int_0^dz e^{i k_m s} e^{i k_n (dz - s)} ds (closed forms)."""
    km = k[:, None]
    kn = k[None, :]
    s = km + kn
    with np.errstate(divide="ignore", invalid="ignore"):
        J1 = np.where(np.abs(s) * dz < 1e-12, dz, (np.exp(1j * s * dz) - 1.0) / (1j * s))
        d = km - kn
        em = np.exp(1j * km * dz)
        en = np.exp(1j * kn * dz)
        J2 = np.where(np.abs(d) * dz < 1e-12, dz * em, (em - en) / (1j * np.where(d == 0, 1.0, d)))
    return J1, J2


def _edge_values(U, k, amp_f, amp_b):
    """psi and dpsi/dz at the reference plane of a slice's forward amplitudes
    (psi = U (e^{ikz} amp_f + e^{-ikz} amp_b) there)."""
    return U @ (amp_f + amp_b), 1j * (U * k[None, :]) @ (amp_f - amp_b)


def grad_T(model, kpar, E, dH_list, lead_shift=None):
    """T(E, k_par) and its derivatives dT/dtheta for parameters that change
    the device slices' Hamiltonians by dH_p/dtheta (dH_list[theta][p-1],
    p = 1..N; None for no device change) and, optionally, translate the two
    electrode potentials transversally at the rates lead_shift[theta] =
    (r_L, r_R) (2-vectors, bohr per unit theta).

    For the slice ODE c'' = (H(z) - E) c, a solution d of the transposed
    problem (H^T) incident from the right electrode in channel i and the
    scattering state c_j incident from the left satisfy
        W(+inf) - W(-inf) = 2 i k_i^R dt_ij,   W = d^T c' - d'^T c,
    and dW/dz = d^T dH c, so a smooth device change gives
        dT = sum_ij Im(conj(t_ij) int d_i^T dH c_j dz) / k_j^L.
    Inside slice p the z-integral of the mode exponentials is closed-form.

    An electrode translated by delta has H' = D H D^H with
    D = diag(e^{-i G.delta}), whose modes are D U.  In the unperturbed
    electrode basis the perturbed state is D^H c on the electrode's side of
    its contact plane and c on the device side, so W jumps there by
    -/+ i (d^T Gd c' - d'^T Gd c), Gd = diag(G.delta) (minus at the left
    contact z = 0, plus at the right contact z = z_N); that jump takes the
    place of the integral."""
    modes = model.modes(kpar)
    n, N = model.n, model.N
    EL, ER = modes[0][0], modes[-1][0]
    oL, oR = open_channels(E, EL), open_channels(E, ER)
    kL = np.sqrt(E - EL[oL])
    kR = np.sqrt(E - ER[oR])
    I = np.eye(n, dtype=np.complex128)
    a, b = dense_amplitudes(model, modes, E, I[:, oL], np.zeros((n, len(oL)), complex))
    t = a[N + 1][oR, :]
    T = float(np.sum((kR[:, None] / kL[None, :]) * np.abs(t) ** 2))
    tmodes = [(Ep, U.conj()) for Ep, U in modes]
    ap, bp = dense_amplitudes(model, tmodes, E, np.zeros((n, len(oR)), complex), I[:, oR])
    W = np.conj(t) / kL[None, :]                       # (nR, nL)
    grads = []
    for th, dH in enumerate(dH_list):
        g = 0.0
        if dH is not None:
            for p in range(1, N + 1):
                U = modes[p][1]
                k = kz(E, modes[p][0])
                J1, J2 = _slice_integrals(k, model.dz[p - 1])
                D = U.conj().T @ dH[p - 1] @ U
                Gam = J1 * (ap[p] @ W @ a[p].T + bp[p] @ W @ b[p].T) + \
                    J2 * (ap[p] @ W @ b[p].T + bp[p] @ W @ a[p].T)
                g += np.imag(np.sum(D * Gam))
        if lead_shift is not None and lead_shift[th] is not None:
            for side, q, sign in ((0, 0, -1.0), (1, N + 1, 1.0)):
                Gd = model.G @ np.asarray(lead_shift[th][side], dtype=np.float64)
                if not np.any(Gd):
                    continue
                k = kz(E, modes[q][0])
                c, cp = _edge_values(modes[q][1], k, a[q], b[q])
                d, dp = _edge_values(tmodes[q][1], k, ap[q], bp[q])
                X = sign * 1j * (d.T @ (Gd[:, None] * cp) - dp.T @ (Gd[:, None] * c))
                g += np.imag(np.sum(W * X))
        grads.append(g)
    return T, np.array(grads)


def well_shift_derivative(model, rates):
    """dH_p/dtheta when every device well i moves transversally at the rate
    rates[i] (2-vector, bohr per unit theta): each well's slice table picks up
    the factor -i dG.rates[i] (its Fourier phase is e^{-i dG.R_i})."""
    inst = model.inst
    z = inst.z_edges
    dG = _dg_grid(inst.a1, inst.a2, model.half)
    per = []
    for p in range(model.N):
        tab = np.zeros(dG.shape[:2], dtype=np.complex128)
        for i in range(len(inst.v0)):
            r = np.asarray(rates[i], dtype=np.float64)
            if not np.any(r):
                continue
            ti = slice_vg_wells(inst.a1, inst.a2, model.half, inst.wells_xyz[i:i + 1],
                                inst.v0[i:i + 1], inst.sigma[i:i + 1], z[p], z[p + 1])
            tab += -1j * (dG[..., 0] * r[0] + dG[..., 1] * r[1]) * ti
        dH = hamiltonian(model.mn, model.G, np.zeros(2), tab, model.half)
        dH[np.diag_indices(model.n)] -= ((model.G) ** 2).sum(-1)   # no kinetic part
        per.append(dH)
    return per


def well_depth_derivatives(model):
    """dH_p/dV0_i for every device well i and slice p: the slice table of well i
    alone divided by its depth (the tables are linear in V0)."""
    inst = model.inst
    z = inst.z_edges
    out = []
    for i in range(len(inst.v0)):
        per = []
        for p in range(model.N):
            tab = slice_vg_wells(inst.a1, inst.a2, model.half, inst.wells_xyz[i:i + 1],
                                 np.ones(1), inst.sigma[i:i + 1], z[p], z[p + 1])
            dH = hamiltonian(model.mn, model.G, np.zeros(2), tab, model.half)
            dH[np.diag_indices(model.n)] -= ((model.G) ** 2).sum(-1)   # no kinetic part
            per.append(dH)
        out.append(per)
    return out
