"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Element-by-element comparisons on seeded synthetic inputs that span several
GEMM/LU tiles and ragged edges (N_G = 1, 5, 21, 64, 97 ...), plus the
closed-form and invariant cases.  FP64 bar: 1e-10 relative on T."""
import math

import numpy as np
import pytest

from oracle import pw_oracle as O
from synthetic import (explicit_barrier, explicit_tables, junction, minimal_cell,
                       random_tables)
from tests.parity import TOL_FP64, TOL_MIXED, rel_T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pw():
    import __graft_entry__ as g
    g.build()
    import paper_1504_01462_gb300 as pw
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pw


def _dev(shape, dtype):
    return torch.zeros(shape, dtype=dtype, device="cuda")


def _gpu_T(pw, inst, precision=0, E=None, k=None, with_t=False, refine_iters=0, with_err=False):
    E = inst.energies if E is None else E
    k = inst.kpar if k is None else k
    with pw.Context.from_instance(inst, precision=precision, refine_iters=refine_iters) as ctx:
        n = ctx.ng
        T = _dev(len(E), torch.float64)
        t = _dev((len(E), n, n), torch.complex128) if with_t else None
        nop = _dev((len(E), 2), torch.int32)
        err = _dev(len(E), torch.float64)
        ctx.transmission(E, k, T, t, nop, err)
        torch.cuda.synchronize()
        out = (T.cpu().numpy(), (t.cpu().numpy() if with_t else None), nop.cpu().numpy())
        return out + (err.cpu().numpy(),) if with_err else out


def _rel(a, b):
    return rel_T(a, b)


# ---------------------------------------------------------------------------
# a1: basis and tables
# ---------------------------------------------------------------------------
def test_basis_matches_oracle(pw):
    for inst in (minimal_cell(), junction(ng=512, n_slices=4, n_e=1, n_k=1),
                 junction(ng=0, ecut=29.34, n_slices=4, n_e=1, n_k=1)):
        mn, _ = O.gvectors(inst.a1, inst.a2, inst.ecut, inst.ng_exact)
        with pw.Context.from_instance(inst) as ctx:
            assert np.array_equal(ctx.gvectors(), mn)


def test_potential_tables_match_oracle(pw):
    inst = minimal_cell()
    m = O.Model(inst)
    with pw.Context.from_instance(inst) as ctx:
        half = ctx.table_half()
        assert half == m.half
        out = _dev((m.N + 2, 2 * half[0] + 1, 2 * half[1] + 1), torch.complex128)
        ctx.potential_tables(out)
        got = out.cpu().numpy()
    ref = np.stack(m.all_tables())
    assert np.abs(got - ref).max() < 1e-13
    # junction: z-averaged electrodes and 48 wells
    inst = junction(ng=128, n_slices=12, n_e=1, n_k=1)
    m = O.Model(inst)
    with pw.Context.from_instance(inst) as ctx:
        half = ctx.table_half()
        out = _dev((m.N + 2, 2 * half[0] + 1, 2 * half[1] + 1), torch.complex128)
        ctx.potential_tables(out)
        got = out.cpu().numpy()
    assert np.abs(got - np.stack(m.all_tables())).max() < 1e-13


# ---------------------------------------------------------------------------
# a2, a3: eigenmodes and overlaps
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ng,nsl", [(21, 16), (97, 6), (21, 330)])
def test_slice_modes_against_oracle_hamiltonians(pw, ng, nsl):
    """FP64 eigenmodes and overlaps.  The last case's 332 matrices are more
    than the solver holds at once (pw_eig_wave: two per SM at this order on a
    152-SM GPU), so its partial last wave runs on the side stream beside the
    overlaps of the slices done before it, and the remaining overlaps follow."""
    if nsl == 330:
        assert 0 < pw.eig_wave(21) < nsl + 2
    _check_slice_modes(pw, ng, nsl, precision=0, tol=1.0)


@pytest.mark.parametrize("ng,nsl", [(21, 4), (64, 3), (512, 2), (21, 330)])
def test_slice_modes_double_float_mixed_form(pw, ng, nsl):
    """The mixed form's double-float eigensolver and overlaps (launch variant
    bit 5; 48-bit arithmetic on the FP32 pipe): same checks, 10x looser.  332
    matrices exceed two per SM on a 152-SM GPU, so the last case also covers
    the reduction tail on the second stream."""
    _check_slice_modes(pw, ng, nsl, precision=1, tol=10.0)


def _check_slice_modes(pw, ng, nsl, precision, tol):
    if ng == 21:
        inst = minimal_cell(n_slices=nsl)
        k = np.array([0.13, -0.27])
    else:
        inst = junction(ng=ng, n_slices=nsl, n_e=1, n_k=1)
        k = np.array([0.21, 0.0])
    m = O.Model(inst)
    n, nq = m.n, m.N + 2
    with pw.Context.from_instance(inst, precision) as ctx:
        if precision == 1:
            ctx.set_sweep_variant(2 | 32)      # the double-float mode stage
        En = _dev((nq, n), torch.float64)
        U = _dev((nq, n, n), torch.complex128)
        Ov = _dev((nq - 1, n, n), torch.complex128)
        ctx.slice_modes(k, En, U)
        ctx.overlaps(k, Ov)
        torch.cuda.synchronize()
        En, U, Ov = En.cpu().numpy(), U.cpu().numpy(), Ov.cpu().numpy()
    # device buffers are column-major n x n: U[q][j][i] = component i of vector j
    U = np.transpose(U, (0, 2, 1))
    Ov = np.transpose(Ov, (0, 2, 1))
    for q, tab in enumerate(m.all_tables()):
        H = O.hamiltonian(m.mn, m.G, k, tab, m.half)
        ref = np.linalg.eigvalsh(H)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(En[q] - ref).max() < 1e-12 * tol * scale
        assert np.abs(H @ U[q] - U[q] * En[q][None, :]).max() < 1e-11 * tol * scale
        assert np.abs(U[q].conj().T @ U[q] - np.eye(n)).max() < 1e-12 * tol
    for p in range(nq - 1):
        assert np.abs(Ov[p] - O.overlap(U[p], U[p + 1])).max() < 1e-12 * tol


# ---------------------------------------------------------------------------
# a4: interface S-matrix;  a5: star product
# ---------------------------------------------------------------------------
def _modes_from_gpu(pw, ctx, k, n, nq):
    En = _dev((nq, n), torch.float64)
    U = _dev((nq, n, n), torch.complex128)
    ctx.slice_modes(k, En, U)
    torch.cuda.synchronize()
    return En.cpu().numpy(), np.transpose(U.cpu().numpy(), (0, 2, 1))


def test_interface_smatrix_matches_eq_scatter(pw):
    inst = minimal_cell(n_slices=16)
    m = O.Model(inst)
    k = np.array([0.1, -0.2])
    E = np.array([0.7, 2.3, 3.9])
    n, nq = m.n, m.N + 2
    with pw.Context.from_instance(inst) as ctx:
        En, U = _modes_from_gpu(pw, ctx, k, n, nq)
        for iface in (0, 5, m.N):
            S = _dev((len(E), 4, n, n), torch.complex128)
            ctx.slice_smatrix(E, np.repeat(k[None], len(E), 0), iface, S)
            torch.cuda.synchronize()
            S = np.transpose(S.cpu().numpy(), (0, 1, 3, 2))
            for i, e in enumerate(E):
                Oi = O.overlap(U[iface], U[iface + 1])
                ref = O.smatrix_from_transfer(*O.transfer_matrix(
                    Oi, O.kz(e, En[iface]), O.kz(e, En[iface + 1]), m.thickness(iface + 1)))
                for b in range(4):
                    scale = max(1.0, np.abs(ref[b]).max())
                    assert np.abs(S[i, b] - ref[b]).max() < 1e-11 * scale, (iface, e, b)


def test_compose_matches_eq_recurrence(pw):
    inst = minimal_cell(n_slices=16)
    m = O.Model(inst)
    k = np.array([0.05, 0.3])
    E = np.array([1.1, 2.9])
    n = m.n
    with pw.Context.from_instance(inst) as ctx:
        Sa = _dev((len(E), 4, n, n), torch.complex128)
        Sb = _dev((len(E), 4, n, n), torch.complex128)
        Sab = _dev((len(E), 4, n, n), torch.complex128)
        kk = np.repeat(k[None], len(E), 0)
        ctx.slice_smatrix(E, kk, 3, Sa)
        ctx.slice_smatrix(E, kk, 4, Sb)
        ctx.compose(len(E), Sa, Sb, Sab)
        torch.cuda.synchronize()
        A = np.transpose(Sa.cpu().numpy(), (0, 1, 3, 2))
        B = np.transpose(Sb.cpu().numpy(), (0, 1, 3, 2))
        C = np.transpose(Sab.cpu().numpy(), (0, 1, 3, 2))
    for i in range(len(E)):
        ref = O.star(tuple(A[i]), tuple(B[i]))
        for b in range(4):
            assert np.abs(C[i, b] - ref[b]).max() < 1e-11 * max(1.0, np.abs(ref[b]).max())


# ---------------------------------------------------------------------------
# a1-a6: the whole forward path, FP64
# ---------------------------------------------------------------------------
def test_transmission_minimal_cell_fp64(pw):
    E = np.array([0.5, 2.3, 3.9, 2.3, 5.5, 0.9])
    k = np.array([[0.0, 0.0], [0.1, -0.2], [0.1, -0.2], [-0.3, 0.25], [0.0, 0.0], [0.6, 0.1]])
    inst = minimal_cell(energies=E, kpar=k)
    ref, ref_t = O.transmission(inst, return_t=True)
    got, t, nop = _gpu_T(pw, inst, 0, with_t=True)
    assert np.all(_rel(got, ref) < TOL_FP64), (got, ref)
    for i in range(len(E)):
        nR, nL = ref_t[i].shape
        assert tuple(nop[i]) == (nL, nR)
        # V = 0 electrodes: the channel basis is the plane waves, so t is unique
        ti = t[i].T[:nR, :nL]
        assert np.abs(ti - ref_t[i]).max() < 1e-10 * max(1.0, np.abs(ref_t[i]).max())


def test_transmission_barrier_closed_form(pw):
    for E, V, d, kk, nsl in [(0.5, 0.3, 1.3, (0.0, 0.0), 3), (0.5, 0.8, 1.3, (0.0, 0.0), 4),
                             (0.9, 0.5, 0.7, (0.3, -0.2), 2), (0.4, 1.5, 3.0, (0.1, 0.1), 7)]:
        inst = explicit_barrier([V] * nsl, [d / nsl] * nsl, energies=(E,), kpar=(kk,))
        got, _, _ = _gpu_T(pw, inst, 0)
        eps = E - kk[0] ** 2 - kk[1] ** 2
        if eps > V:
            q = math.sqrt(eps - V)
            Tc = 1 / (1 + V * V * math.sin(q * d) ** 2 / (4 * eps * (eps - V)))
        else:
            kap = math.sqrt(V - eps)
            Tc = 1 / (1 + V * V * math.sinh(kap * d) ** 2 / (4 * eps * (V - eps)))
        assert abs(got[0] - Tc) < 1e-12


def test_free_device_counts_channels(pw):
    E = np.array([0.5, 3.0, 2.2, 6.0])
    k = np.array([[0.0, 0.0], [0.0, 0.0], [0.21, -0.4], [0.5, 0.5]])
    inst = minimal_cell(energies=E, kpar=k)
    inst.v0[:] = 0.0
    got, _, nop = _gpu_T(pw, inst, 0)
    mn, G = O.gvectors(inst.a1, inst.a2, inst.ecut, 0)
    for i in range(len(E)):
        nopen = int((((G + k[i]) ** 2).sum(1) < E[i]).sum())
        assert abs(got[i] - nopen) < 1e-11
        assert tuple(nop[i]) == (nopen, nopen)


@pytest.mark.parametrize("seed", [1, 2])
def test_transmission_random_tables_ragged(pw, seed):
    """Random Fourier tables, N_G = 5 .. 45, uneven slice thicknesses."""
    rng = np.random.default_rng(100 + seed)
    a = 4.0
    b = 2 * math.pi / a
    half = (6, 6)
    nsl = 9
    tabs = random_tables(rng, nsl, half, 0.3)
    lt = random_tables(rng, 2, half, 0.2)
    z = np.concatenate([[0.0], np.cumsum(rng.uniform(0.1, 0.5, nsl))])
    E = rng.uniform(0.5, 6.0, 5)
    kp = rng.uniform(-0.5, 0.5, (5, 2))
    for shells in (1.0, 5.0, 10.0):
        inst = explicit_tables([a, 0], [0, a], shells * b * b * (1 + 1e-9), z, tabs, lt[0], lt[1],
                               half, E, kp)
        ref = O.transmission(inst)
        got, _, _ = _gpu_T(pw, inst, 0)
        assert np.all(_rel(got, ref) < TOL_FP64), (shells, got, ref)


def test_transmission_small_junction_fp64(pw):
    inst = junction(ng=64, n_slices=40, n_e=3, n_k=4)
    sel = [1, 4, 7, 10]
    ref = O.transmission(inst, points=sel)
    got, _, _ = _gpu_T(pw, inst, 0, E=inst.energies[sel], k=inst.kpar[sel])
    assert np.all(_rel(got, ref) < TOL_FP64), (got, ref)


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_MIXED)])
def test_transmission_sweep_beside_eigensolver_partial_wave(pw, precision, tol):
    """332 slice Hamiltonians of one k_par (N_G = 48, 330 slices) are more
    than the eigensolver holds at once, so pw_transmission leaves the partial
    wave (the last device slices) running beside the first interfaces of the
    sweep, the right electrode in the full wave (its last CTA); T against the
    oracle, and the slice modes afterwards (the wave joined) against LAPACK."""
    assert 0 < pw.eig_wave(48) < 332
    inst = junction(ng=48, n_slices=330, n_e=5, n_k=1)
    sel = [0, 2, 4]
    E, k = inst.energies[sel], inst.kpar[sel]
    ref = O.transmission(inst, points=sel)
    with pw.Context.from_instance(inst, precision=precision) as ctx:
        T = _dev(len(E), torch.float64)
        ctx.transmission(E, k, T)
        En = _dev((332, 48), torch.float64)
        ctx.slice_modes(k[0], En)
        torch.cuda.synchronize()
        got, En = T.cpu().numpy(), En.cpu().numpy()
    assert np.all(_rel(got, ref) < tol), (got, ref)
    m = O.Model(inst)
    for q in (0, 300, 331):
        H = O.hamiltonian(m.mn, m.G, k[0], m.all_tables()[q], m.half)
        assert np.abs(En[q] - np.linalg.eigvalsh(H)).max() < 1e-11


def test_threshold_point_reports_and_continues(pw):
    inst = minimal_cell(energies=(2.0,), kpar=((0.0, 0.0),))
    b = 2 * math.pi / 5.0
    E = np.array([b * b, 2.0])           # first energy sits on the |G| = b channel threshold
    k = np.zeros((2, 2))
    with pw.Context.from_instance(inst) as ctx:
        T = _dev(2, torch.float64)
        st = ctx.transmission(E, k, T, allow_threshold=True)
        torch.cuda.synchronize()
        got = T.cpu().numpy()
    assert st == 5
    assert np.isnan(got[0]) and np.isfinite(got[1])


def test_empty_call(pw):
    inst = minimal_cell()
    with pw.Context.from_instance(inst) as ctx:
        T = _dev(1, torch.float64)
        ctx.transmission(np.zeros(0), np.zeros((0, 2)), T)


# ---------------------------------------------------------------------------
# mixed form: FP32 sweep, then FP64 iterative refinement of the whole system
# ---------------------------------------------------------------------------
def test_transmission_mixed_fp32_unrefined(pw):
    """The plain FP32 sweep (no refinement) is accurate to FP32 level only."""
    E = np.array([0.5, 2.3, 3.9, 5.5])
    k = np.array([[0.0, 0.0], [0.1, -0.2], [0.1, -0.2], [0.0, 0.0]])
    inst = minimal_cell(energies=E, kpar=k)
    ref = O.transmission(inst)
    got, _, _ = _gpu_T(pw, inst, 1, refine_iters=-1)
    assert np.all(_rel(got, ref) < 1e-4), (got, ref)


def test_transmission_mixed_refined_minimal_cell(pw):
    E = np.array([0.5, 2.3, 3.9, 5.5, 2.3])
    k = np.array([[0.0, 0.0], [0.1, -0.2], [0.1, -0.2], [0.0, 0.0], [-0.3, 0.25]])
    inst = minimal_cell(energies=E, kpar=k)
    ref, ref_t = O.transmission(inst, return_t=True)
    got, t, _, err = _gpu_T(pw, inst, 1, with_t=True, with_err=True)
    assert np.all(_rel(got, ref) < TOL_MIXED), (got, ref)
    assert np.all((err >= 0) & (err < 1e-6)), err
    for i in range(len(E)):
        nR, nL = ref_t[i].shape
        assert np.abs(t[i].T[:nR, :nL] - ref_t[i]).max() < 1e-8


@pytest.mark.parametrize("iters", [1, 2])
def test_transmission_mixed_refined_junction(pw, iters):
    inst = junction(ng=97, n_slices=60, n_e=4, n_k=4)
    sel = [1, 2, 5, 6, 9, 10]
    ref = O.transmission(inst, points=sel)
    got, _, _ = _gpu_T(pw, inst, 1, E=inst.energies[sel], k=inst.kpar[sel], refine_iters=iters)
    assert np.all(_rel(got, ref) < TOL_MIXED), (iters, got, ref)


def test_transmission_mixed_refined_one_kpar(pw):
    """Points that all share one k_par share their overlaps: [W|Y] then runs
    for point pairs against one B tile and the refinement's backward product
    is one tensor-core product for every point.  Four junction points, and an
    odd count (the last point of the launch unpaired) on the minimal cell."""
    inst = junction(ng=97, n_slices=60, n_e=4, n_k=4)
    sel = [0, 1, 2, 3]   # the four energies of the first k_par
    assert np.all(inst.kpar[sel] == inst.kpar[sel[0]])
    ref = O.transmission(inst, points=sel)
    got, _, _ = _gpu_T(pw, inst, 1, E=inst.energies[sel], k=inst.kpar[sel])
    assert np.all(_rel(got, ref) < TOL_MIXED), (got, ref)
    E = np.array([0.5, 1.7, 2.3, 3.9, 5.5])
    k = np.tile([[0.1, -0.2]], (5, 1))
    inst = minimal_cell(energies=E, kpar=k)
    ref = O.transmission(inst)
    got, _, _ = _gpu_T(pw, inst, 1)
    assert np.all(_rel(got, ref) < TOL_MIXED), (got, ref)


@pytest.mark.parametrize("ng,nsl", [(128, 40), (512, 6)])
@pytest.mark.parametrize("variant", [2, 18, 26])
def test_transmission_mixed_sliced_residual(pw, ng, nsl, variant):
    """Points of one k_par with a basis that is a multiple of 4 and at most 512:
    with variant bit 4 the refinement's residual products O y run as exact
    BF16 slice products on the tensor cores (bit 3 adds the 128-row LU
    blocks), without it on the CUDA cores in double-float.  N_G = 128 spans
    two row tiles and a ragged column tile; N_G = 512 puts 1024 terms in each
    exact sum."""
    inst = junction(ng=ng, n_slices=nsl, n_e=4, n_k=1)
    ref = O.transmission(inst)
    T = _dev(len(inst.energies), torch.float64)
    with pw.Context.from_instance(inst, precision=1) as ctx:
        ctx.set_sweep_variant(variant)
        ctx.transmission(inst.energies, inst.kpar, T)
        torch.cuda.synchronize()
    got = T.cpu().numpy()
    assert np.all(_rel(got, ref) < TOL_MIXED), (got, ref)


def test_transmission_largest_basis_mixed(pw):
    """N_G = 1024, the largest basis pw_setup accepts (the panel LU then takes
    its global-memory path, the eigensolver its largest shared-memory carves),
    mixed form: two slices, two energies at one k_par."""
    inst = junction(ng=1024, n_slices=2, n_e=2, n_k=1)
    ref = O.transmission(inst)
    got, _, _ = _gpu_T(pw, inst, 1)
    assert np.all(_rel(got, ref) < TOL_MIXED), (got, ref)


def test_transmission_mixed_refined_random_tables(pw):
    rng = np.random.default_rng(7)
    a = 4.0
    b = 2 * math.pi / a
    half = (6, 6)
    nsl = 11
    tabs = random_tables(rng, nsl, half, 0.3)
    lt = random_tables(rng, 2, half, 0.2)
    z = np.concatenate([[0.0], np.cumsum(rng.uniform(0.1, 0.5, nsl))])
    E = rng.uniform(0.5, 6.0, 5)
    kp = rng.uniform(-0.5, 0.5, (5, 2))
    inst = explicit_tables([a, 0], [0, a], 10.0 * b * b * (1 + 1e-9), z, tabs, lt[0], lt[1],
                           half, E, kp)
    ref = O.transmission(inst)
    got, _, _ = _gpu_T(pw, inst, 1)
    assert np.all(_rel(got, ref) < TOL_MIXED), (got, ref)
