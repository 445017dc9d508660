"""Parity of the GPU layer doubling (App. A Eq. recurrence2 with the switch to
Eq. recurrence) with the oracle: the interface elements and one mixed step
element by element (the oracle fed the GPU's eigenmodes, so that the
eigenvector phases match), and T and the number of mixed levels of the whole
doubling against the oracle's doubling on the same modes and against the
oracle's left-to-right sweep."""
import numpy as np
import pytest

from oracle import pw_oracle as O
from synthetic import junction, minimal_cell
from tests.parity import TOL_FP64, rel_T

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


def _gpu_modes(ctx, k, n, nq):
    En = _dev(nq * n, torch.float64)
    U = _dev((nq, n, n), torch.complex128)
    ctx.slice_modes(k, En, U)
    torch.cuda.synchronize()
    En = En.cpu().numpy().reshape(nq, n)
    U = np.transpose(U.cpu().numpy(), (0, 2, 1))
    return [(En[q], U[q]) for q in range(nq)]


def _blocks(t):
    return np.transpose(t.cpu().numpy(), (0, 1, 3, 2))


def _close(x, ref, tol):
    return np.abs(x - ref).max() <= tol * max(1.0, np.abs(ref).max())


def test_interface_elements_match_eq_transfer_and_scatter(pw):
    """I11 = P E-, I12 = Q E+ of Eq. transfer and S21, S22 of Eq. scatter, at
    the first, an inner and the right-electrode interface (dz = 0 there)."""
    inst = junction(ng=48, n_slices=20, n_e=1, n_k=1)
    m = O.Model(inst)
    k = np.asarray(inst.kpar[0])
    E = np.array([float(inst.energies[0]), 0.31])
    with pw.Context.from_instance(inst) as ctx:
        md = _gpu_modes(ctx, k, m.n, m.N + 2)
        for iface in (0, 7, m.N):
            T = _dev((len(E), 4, m.n, m.n), torch.complex128)
            ctx.slice_mixed(E, np.repeat(k[None], len(E), 0), iface, T)
            torch.cuda.synchronize()
            T = _blocks(T)
            for i, e in enumerate(E):
                ref = m.interface_mixed(md, float(e), iface)
                for b in range(4):
                    assert _close(T[i, b], ref[b], 1e-11), (iface, e, b)


def test_mixed_step_matches_eq_recurrence2(pw):
    inst = minimal_cell(n_slices=16)
    m = O.Model(inst)
    k = np.array([0.05, 0.3])
    E = np.array([1.1, 2.9])
    n = m.n
    with pw.Context.from_instance(inst) as ctx:
        kk = np.repeat(k[None], len(E), 0)
        Ta = _dev((len(E), 4, n, n), torch.complex128)
        Tb = _dev((len(E), 4, n, n), torch.complex128)
        Tab = _dev((len(E), 4, n, n), torch.complex128)
        ctx.slice_mixed(E, kk, 3, Ta)
        ctx.slice_mixed(E, kk, 4, Tb)
        ctx.compose_mixed(len(E), Ta, Tb, Tab)
        torch.cuda.synchronize()
        A, B, C = _blocks(Ta), _blocks(Tb), _blocks(Tab)
    for i in range(len(E)):
        ref = O.star_mixed(tuple(A[i]), tuple(B[i]))
        for b in range(4):
            assert _close(C[i, b], ref[b], 1e-11), (i, b)


@pytest.mark.parametrize("which", ["minimal", "junction"])
def test_doubling_transmission_and_levels(pw, which):
    """T of the whole doubling against the oracle's doubling on the GPU's modes
    (same switching decisions: the mixed level counts agree) and against the
    oracle's left-to-right sweep; the minimal cell doubles 17 interfaces (odd
    blocks on the way), the junction 41 with the switch part way."""
    if which == "minimal":
        inst = minimal_cell(energies=(0.8, 2.3, 4.1), kpar=((0.1, -0.2), (0.1, -0.2), (0.0, 0.0)))
    else:
        inst = junction(ng=48, n_slices=40, n_e=2, n_k=1)
    m = O.Model(inst)
    E, k = inst.energies, inst.kpar
    ref = O.transmission(inst)
    with pw.Context.from_instance(inst) as ctx:
        T = _dev(len(E), torch.float64)
        levels = ctx.transmission_doubling(E, k, T)
        torch.cuda.synchronize()
        T = T.cpu().numpy()
        for i in range(len(E)):
            md = _gpu_modes(ctx, np.asarray(k[i]), m.n, m.N + 2)
            S, lv = m.total_s_doubling(md, float(E[i]))
            _, Td = O.transmission_from_s(S, float(E[i]), md[0][0], md[-1][0])
            assert levels[i] == lv, (i, levels[i], lv)
            assert rel_T(T[i], Td) < TOL_FP64
            assert rel_T(T[i], ref[i]) < TOL_FP64


def test_doubling_criterion_and_fp64_sweep(pw):
    """A criterion below every interface's I11 norm switches before any mixed
    level (level 0, Eq. recurrence throughout); the result equals the FP64
    sweep of pw_transmission on the same points."""
    inst = junction(ng=48, n_slices=40, n_e=2, n_k=1)
    E, k = inst.energies, inst.kpar
    with pw.Context.from_instance(inst) as ctx:
        T0 = _dev(len(E), torch.float64)
        lv0 = ctx.transmission_doubling(E, k, T0, cond_max=0.5)
        Ts = _dev(len(E), torch.float64)
        ctx.transmission(E, k, Ts)
        torch.cuda.synchronize()
        T0, Ts = T0.cpu().numpy(), Ts.cpu().numpy()
    assert np.all(lv0 == 0)
    assert np.all(rel_T(T0, Ts) < TOL_FP64)


def test_doubling_threshold_and_invalid_criterion(pw):
    """A point on an electrode channel threshold gets T = NaN and level -1
    while the next point is computed; a non-positive criterion is rejected."""
    import math
    inst = minimal_cell(energies=(2.0,), kpar=((0.0, 0.0),))
    b = 2 * math.pi / 5.0
    E = np.array([b * b, 2.0])   # the first energy sits on the |G| = b threshold
    with pw.Context.from_instance(inst) as ctx:
        T = _dev(2, torch.float64)
        lv = ctx.transmission_doubling(E, np.zeros((2, 2)), T, allow_threshold=True)
        torch.cuda.synchronize()
        got = T.cpu().numpy()
        assert lv[0] == -1 and np.isnan(got[0])
        assert lv[1] >= 0 and np.isfinite(got[1])
        with pytest.raises(pw.PwError):
            ctx.transmission_doubling(np.array([2.3]), np.zeros((1, 2)), T, cond_max=0.0)
