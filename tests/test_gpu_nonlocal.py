"""Separable nonlocal projector terms on the GPU (pw_set_projectors,
pw_transmission_nonlocal) against the oracle's one-system solve
(oracle/separable.py, Eqs. nloc, gsol_p0, calm_0): T and the projector
coefficients C on cells with random slice potentials and V = 0 electrodes
(there t and C are unique), T on the junction, the local path when D = 0,
and flux conservation for Hermitian D."""
import math

import numpy as np
import pytest

from oracle import pw_oracle as O
from oracle import separable as NL
from synthetic import explicit_tables, junction, random_tables
from tests.parity import TOL_FP64, rel_T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

A4 = 4.0
B4 = 2 * math.pi / A4


@pytest.fixture(scope="module")
def pw():
    import __graft_entry__ as g
    g.build()
    import paper_1504_01462_gb300 as pw
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pw


def _cell(seed, nsl=5, shells=2.0):
    rng = np.random.default_rng(seed)
    dz = rng.uniform(0.3, 0.6, nsl)
    z = np.concatenate([[0.0], np.cumsum(dz)])
    tabs = random_tables(rng, nsl, (2, 2), 0.4)
    return explicit_tables([A4, 0.0], [0.0, A4], shells * B4 * B4 * (1 + 1e-9), z, tabs, None, None, (2, 2),
                           [3.3], [(0.07, 0.19)])


def _oracle(inst, E, k, params, D, q=16):
    m = O.Model(inst)
    area = O.cell_area(inst.a1, inst.a2)
    projs = [NL.gaussian_projector(m.G, k, area, p[:3], p[3], p[4], p[5]) for p in params]
    t, r, T, aN1, C = NL.transmission_nonlocal(m.modes(np.asarray(k)), m.dz, E, projs, D, area, q=q)
    return T, C, t


def _gpu(pw, inst, E, k, params, D, q=16, prec=0):
    with pw.Context.from_instance(inst, precision=prec) as ctx:
        ctx.set_projectors(params, D, q)
        n = ctx.ng
        T = torch.zeros(len(E), dtype=torch.float64, device="cuda")
        C = torch.zeros((len(E), len(params), n), dtype=torch.complex128, device="cuda")
        ctx.transmission_nonlocal(E, k, T, C)
        torch.cuda.synchronize()
        return T.cpu().numpy(), C.cpu().numpy()


@pytest.mark.parametrize("seed,D", [(3, np.diag([0.8, -1.3])),
                                    (4, np.array([[0.8, 0.3 + 0.2j], [0.3 - 0.2j, -1.3]])),
                                    (5, np.array([[2.0, -0.4j], [0.7, 0.5]]))])
def test_nonlocal_cell_against_oracle(pw, seed, D):
    inst = _cell(seed)
    zN = float(inst.z_edges[-1])
    params = np.array([[1.1, 2.3, 0.45 * zN, 0.45, 0.0, zN], [3.0, 0.6, 0.6 * zN, 0.5, 0.0, zN]])
    E = np.array([3.3, 2.1, 4.4])
    k = np.array([[0.07, 0.19], [0.07, 0.19], [-0.2, 0.1]])
    T, C = _gpu(pw, inst, E, k, params, D)
    for i in range(len(E)):
        Tr, Cr, _ = _oracle(inst, float(E[i]), k[i], params, D)
        assert rel_T(T[i], Tr) < TOL_FP64, (i, T[i], Tr)
        nL = int(np.sum(np.sum((np.asarray(k[i]) + O.gvectors(inst.a1, inst.a2, inst.ecut, 0)[1]) ** 2, 1)
                        < E[i]))
        assert np.abs(C[i][:, :nL] - Cr[:, :nL]).max() < 1e-10 * max(1.0, np.abs(Cr).max())


def test_nonlocal_with_zero_coupling_is_the_local_path(pw):
    inst = _cell(7)
    zN = float(inst.z_edges[-1])
    params = np.array([[1.1, 2.3, 0.5 * zN, 0.4, 0.0, zN]])
    E = np.array([3.3, 1.7])
    k = np.array([[0.07, 0.19], [0.0, 0.0]])
    T, C = _gpu(pw, inst, E, k, params, np.zeros((1, 1)))
    with pw.Context.from_instance(inst) as ctx:
        T0 = torch.zeros(len(E), dtype=torch.float64, device="cuda")
        ctx.transmission(E, k, T0)
        torch.cuda.synchronize()
    assert np.all(rel_T(T, T0.cpu().numpy()) < 1e-12)
    assert np.abs(C).max() == 0.0


def test_nonlocal_hermitian_coupling_conserves_flux_and_junction(pw):
    """T <= open channels for Hermitian D on the junction (N_G = 48, 16
    slices, projectors on two wells of the overlap region) against the oracle,
    in both precisions of the context (the nonlocal solve is FP64 in both)."""
    inst = junction(ng=48, n_slices=16, n_e=3, n_k=2)
    zN = float(inst.z_edges[-1])
    w = inst.wells_xyz
    params = np.array([[w[10, 0], w[10, 1], w[10, 2], 0.6, 0.0, zN],
                       [w[30, 0], w[30, 1], w[30, 2], 0.6, 0.0, zN]])
    D = np.array([[-1.5, 0.2 + 0.1j], [0.2 - 0.1j, -0.8]])
    sel = [1, 4]
    E, k = inst.energies[sel], inst.kpar[sel]
    for prec in (0, 1):
        T, _ = _gpu(pw, inst, E, k, params, D, prec=prec)
        for i in range(len(sel)):
            Tr, _, _ = _oracle(inst, float(E[i]), k[i], params, D)
            assert rel_T(T[i], Tr) < TOL_FP64, (prec, i, T[i], Tr)
