"""Periodic electrodes on the GPU (pw_set_periodic_electrode,
pw_transmission_periodic; App. B Eq. cmp, App. C) against the oracle's
complex bands (oracle/complex_bands.py), and the device Schur kernels they
use against LAPACK (numpy): random cells of different periods on both sides
of a random device, a screw-tilted perfect crystal (reflectionless with the
tilt phases), and z-uniform cells that must reproduce the z-invariant
electrodes of the star-product path."""
import math

import numpy as np
import pytest

from oracle import complex_bands as CB
from oracle import pw_oracle as O
from synthetic import explicit_tables, random_tables
from tests.parity import TOL_FP64, rel_T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

A = 4.0
B = 2 * math.pi / A
HALF = (2, 2)


@pytest.fixture(scope="module")
def pw():
    import __graft_entry__ as g
    g.build()
    import paper_1504_01462_gb300 as pw
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pw


@pytest.mark.parametrize("N,seed", [(40, 1), (96, 2)])
def test_device_schur_form_against_lapack(pw, N, seed):
    rng = np.random.default_rng(seed)
    Am = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    T, Z, _ = pw.selftest_schur(Am)
    nrm = np.abs(Am).max()
    assert np.abs(np.tril(T, -1)).max() < 1e-13 * nrm
    assert np.abs(Z.conj().T @ Z - np.eye(N)).max() < 1e-12
    assert np.abs(Am @ Z - Z @ T).max() < 1e-11 * nrm
    ev = np.sort_complex(np.diag(T))
    ref = np.sort_complex(np.linalg.eigvals(Am))
    assert np.abs(ev - ref).max() < 1e-10 * nrm
    T, Z, cnt = pw.selftest_schur(Am, select=True)
    assert cnt == int(np.sum(ref.real < 0))
    d = np.diag(T)
    assert np.all(d[:cnt].real < 0) and np.all(d[cnt:].real >= 0)
    Z1 = Z[:, :cnt]
    assert np.abs(Am @ Z1 - Z1 @ T[:cnt, :cnt]).max() < 1e-11 * nrm


def _instance(dev_tabs, dd, E, k):
    z = np.concatenate([[0.0], np.cumsum(dd)])
    return explicit_tables([A, 0.0], [0.0, A], 2.0 * B * B * (1 + 1e-9), z, dev_tabs, None, None, HALF, E, k)


def _random_setup(seed):
    rng = np.random.default_rng(seed)
    cellL = (random_tables(rng, 3, HALF, 0.5), [0.3, 0.5, 0.4])
    cellR = (random_tables(rng, 2, HALF, 0.5), [0.6, 0.35])
    dev = random_tables(rng, 5, HALF, 0.5)
    dd = rng.uniform(0.2, 0.6, 5)
    return cellL, cellR, dev, dd


def _gpu_T(pw, inst, cellL, cellR, a3L=(0.0, 0.0), a3R=(0.0, 0.0)):
    with pw.Context.from_instance(inst) as ctx:
        ctx.set_periodic_electrode(0, cellL[0], cellL[1], a3L)
        ctx.set_periodic_electrode(1, cellR[0], cellR[1], a3R)
        T = torch.zeros(len(inst.energies), dtype=torch.float64, device="cuda")
        ctx.transmission_periodic(inst.energies, inst.kpar, T)
        torch.cuda.synchronize()
        return T.cpu().numpy()


@pytest.mark.parametrize("seed", [4, 5])
def test_random_periodic_electrodes_against_oracle(pw, seed):
    cellL, cellR, dev, dd = _random_setup(seed)
    E = np.array([3.7, 2.6, 4.3])
    k = np.array([[0.13, -0.21], [0.0, 0.3], [0.2, 0.1]])
    inst = _instance(dev, dd, E, k)
    got = _gpu_T(pw, inst, cellL, cellR)
    mn, G = O.gvectors([A, 0.0], [0.0, A], 2.0 * B * B * (1 + 1e-9))
    for i in range(len(E)):
        _, _, T, _ = CB.transmission_periodic(mn, G, HALF, k[i], float(E[i]), dev, dd, cellL, cellR)
        assert rel_T(got[i], T) < TOL_FP64, (i, got[i], T)


def _translate(table, s):
    """The table of the potential moved by s (input construction)."""
    dm, dn = (table.shape[0] - 1) // 2, (table.shape[1] - 1) // 2
    im = np.arange(-dm, dm + 1)[:, None]
    inn = np.arange(-dn, dn + 1)[None, :]
    return table * np.exp(-1j * (im * B * s[0] + inn * B * s[1]))


def test_tilted_perfect_crystal_is_reflectionless(pw):
    """A screw-periodic electrode (each slice the previous one moved by s, so
    the cell repeats along a3 = (3 s, d)) on both sides of two more of its
    periods: with the tilt phases every right-going propagating state passes
    (T = their number), as in the oracle."""
    rng = np.random.default_rng(9)
    base = random_tables(rng, 1, HALF, 0.6)[0]
    s = np.array([0.37, 0.21])
    M, d = 3, [0.4, 0.3, 0.5]

    def cell(kappa):
        return [_translate(base, (kappa * M + j) * s) for j in range(M)]
    a3p = M * s
    E, k = np.array([3.3]), np.array([[0.11, 0.07]])
    inst = _instance(cell(1) + cell(2), d + d, E, k)
    got = _gpu_T(pw, inst, (cell(0), d), (cell(3), d), a3p, a3p)
    mn, G = O.gvectors([A, 0.0], [0.0, A], 2.0 * B * B * (1 + 1e-9))
    D = CB.tilt_phases(G, a3p)
    _, _, T, info = CB.transmission_periodic(mn, G, HALF, k[0], 3.3, cell(1) + cell(2), d + d, (cell(0), d),
                                             (cell(3), d), D, D)
    nprop = int(info["left"]["propR"].sum())
    assert abs(got[0] - nprop) < 1e-10 and rel_T(got[0], T) < TOL_FP64


def test_uniform_cells_reproduce_z_invariant_electrodes(pw):
    """Cells cut from the context's own z-invariant electrodes (their tables
    as the device computes them) into one or several slices: T equals the
    star-product path's T with z-invariant electrodes."""
    rng = np.random.default_rng(3)
    dev = random_tables(rng, 4, HALF, 0.5)
    dd = rng.uniform(0.2, 0.6, 4)
    lt = random_tables(rng, 2, HALF, 0.3)
    z = np.concatenate([[0.0], np.cumsum(dd)])
    E = np.array([2.9, 4.1])
    k = np.array([[0.1, -0.2], [0.0, 0.25]])
    inst = explicit_tables([A, 0.0], [0.0, A], 2.0 * B * B * (1 + 1e-9), z, dev, lt[0], lt[1], HALF, E, k)
    with pw.Context.from_instance(inst) as ctx:
        half = ctx.table_half()
        tabs = torch.zeros((len(dd) + 2, 2 * half[0] + 1, 2 * half[1] + 1), dtype=torch.complex128, device="cuda")
        ctx.potential_tables(tabs)
        T0 = torch.zeros(len(E), dtype=torch.float64, device="cuda")
        ctx.transmission(E, k, T0)
        torch.cuda.synchronize()
        tabs = tabs.cpu().numpy()
        T0 = T0.cpu().numpy()
    vl, vr = tabs[0], tabs[-1]
    for cl, cr in ((([vl], [0.7]), ([vr], [1.3])), (([vl] * 2, [0.35, 0.35]), ([vr] * 3, [0.2, 0.5, 0.4]))):
        got = _gpu_T(pw, inst, cl, cr)
        assert np.all(rel_T(got, T0) < TOL_FP64), (got, T0)
