"""pw_grad (adjoint of the summed transmission with respect to the device
wells' depths) against the oracle's adjoint and central differences."""
import copy

import numpy as np
import pytest

from oracle import pw_oracle as O
from synthetic import junction, minimal_cell

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


def _oracle_grad(inst, E, k, w):
    m = O.Model(inst)
    dH = O.well_depth_derivatives(m)
    tot, g = 0.0, np.zeros(len(inst.v0))
    for Ei, ki, wi in zip(E, k, w):
        T, gi = O.grad_T(m, np.asarray(ki), float(Ei), dH)
        tot += wi * T
        g += wi * gi
    return tot, g


def test_grad_minimal_cell_against_oracle_adjoint_and_fd(pw):
    E = np.array([2.3, 4.1, 0.7, 2.9])
    k = np.array([[0.1, -0.2], [0.0, 0.3], [0.0, 0.0], [0.1, -0.2]])
    w = np.array([1.0, 0.5, 2.0, 1.5])
    inst = minimal_cell(n_wells=3, n_slices=6, energies=E, kpar=k)
    with pw.Context.from_instance(inst) as ctx:
        sumT, g = ctx.grad(E, k, w, n_wells=len(inst.v0))
    ref_T, ref_g = _oracle_grad(inst, E, k, w)
    assert abs(sumT - ref_T) < 1e-10 * max(1.0, ref_T)
    assert np.abs(g - ref_g).max() < 1e-9 * max(1.0, np.abs(ref_g).max())
    h = 1e-5
    for i in range(len(inst.v0)):
        ip, im = copy.deepcopy(inst), copy.deepcopy(inst)
        ip.v0[i] += h
        im.v0[i] -= h
        fd = (np.dot(w, O.transmission(ip)) - np.dot(w, O.transmission(im))) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd))


def test_grad_small_junction_against_oracle_adjoint(pw):
    inst = junction(ng=48, n_slices=16, n_e=3, n_k=4)
    sel = [1, 5, 6, 9]
    E, k = inst.energies[sel], inst.kpar[sel]
    with pw.Context.from_instance(inst) as ctx:
        sumT, g = ctx.grad(E, k, None, n_wells=len(inst.v0))
    ref_T, ref_g = _oracle_grad(inst, E, k, np.ones(len(sel)))
    assert abs(sumT - ref_T) < 1e-10 * max(1.0, ref_T)
    assert np.abs(g - ref_g).max() < 1e-8 * max(1.0, np.abs(ref_g).max())


def test_grad_rejects_gap_and_tables(pw):
    inst = minimal_cell(n_wells=2, n_slices=3)
    import ctypes
    with pw.Context.from_instance(inst) as ctx:
        E = np.array([2.0])
        k = np.zeros((1, 2))
        s = np.zeros(1)
        gap = np.zeros(1)
        dp = ctypes.POINTER(ctypes.c_double)
        st = pw.lib().pw_grad(ctx.handle, 1, E.ctypes.data_as(dp), k.ctypes.data_as(dp), None,
                              s.ctypes.data_as(dp), None, gap.ctypes.data_as(dp))
        assert st == 1
