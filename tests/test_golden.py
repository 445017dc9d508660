"""The oracle and the CUDA path against stored 40-digit results.

tests/golden/brute_tiny.json holds T and t of five seeded tiny slice models
(4 bohr square cell, 5 plane waves, 3-6 random slices, V = 0 electrodes),
written by tests/golden/make_brute_golden.py with oracle/brute.py: an exact
matrix-exponential integration of each slice's ODE (Sec. II A, Eq. loc with
the z-dependence kept), which shares none of the method's machinery (no
eigenmodes, no transfer or scattering matrices).  The brute-force t lists
open channels in G-list order; the oracle and the library order them by
ascending |k+G|^2, the electrodes' E_n."""
import json
import os

import numpy as np
import pytest

from oracle import pw_oracle as O
from tests.golden.cases import tiny_instance
from tests.parity import rel_T

with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "brute_tiny.json")) as _f:
    GOLDEN = json.load(_f)["cases"]


def _brute_t_by_energy(c, kg2):
    """The stored t with its open channels reordered by ascending |k+G|^2."""
    tb = np.array(c["t_re"]) + 1j * np.array(c["t_im"])
    opn = [i for i in range(len(kg2)) if kg2[i] < c["E"]]
    order = [i for i in np.argsort(kg2, kind="stable") if kg2[i] < c["E"]]
    perm = [opn.index(i) for i in order]
    return tb[np.ix_(perm, perm)]


def _case(c):
    inst, _ = tiny_instance(c["seed"], c["E"], tuple(c["kpar"]), c["slices"])
    m = O.Model(inst)
    kg2 = ((m.G + np.array(c["kpar"])) ** 2).sum(1)
    return inst, kg2


@pytest.mark.parametrize("c", GOLDEN, ids=[str(c["seed"]) for c in GOLDEN])
def test_oracle_matches_stored_brute_force(c):
    inst, kg2 = _case(c)
    T, ts = O.transmission(inst, return_t=True)
    assert rel_T(T[0], c["T"]) < 1e-12
    assert np.abs(ts[0] - _brute_t_by_energy(c, kg2)).max() < 1e-12


@pytest.fixture(scope="module")
def pw():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    import paper_1504_01462_gb300 as pw
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pw


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-8)])
def test_cuda_path_matches_stored_brute_force(pw, precision, tol):
    import torch
    for c in GOLDEN:
        inst, kg2 = _case(c)
        with pw.Context.from_instance(inst, precision=precision) as ctx:
            n = ctx.ng
            T = torch.empty(1, dtype=torch.float64, device="cuda")
            t = torch.empty((1, n, n), dtype=torch.complex128, device="cuda")
            nop = torch.empty((1, 2), dtype=torch.int32, device="cuda")
            ctx.transmission(inst.energies, inst.kpar, T, t, nop)
            torch.cuda.synchronize()
            T, t, nop = T.cpu().numpy(), t.cpu().numpy(), nop.cpu().numpy()
        assert rel_T(T[0], c["T"]) < tol, (c["seed"], T[0], c["T"])
        nL, nR = int(nop[0, 0]), int(nop[0, 1])
        tb = _brute_t_by_energy(c, kg2)
        assert tb.shape == (nR, nL)
        # device slots are column-major n x n: element (i, j) at t[.., j, i]
        assert np.abs(t[0].T[:nR, :nL] - tb).max() < 10 * tol, c["seed"]
