"""Convergence pin of the slice model against the continuous-z problem: the
slice model's T (exact slice averages of the wells, Eqs. loc, transfer,
scatter, recurrence) extrapolated in the slice thickness, and an independent
three-point finite-difference solve of the continuous problem (its own
potential evaluation, exact discrete transparent electrodes) extrapolated in
the grid step, agree.  Both errors are second order, so Richardson over
three halvings leaves about 1e-9."""
import math

import numpy as np
import pytest

from oracle import continuum as CT
from oracle import pw_oracle as O
from synthetic.junction import Instance, Lead

A = 4.0
B = 2 * math.pi / A
WELLS = np.array([[1.1, 2.3, 1.6], [2.9, 0.7, 2.2], [0.4, 3.1, 2.5]])
V0 = np.array([1.5, 2.2, 1.2])
SIG = np.full(3, 0.3)
L = 4.0


def _inst(N, E, k):
    return Instance(a1=np.array([A, 0.0]), a2=np.array([0.0, A]), ecut=2.0 * B * B * (1 + 1e-9), ng_exact=0,
                    z_edges=np.linspace(0.0, L, N + 1), wells_xyz=WELLS, v0=V0, sigma=SIG,
                    lead_left=Lead.free(), lead_right=Lead.free(), energies=np.array([E]),
                    kpar=np.asarray(k, float)[None, :])


@pytest.mark.parametrize("E,k", [(2.1, (0.13, -0.07)), (3.4, (0.3, 0.2))])
def test_slice_model_converges_to_the_continuum(E, k):
    slices = [O.transmission(_inst(N, E, k))[0] for N in (32, 64, 128)]
    m = O.Model(_inst(8, E, k))
    area = O.cell_area(m.inst.a1, m.inst.a2)
    fd = [CT.transmission_fd(m.G, np.asarray(k), E, area, WELLS, V0, SIG, L, h) for h in (0.02, 0.01, 0.005)]
    Ts, Tf = CT.richardson(slices), CT.richardson(fd)
    assert abs(Ts - Tf) < 1e-7 * max(1.0, Tf), (Ts, Tf)
    # and the unextrapolated models are visibly apart (the pin is not vacuous)
    assert abs(slices[0] - Tf) > 1e-6
