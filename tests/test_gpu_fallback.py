"""The mixed form's FP64 fallback (pw_set_fp64_fallback, pw_get_fp64_fallback):
points whose interface blocks W_p have a large LU diagonal spread, or whose
refinement leaves a large estimated error, are solved again by the FP64 sweep
(Sec. II A's pivoted LU of the interface blocks kept in FP64).  Each trigger
is driven by its threshold: every point rerouted must reproduce the FP64
form's T (the same FP64 kernels on the same FP64 modes), and on the junction
with the default thresholds no point is rerouted and the mixed T still meets
its tolerance against the oracle."""
import numpy as np
import pytest

from oracle import pw_oracle as O
from synthetic import junction
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


@pytest.fixture(scope="module")
def case(pw):
    inst = junction(ng=48, n_slices=16, n_e=6, n_k=2)
    E, k = inst.energies, inst.kpar
    with pw.Context.from_instance(inst, precision=pw.FP64) as ctx:
        T64 = torch.zeros(len(E), dtype=torch.float64, device="cuda")
        ctx.transmission(E, k, T64)
        torch.cuda.synchronize()
    return inst, E, k, T64.cpu().numpy()


def _mixed(pw, inst, E, k, fallback=None):
    with pw.Context.from_instance(inst, precision=pw.MIXED_FP32) as ctx:
        if fallback is not None:
            ctx.set_fp64_fallback(*fallback)
        T = torch.zeros(len(E), dtype=torch.float64, device="cuda")
        err = torch.zeros(len(E), dtype=torch.float64, device="cuda")
        ctx.transmission(E, k, T, None, None, err)
        torch.cuda.synchronize()
        return T.cpu().numpy(), err.cpu().numpy(), ctx.fp64_fallback()


def test_default_thresholds_keep_the_junction_in_mixed_precision(pw, case):
    inst, E, k, T64 = case
    T, err, (npts, spread) = _mixed(pw, inst, E, k)
    assert npts == 0
    assert 1.0 <= spread < 1e6
    assert np.all(rel_T(T, T64) < TOL_MIXED)
    Tr = O.transmission(inst, points=[0, 7])
    assert np.all(rel_T(T[[0, 7]], Tr) < TOL_MIXED)
    assert np.all(rel_T(T64[[0, 7]], Tr) < TOL_FP64)


def test_every_point_rerouted_reproduces_the_fp64_form(pw, case):
    inst, E, k, T64 = case
    T, err, (npts, _) = _mixed(pw, inst, E, k, fallback=(0.0, 1e-8))
    assert npts == len(E)
    assert np.all(rel_T(T, T64) < 1e-13)
    assert np.all(err == 0.0)


def test_error_criterion_reroutes(pw, case):
    """err_max = 0 reroutes every point whose refinement made a correction;
    points without an open channel on one side (T = 0) make none."""
    inst, E, k, T64 = case
    T, _, (npts, _) = _mixed(pw, inst, E, k, fallback=(1e6, 0.0))
    assert np.sum(T64 > 0) <= npts <= len(E)
    assert np.all(rel_T(T, T64) < 1e-13)


def test_spread_threshold_reroutes_the_worst_points(pw, case):
    inst, E, k, T64 = case
    _, _, (_, spread) = _mixed(pw, inst, E, k)
    T, _, (npts, spread2) = _mixed(pw, inst, E, k, fallback=(0.999 * spread, 1e-8))
    assert spread2 == spread
    assert 1 <= npts < len(E)
    assert np.all(rel_T(T, T64) < TOL_MIXED)
    T, _, (npts, _) = _mixed(pw, inst, E, k, fallback=(-1.0, 0.0))
    assert npts == 0


def test_fallback_arguments(pw, case):
    inst = case[0]
    with pw.Context.from_instance(inst, precision=pw.MIXED_FP32) as ctx:
        with pytest.raises(pw.PwError):
            ctx.set_fp64_fallback(float("nan"), 1e-8)
        with pytest.raises(pw.PwError):
            ctx.set_fp64_fallback(1e6, -1.0)
