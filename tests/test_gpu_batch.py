"""pw_setup_batch / pw_transmission_batch: independent instances of uneven
basis size and slice count, one (E, k_par) point each, against the oracle and
against the one-problem path."""
import numpy as np
import pytest

from oracle import pw_oracle as O
from synthetic import uneven_batch
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


def _points(insts):
    E = np.array([float(x.energies[0]) for x in insts])
    k = np.array([x.kpar[0] for x in insts])
    return E, k


def _small_batch():
    """Several sizes, slice counts from 3 to 14, and points near the zone
    centre so that most instances have open channels."""
    insts = uneven_batch(14, ng_choices=(16, 24, 32, 48), ns_range=(3, 14), seed_cfg=41)
    for x in insts:
        x.kpar = x.kpar * 0.3
    return insts


@pytest.fixture(scope="module")
def small():
    insts = _small_batch()
    ref = np.array([O.transmission(x)[0] for x in insts])
    return insts, ref


def _run(pw, insts, precision=0, refine_iters=0, use_graph=True, variant=-1):
    E, k = _points(insts)
    T = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    err = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    with pw.Batch.from_instances(insts, precision, refine_iters) as b:
        b.set_options(use_graph, variant)
        b.transmission(E, k, T, err_out=err)
        stats = b.stats()
    torch.cuda.synchronize()
    return T.cpu().numpy(), err.cpu().numpy(), stats


@pytest.mark.parametrize("use_graph,variant", [(True, -1), (False, 0), (True, 1)])
def test_batch_fp64_matches_oracle(pw, small, use_graph, variant):
    insts, ref = small
    T, _, stats = _run(pw, insts, use_graph=use_graph, variant=variant)
    assert np.count_nonzero(ref > 0.5) >= 5
    assert np.all(rel_T(T, ref) <= TOL_FP64), (T, ref)
    assert stats["chunks"] == 4                 # one per basis size
    assert stats["graph_launches"] == (4 if use_graph else 0)
    if variant < 0:
        assert set(stats["variant"]) == {16, 24, 32, 48}


def test_batch_equals_one_problem_path(pw, small):
    """The batch runs the same kernels on the same data in another layout:
    with the same tile variant its T equals the one-problem path's."""
    insts, _ = small
    T, _, _ = _run(pw, insts, use_graph=True, variant=0)
    for x, tb in zip(insts, T):
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pw.Context.from_instance(x) as ctx:
            ctx.transmission(x.energies, x.kpar, out)
        torch.cuda.synchronize()
        assert rel_T(out.item(), tb) <= 1e-13


def test_batch_mixed_refined_matches_oracle(pw, small):
    insts, ref = small
    T, err, _ = _run(pw, insts, precision=1, refine_iters=4)
    assert np.all(rel_T(T, ref) <= TOL_MIXED), (T, ref)
    assert np.all(err < 1e-6)


def test_batch_sampled_uneven_instances(pw):
    """Draws of the 2048-instance uneven workload (N_G 128..768, 60..400
    slices): the smallest ones the oracle finishes in seconds, mixed form
    with refinement, in one batch with a second size."""
    allb = uneven_batch(2048)
    pick = [x for x in allb if x.ng_exact == 128 and x.n_slices <= 90][:2] + \
           [x for x in allb if x.ng_exact == 192 and x.n_slices <= 70][:1]
    assert len(pick) == 3
    ref = np.array([O.transmission(x)[0] for x in pick])
    T, err, stats = _run(pw, pick, precision=1, refine_iters=4)
    assert np.all(rel_T(T, ref) <= TOL_MIXED), (T, ref)
    assert stats["chunks"] == 2


def test_batch_first_96_uneven_instances_against_stored_oracle(pw):
    """The first 96 of the 2048 uneven instances (N_G 128..768, 60..400
    slices) in one batch call, mixed form with refinement: eight of them
    against oracle values stored by tests/golden/make_fullsize_golden.py
    (1e-8 relative on T), every instance finite and within its channel
    bounds."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "uneven96.json")
    with open(path) as f:
        gold = json.load(f)
    insts = uneven_batch(2048)[:96]
    E, k = _points(insts)
    T = torch.zeros(96, dtype=torch.float64, device="cuda")
    nop = torch.zeros((96, 2), dtype=torch.int32, device="cuda")
    err = torch.zeros(96, dtype=torch.float64, device="cuda")
    with pw.Batch.from_instances(insts, 1, 4) as b:
        b.transmission(E, k, T, nop, err, allow_threshold=True)
    torch.cuda.synchronize()
    T, nop, err = T.cpu().numpy(), nop.cpu().numpy(), err.cpu().numpy()
    ok = np.isfinite(T)
    assert ok.sum() >= 94
    assert np.all(T[ok] >= -1e-9) and np.all(T[ok] <= np.minimum(nop[ok, 0], nop[ok, 1]) + 1e-9)
    assert np.all(err[ok] < 1e-8)
    idx = np.array(gold["index"])
    have = np.array([t is not None for t in gold["T"]])
    assert have.sum() >= 4
    ref = np.array([t for t in gold["T"] if t is not None])
    assert np.all(rel_T(T[idx[have]], ref) < TOL_MIXED), (T[idx[have]], ref)
    assert np.array_equal(nop[idx[have]], np.array([x for x in gold["nopen"] if x is not None]))
