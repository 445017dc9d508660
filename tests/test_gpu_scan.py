"""The conductance sums of Sec. II B on the device (pw_reduce_transmission) and
the second workload's driver (Tbar of Eq. T1_d / T2_d over a k_x mesh for
junctions of given overlap, gap and stacking), against NumPy sums and the
oracle's T point by point."""
import numpy as np
import pytest

from oracle import pw_oracle as O
from synthetic import junction
from tests.parity import TOL_MIXED, rel_T

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


@pytest.mark.parametrize("npts", [0, 1, 7, 1000])
def test_reduce_transmission_matches_numpy(pw, npts):
    rng = np.random.default_rng(npts)
    T = rng.uniform(0, 3, npts)
    if npts > 3:
        T[2] = np.nan                       # a threshold point
    nop = rng.integers(0, 3, (npts, 2)).astype(np.int32)
    w = rng.uniform(0.5, 2, npts)
    Td = torch.tensor(T, device="cuda")
    nd = torch.tensor(nop, device="cuda")
    wd = torch.tensor(w, device="cuda")
    out = pw.reduce_transmission(Td, nd, wd).cpu().numpy()
    ok = ~np.isnan(T)
    ch = ok & (nop[:, 0] > 0)
    assert abs(out[0] - np.sum(w[ok] * T[ok])) <= 1e-13 * max(1.0, np.sum(np.abs(T[ok])))
    assert out[2] == ch.sum()
    assert abs(out[1] - (T[ch].mean() if ch.any() else 0.0)) <= 1e-14 * max(1.0, out[1])
    out = pw.reduce_transmission(Td).cpu().numpy()
    assert abs(out[0] - np.sum(T[ok])) <= 1e-13 * max(1.0, np.sum(np.abs(T[ok])))


@pytest.mark.parametrize("stacking,cells,gap", [("AA", 5, 3.35), ("AB", 7, 4.5)])
def test_scan_tbar_against_oracle(pw, stacking, cells, gap):
    """One junction of the scan (overlap cells - 4, 4 slices per cell, N_G =
    48) at E_ref over an 8-point k_x mesh: T of every point against the
    oracle (mixed form, 1e-8) and Tbar against the mean over the oracle's
    points with an open left-electrode channel."""
    import bench
    inst = junction(ng=48, n_slices=4 * cells, cells=cells, stacking=stacking, gap_angstrom=gap, n_e=1, n_k=1)
    E, nk = 0.2, 8
    stream = torch.cuda.current_stream()
    tbar, nch, T = bench.scan_tbar(pw, torch, inst, E, nk, pw.MIXED_FP32, stream)
    k = bench.kline(nk, inst.a1[0])
    inst.energies = np.full(nk, E)
    inst.kpar = k
    m = O.Model(inst)
    ref = O.transmission(inst, model=m)
    assert np.all(rel_T(T, ref) < TOL_MIXED), (T, ref)
    nL = np.array([len(O.open_channels(E, m.modes(kk)[0][0])) for kk in k])
    assert nch == int((nL > 0).sum())
    want = ref[nL > 0].mean() if (nL > 0).any() else 0.0
    assert abs(tbar - want) <= TOL_MIXED * max(want, 1e-6)
