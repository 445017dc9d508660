"""Parity at the benchmark's full size: the N_G = 512, 320-slice AB junction,
one k_par x 128 energies in one call (the launch configuration the benchmark
times, mixed form with its default refinement).  Sampled energies are checked
against the oracle computed point by point (mixed to 1e-8, and the FP64 form
on the same points to 1e-10); every point of the call is checked for the
properties that hold at any size: T finite, 0 <= T <= the open channels of
either electrode, the refinement's error estimate below the target."""
import numpy as np
import pytest

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


def test_full_size_step_against_oracle(pw):
    from oracle import pw_oracle as O
    from synthetic import junction
    inst = junction(ng=512, n_slices=320, n_e=128, n_k=32)
    n_e, kk = 128, 5
    idx = np.arange(kk * n_e, (kk + 1) * n_e)
    E, k = inst.energies[idx], inst.kpar[idx]
    with pw.Context.from_instance(inst, precision=pw.MIXED_FP32) as ctx:
        assert (ctx.ng, ctx.n_slices) == (512, 320)
        T = torch.empty(n_e, dtype=torch.float64, device="cuda")
        nop = torch.empty((n_e, 2), dtype=torch.int32, device="cuda")
        err = torch.zeros(n_e, dtype=torch.float64, device="cuda")
        ctx.transmission(E, k, T, None, nop, err)
        torch.cuda.synchronize()
        T, nop, err = T.cpu().numpy(), nop.cpu().numpy(), err.cpu().numpy()
    assert np.all(np.isfinite(T))
    assert np.all(T >= -1e-9)
    assert np.all(T <= np.minimum(nop[:, 0], nop[:, 1]) + 1e-9)
    assert np.all((err >= 0) & (err < 1e-8)), err.max()

    sel = [60, 110]   # two energies of the step (open channels in both electrodes), one by one by the oracle
    ref = O.transmission(inst, points=list(idx[sel]))
    rel = np.abs(T[sel] - ref) / np.maximum(1.0, np.abs(ref))
    assert np.all(rel < 1e-8), (T[sel], ref)
    with pw.Context.from_instance(inst, precision=pw.FP64) as c64:
        T64 = torch.empty(len(sel), dtype=torch.float64, device="cuda")
        c64.transmission(E[sel], k[sel], T64)
        torch.cuda.synchronize()
        T64 = T64.cpu().numpy()
    rel64 = np.abs(T64 - ref) / np.maximum(1.0, np.abs(ref))
    assert np.all(rel64 < 1e-10), (T64, ref)
