"""The tcgen05 tensor-core path: one TF32 tile product and the three-product
split against an FP64 product of the same inputs."""
import pytest

from tests.parity import rel_T

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


def test_tcgen05_tile_product(pw):
    e1, e3 = pw.selftest_tensor_core()
    # TF32 keeps 10 explicit mantissa bits (2^-11 relative rounding per input)
    assert 1e-6 < e1 < 5e-3, e1
    # hi/lo split: FP32-level products, FP32 accumulation over K = 32
    assert e3 < 2e-6, e3
    assert e3 < e1 / 50


@pytest.mark.parametrize("n,ncol", [(512, 256), (100, 200), (4, 3)])
def test_exact_slice_product(pw, n, ncol):
    """The residual's slice product: 7-bit slices in BF16 on tcgen05 with FP32
    accumulation are exact for 2n <= 1024 inner terms (sums up to 2^24 units at
    n = 512); every slice pair summed in double-float is accurate to about
    2^-48.  n = 100 and ncol = 200 leave ragged row, column and K tiles."""
    bad, rel = pw.selftest_slice_product(n, ncol)
    assert bad == 0, bad
    assert rel < 1e-13, rel


def test_fp16_split_tile_product(pw):
    """The FP16 split's layout, descriptors and headroom on one tile: FP32-level
    accuracy like the TF32 split."""
    e = pw.selftest_f16_split()
    assert e < 2e-6, e


def _T(pw, inst, E, k, variant, refine_iters):
    T = torch.zeros(len(E), dtype=torch.float64, device="cuda")
    with pw.Context.from_instance(inst, pw.MIXED_FP32, refine_iters) as ctx:
        ctx.set_sweep_variant(variant)
        ctx.transmission(E, k, T)
    torch.cuda.synchronize()
    return T.cpu().numpy()


@pytest.mark.parametrize("variant", [2, 3, 10, 11, 26])
def test_sweep_with_tensor_core_products(pw, variant):
    """The sweep with its GEMM phases on tcgen05 (TF32 hi/lo split): the
    unrefined sweep is FP32-accurate, the refined one meets 1e-8; the junction
    size (N_G = 97, 60 slices) spans two M tiles, a ragged N tile and 8
    K stages.  Bit 3: LAPACK-ordered pivots and 128-row triangular blocks
    (one ragged block of 97 rows); bit 4: the residual as slice products
    (these points do not share a k_par, so the CUDA-core residual runs)."""
    import numpy as np
    from oracle import pw_oracle as O
    from synthetic import junction
    inst = junction(ng=97, n_slices=60, n_e=4, n_k=4)
    sel = [1, 2, 5, 6, 9, 10]
    E, k = inst.energies[sel], inst.kpar[sel]
    ref = O.transmission(inst, points=sel)
    scale = np.maximum(1.0, np.abs(ref))
    raw = _T(pw, inst, E, k, variant, -1)
    assert np.all(np.abs(raw - ref) / scale < 1e-4), (raw, ref)
    simt = _T(pw, inst, E, k, variant & 1, -1)
    assert np.all(np.abs(raw - simt) / scale < 1e-4)
    got = _T(pw, inst, E, k, variant, 4)
    assert np.all(rel_T(got, ref) < 1e-8), (got, ref)


@pytest.mark.parametrize("variant", [6, 7, 14, 30])
def test_sweep_with_fp16_split_point_pairs(pw, variant):
    """The paired [W|Y] in the FP16 split (sweep variant bit 2, four points of
    one k_par so that pairs share the overlap): the unrefined sweep agrees
    with the TF32-split sweep and the oracle at FP32 level, the refined one
    meets 1e-8."""
    import numpy as np
    from oracle import pw_oracle as O
    from synthetic import junction
    inst = junction(ng=97, n_slices=60, n_e=4, n_k=1)
    E, k = inst.energies, inst.kpar
    ref = O.transmission(inst)
    scale = np.maximum(1.0, np.abs(ref))
    raw = _T(pw, inst, E, k, variant, -1)
    assert np.all(np.abs(raw - ref) / scale < 1e-4), (raw, ref)
    tf32 = _T(pw, inst, E, k, variant & 3, -1)
    assert np.all(np.abs(raw - tf32) / scale < 1e-4)
    got = _T(pw, inst, E, k, variant, 4)
    assert np.all(rel_T(got, ref) < 1e-8), (got, ref)



def test_bounded_wait_runs_out_and_reports(pw):
    """A tensor-core completion wait on an mbarrier that nothing completes gives
    up after its poll limit (1000 polls of 64 ns) with PW_ETIMEOUT instead of
    hanging; the same wait completes when the barrier is signalled, and the
    device stays usable afterwards (the tile self-test runs again)."""
    lib = pw.lib()
    assert lib.pw_selftest_bounded_wait(1000, 0) == 6     # PW_ETIMEOUT
    assert lib.pw_selftest_bounded_wait(1000, 1) == 0
    assert lib.pw_selftest_bounded_wait(0, 0) == 1        # PW_EINVAL
    e1, e3 = pw.selftest_tensor_core()
    assert e3 < 1e-5


def test_sweep_as_two_point_groups(pw):
    """Sweep variant bit 6: 40 points of one k_par swept as two groups of 20
    on two streams give the T of one group (each point runs the same kernels,
    and the point pairs of the [W|Y] product stay together), and meet 1e-8
    against the oracle."""
    import numpy as np
    from oracle import pw_oracle as O
    from synthetic import junction
    inst = junction(ng=97, n_slices=30, n_e=40, n_k=1)
    E, k = inst.energies, inst.kpar
    one = _T(pw, inst, E, k, 2, 4)
    two = _T(pw, inst, E, k, 2 | 64, 4)
    assert np.all(np.abs(one - two) <= 1e-14 * np.maximum(1.0, np.abs(one))), np.abs(one - two).max()
    sel = [3, 17, 25, 38]
    ref = O.transmission(inst, points=sel)
    assert np.all(rel_T(two[sel], ref) < 1e-8), (two[sel], ref)
