"""pw_compose_noalloc: the star product for callers that must not let the
library allocate device memory (its only scratch is a fixed array in the
library's device image).  Checked against pw_compose on the same inputs, on
two calls in a row, and its size limit is checked without any device work.
Collected last on purpose (file name) so that a failure here comes after every
other test has run."""
import numpy as np
import pytest

from synthetic import minimal_cell

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


def test_noalloc_compose_matches_compose_twice(pw):
    inst = minimal_cell(n_slices=16)
    E = np.array([1.1, 2.9, 4.2])
    k = np.repeat(np.array([[0.05, 0.3]]), len(E), 0)
    with pw.Context.from_instance(inst) as ctx:
        n = ctx.ng
        Sa = torch.zeros((len(E), 4, n, n), dtype=torch.complex128, device="cuda")
        Sb = torch.zeros_like(Sa)
        ref = torch.zeros_like(Sa)
        ctx.slice_smatrix(E, k, 3, Sa)
        ctx.slice_smatrix(E, k, 4, Sb)
        ctx.compose(len(E), Sa, Sb, ref)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
    scale = max(1.0, np.abs(ref).max())
    for _ in range(2):
        out = torch.full_like(Sa, complex(np.nan, np.nan))
        pw.compose_noalloc(n, len(E), Sa, Sb, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() < 1e-11 * scale


def _pair_vs_compose(pw, ng, n_e):
    """Interface S-matrices of a small junction with N_G = ng at n_e energies,
    their star product by pw_compose, and by pw_compose_noalloc twice."""
    from synthetic import junction
    inst = junction(ng=ng, n_slices=3, n_e=n_e, n_k=1)
    E, k = inst.energies, inst.kpar
    with pw.Context.from_instance(inst) as ctx:
        n = ctx.ng
        assert n == ng
        Sa = torch.zeros((len(E), 4, n, n), dtype=torch.complex128, device="cuda")
        Sb = torch.zeros_like(Sa)
        ref = torch.zeros_like(Sa)
        ctx.slice_smatrix(E, k, 1, Sa)
        ctx.slice_smatrix(E, k, 2, Sb)
        ctx.compose(len(E), Sa, Sb, ref)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
    scale = max(1.0, np.abs(ref).max())
    for _ in range(2):
        out = torch.full_like(Sa, complex(np.nan, np.nan))
        pw.compose_noalloc(n, len(E), Sa, Sb, out)
        torch.cuda.synchronize()
        assert np.abs(out.cpu().numpy() - ref).max() < 1e-11 * scale


@pytest.mark.parametrize("ng,n_e", [(362, 2), (181, 8), (8, 300)])
def test_noalloc_limits_and_chunks(pw, ng, n_e):
    """N_G = 362, the largest size (one point per launch through the array);
    N_G = 181 with 8 points (three points per launch, three launches); 300
    points at N_G = 8 (more than the 256 points one launch takes)."""
    _pair_vs_compose(pw, ng, n_e)


def test_noalloc_rejects_oversize_before_device_work(pw):
    lib = pw.lib()
    assert lib.pw_compose_noalloc(363, 1, 16, 16, 16, None) == 1     # n > 362
    assert lib.pw_compose_noalloc(400, 1, 16, 16, 16, None) == 1
    assert lib.pw_compose_noalloc(0, 1, 16, 16, 16, None) == 1
    assert lib.pw_compose_noalloc(8, 0, None, None, None, None) == 0
