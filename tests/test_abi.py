"""The C-ABI library loads without a GPU and exports every entry point that
include/pw.h declares; argument validation that needs no device works."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pw_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def pw():
    import __graft_entry__ as g
    g.build()
    import paper_1504_01462_gb300 as pw
    return pw


def test_every_declared_symbol_is_exported(pw):
    names = _declared()
    assert len(names) >= 13
    lib = pw.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pw.EXPORTS) <= set(names)


def test_status_strings(pw):
    lib = pw.lib()
    for code in range(8):
        assert lib.pw_status_str(code)
    assert lib.pw_status_str(0) == b"ok"


def test_invalid_descriptors_rejected_before_any_device_call(pw):
    lib = pw.lib()
    h = ctypes.c_void_p()
    assert lib.pw_setup(None, None, ctypes.byref(h)) == 1
    d = pw.SetupDesc()
    d.a1[:] = [5.0, 0.0]
    d.a2[:] = [0.0, 5.0]
    d.ecut = 8.0
    d.n_slices = 0
    assert lib.pw_setup(ctypes.byref(d), None, ctypes.byref(h)) == 1       # no slices
    z = np.array([0.0, 1.0, 1.0])                                           # not increasing
    d.n_slices = 2
    d.z_edges = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.pw_setup(ctypes.byref(d), None, ctypes.byref(h)) == 1
    z2 = np.array([0.0, 1.0, 2.0])
    d.z_edges = z2.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.precision = 7                                                          # unknown precision
    assert lib.pw_setup(ctypes.byref(d), None, ctypes.byref(h)) == 1
    d.precision = 0
    d.a2[:] = [10.0, 0.0]                                                    # degenerate cell
    assert lib.pw_setup(ctypes.byref(d), None, ctypes.byref(h)) == 1
    assert lib.pw_ng(None) == 0 and lib.pw_n_slices(None) == 0
    assert lib.pw_get_error(None) == 1
    lib.pw_destroy(None)


def test_batch_arguments_rejected_before_any_device_call(pw):
    """pw_setup_batch refuses an empty batch and mixed precisions before it
    sets any instance up; the batch calls refuse null handles."""
    lib = pw.lib()
    h = ctypes.c_void_p()
    descs = (pw.SetupDesc * 2)()
    assert lib.pw_setup_batch(0, descs, None, ctypes.byref(h)) == 1
    assert lib.pw_setup_batch(2, None, None, ctypes.byref(h)) == 1
    descs[0].precision = 0
    descs[1].precision = 1
    assert lib.pw_setup_batch(2, descs, None, ctypes.byref(h)) == 1
    descs[1].precision = 0
    descs[1].refine_iters = 3
    assert lib.pw_setup_batch(2, descs, None, ctypes.byref(h)) == 1
    e = np.zeros(1)
    assert lib.pw_transmission_batch(None, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, None,
                                     None) == 1
    assert lib.pw_batch_set_options(None, 1, -1) == 1
    assert lib.pw_batch_get_stats(None, None, None, None, 0, None) == 1
    lib.pw_batch_destroy(None)


def test_binding_marshals_batches_and_contexts(pw):
    """The ctypes binding builds every descriptor of a batch and of a context
    from problem objects; without a CUDA device the library answers with a
    CUDA status (never a Python error from the marshalling)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present: the GPU tests cover this path")
    from synthetic import minimal_cell, uneven_batch
    insts = uneven_batch(3, ng_choices=(16, 24), ns_range=(3, 5))
    with pytest.raises(pw.PwError) as e:
        pw.Batch.from_instances(insts, pw.MIXED_FP32, 2)
    assert e.value.code == 3      # PW_ECUDA
    with pytest.raises(pw.PwError) as e:
        pw.Context.from_instance(insts[0], pw.MIXED_FP32, 2)
    assert e.value.code == 3      # PW_ECUDA
    with pytest.raises(pw.PwError) as e:
        pw.Context.from_instance(minimal_cell())
    assert e.value.code == 3      # PW_ECUDA


def test_product_and_generators_never_use_the_oracle():
    """The oracle is test infrastructure: no module of the package, the CUDA
    sources or the shared input generators imports or names it, and the
    oracle imports nothing from the package (the two share no code)."""
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|\boracle\.", re.M)
    for base in ("paper_1504_01462_gb300", "synthetic"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, base)):
            if "_build" in dirpath or "__pycache__" in dirpath:
                continue
            for f in files:
                if f.endswith((".py", ".cu", ".cuh", ".h")):
                    src = open(os.path.join(dirpath, f)).read()
                    assert not pat.search(src), os.path.join(dirpath, f)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1504_01462_gb300" not in src and "ctypes" not in src, f
