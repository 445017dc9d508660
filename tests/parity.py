"""The parity bar on T shared by the GPU tests.

T is compared relative to itself: |T_gpu - T_oracle| / |T_oracle|.  Below
T_FLOOR the relative error of a tunnelling T stops being meaningful (T = 0
exactly when an electrode has no open channel), so there the bound is
absolute: |T_gpu - T_oracle| <= tol * T_FLOOR."""
import numpy as np

T_FLOOR = 1e-6
TOL_FP64 = 1e-10     # FP64 form against the oracle
TOL_MIXED = 1e-8     # mixed form after refinement against the oracle


def rel_T(got, ref):
    """Elementwise |got - ref| / max(|ref|, T_FLOOR)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), T_FLOOR)
