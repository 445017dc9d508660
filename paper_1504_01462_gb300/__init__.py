"""GB300 plane-wave multiple-scattering transport: Python binding of libpw.

A thin ctypes layer over the C ABI in include/pw.h.  It only marshals
arguments: every step of the computation runs in the CUDA kernels of
libpw.so.  Device buffers are passed as objects with a ``data_ptr()`` method
(e.g. torch CUDA tensors) or as raw integer addresses; host arrays as NumPy
arrays.  If the compiled library is missing, importing this package raises:
there is no CPU fallback.

    ctx = Context.from_instance(inst, precision=FP64)
    T = torch.empty(npts, dtype=torch.float64, device="cuda")
    ctx.transmission(E, kpar, T)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpw.so")

FP64 = 0
MIXED_FP32 = 1

STATUS = {0: "PW_OK", 1: "PW_EINVAL", 2: "PW_ENOMEM", 3: "PW_ECUDA", 4: "PW_ESINGULAR",
          5: "PW_ETHRESH", 6: "PW_ETIMEOUT", 7: "PW_ENOTCONV"}
PW_ETHRESH = 5

EXPORTS = ["pw_setup", "pw_destroy", "pw_status_str", "pw_get_error", "pw_ng", "pw_n_slices",
           "pw_get_gvectors", "pw_potential_tables", "pw_slice_modes", "pw_overlaps",
           "pw_slice_smatrix", "pw_compose", "pw_transmission", "pw_set_profiling",
           "pw_get_profile", "pw_compose_noalloc", "pw_grad", "pw_setup_batch",
           "pw_transmission_batch", "pw_batch_set_options", "pw_batch_get_stats",
           "pw_batch_destroy", "pw_get_error_detail", "pw_selftest_tensor_core",
           "pw_set_sweep_variant", "pw_selftest_slice_product", "pw_slice_mixed", "pw_compose_mixed",
           "pw_transmission_doubling", "pw_selftest_f16_split", "pw_kernel_kinds",
           "pw_kernel_kind_name", "pw_get_kernel_profile", "pw_measure_peaks",
           "pw_set_grad_checkpoint", "pw_workspace_bytes", "pw_selftest_bounded_wait",
           "pw_reduce_transmission", "pw_set_projectors", "pw_transmission_nonlocal",
           "pw_set_periodic_electrode", "pw_transmission_periodic", "pw_selftest_schur",
           "pw_eig_wave", "pw_set_fp64_fallback", "pw_get_fp64_fallback"]


class PwError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({_lib.pw_status_str(code).decode()})")


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p


class SetupDesc(ctypes.Structure):
    _fields_ = [
        ("a1", ctypes.c_double * 2), ("a2", ctypes.c_double * 2),
        ("ecut", ctypes.c_double), ("ng_exact", ctypes.c_int),
        ("n_slices", ctypes.c_int), ("z_edges", _dp),
        ("n_wells", ctypes.c_int), ("well_xyz", _dp), ("well_v0", _dp), ("well_sigma", _dp),
        ("lead_n_wells", ctypes.c_int * 2), ("lead_well_xy", _dp * 2),
        ("lead_well_v0", _dp * 2), ("lead_well_sigma", _dp * 2),
        ("lead_period", ctypes.c_double * 2),
        ("vg_half", ctypes.c_int * 2),
        ("slice_vg", _vp), ("lead_vg", _vp * 2),
        ("precision", ctypes.c_int),
        ("refine_iters", ctypes.c_int),
        ("well_shift_rate", _dp),
        ("lead_shift_rate", (ctypes.c_double * 2) * 2),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpw.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    lib.pw_setup.argtypes = [ctypes.POINTER(SetupDesc), _vp, ctypes.POINTER(_vp)]
    lib.pw_destroy.argtypes = [_vp]
    lib.pw_destroy.restype = None
    lib.pw_status_str.argtypes = [ctypes.c_int]
    lib.pw_status_str.restype = ctypes.c_char_p
    lib.pw_get_error.argtypes = [_vp]
    lib.pw_ng.argtypes = [_vp]
    lib.pw_n_slices.argtypes = [_vp]
    lib.pw_get_gvectors.argtypes = [_vp, _ip]
    lib.pw_potential_tables.argtypes = [_vp, _vp, _ip]
    lib.pw_slice_modes.argtypes = [_vp, _dp, _vp, _vp]
    lib.pw_overlaps.argtypes = [_vp, _dp, _vp]
    lib.pw_slice_smatrix.argtypes = [_vp, ctypes.c_int, _dp, _dp, ctypes.c_int, _vp]
    lib.pw_compose.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
    lib.pw_slice_mixed.argtypes = lib.pw_slice_smatrix.argtypes
    lib.pw_compose_mixed.argtypes = lib.pw_compose.argtypes
    lib.pw_transmission_doubling.argtypes = [_vp, ctypes.c_int, _dp, _dp, ctypes.c_double, _vp, _ip]
    lib.pw_transmission.argtypes = [_vp, ctypes.c_int, _dp, _dp, _vp, _vp, _vp, _vp]
    lib.pw_compose_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
    lib.pw_grad.argtypes = [_vp, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    lib.pw_set_profiling.argtypes = [_vp, ctypes.c_int]
    lib.pw_get_profile.argtypes = [_vp, _dp, ctypes.c_int]
    lib.pw_setup_batch.argtypes = [ctypes.c_int, ctypes.POINTER(SetupDesc), _vp, ctypes.POINTER(_vp)]
    lib.pw_transmission_batch.argtypes = [_vp, _dp, _dp, _vp, _vp, _vp]
    lib.pw_batch_set_options.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    lib.pw_batch_get_stats.argtypes = [_vp, _dp, _ip, _ip, ctypes.c_int, _ip]
    lib.pw_batch_destroy.argtypes = [_vp]
    lib.pw_get_error_detail.argtypes = [_vp, ctypes.c_char_p, ctypes.c_int]
    lib.pw_selftest_tensor_core.argtypes = [_dp, _dp]
    lib.pw_selftest_slice_product.argtypes = [ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_longlong), _dp]
    lib.pw_selftest_f16_split.argtypes = [_dp]
    lib.pw_set_sweep_variant.argtypes = [_vp, ctypes.c_int]
    lib.pw_kernel_kinds.argtypes = []
    lib.pw_kernel_kind_name.argtypes = [ctypes.c_int]
    lib.pw_kernel_kind_name.restype = ctypes.c_char_p
    lib.pw_get_kernel_profile.argtypes = [_vp, _dp, ctypes.c_int]
    lib.pw_measure_peaks.argtypes = [_dp]
    lib.pw_set_grad_checkpoint.argtypes = [_vp, ctypes.c_int]
    lib.pw_workspace_bytes.argtypes = [_vp, _dp]
    lib.pw_selftest_bounded_wait.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.pw_reduce_transmission.argtypes = [ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
    lib.pw_set_projectors.argtypes = [_vp, ctypes.c_int, _dp, _vp, ctypes.c_int]
    lib.pw_transmission_nonlocal.argtypes = [_vp, ctypes.c_int, _dp, _dp, _vp, _vp]
    lib.pw_set_periodic_electrode.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _dp, _dp]
    lib.pw_transmission_periodic.argtypes = [_vp, ctypes.c_int, _dp, _dp, _vp]
    lib.pw_selftest_schur.argtypes = [ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _ip]
    lib.pw_eig_wave.argtypes = [ctypes.c_int, _ip]
    lib.pw_set_fp64_fallback.argtypes = [_vp, ctypes.c_double, ctypes.c_double]
    lib.pw_get_fp64_fallback.argtypes = [_vp, _ip, _dp]
    lib.pw_batch_destroy.restype = None
    return lib


_lib = _load()


def lib():
    """The loaded ctypes library (for symbol checks and direct calls)."""
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _as_dp(a):
    return a.ctypes.data_as(_dp) if a is not None and a.size else None


def compose_noalloc(n, npts, Sa, Sb, Sab, stream=None):
    """Star products Sab = Sa * Sb (Eq. recurrence) without any device
    allocation by the library: for callers that cannot let a library call
    cudaMalloc (the library's fixed 8 MiB device array is the only scratch;
    n <= 362).  Raises PwError on failure."""
    st = _lib.pw_compose_noalloc(int(n), int(npts), _ptr(Sa), _ptr(Sb), _ptr(Sab), stream)
    if st != 0:
        raise PwError(st, "pw_compose_noalloc")


def _build_desc(*, a1, a2, z_edges, ecut=0.0, ng_exact=0, wells_xyz=None, v0=None, sigma=None,
                leads=((None, None, None, 1.0), (None, None, None, 1.0)), slice_vg=None,
                lead_vg=(None, None), vg_half=(0, 0), precision=FP64, refine_iters=0,
                well_shift_rate=None, lead_shift_rate=None):
    """A pw_setup_desc and the host arrays it points into (keep them alive
    until pw_setup returns), and whether it carries a geometry motion."""
    keep = []
    d = SetupDesc()
    d.a1[:] = [float(v) for v in a1]
    d.a2[:] = [float(v) for v in a2]
    d.ecut = float(ecut)
    d.ng_exact = int(ng_exact)
    z = _f64(z_edges)
    keep.append(z)
    d.n_slices = len(z) - 1
    d.z_edges = _as_dp(z)
    if wells_xyz is not None and len(wells_xyz):
        w, v, s = _f64(wells_xyz).reshape(-1, 3), _f64(v0), _f64(sigma)
        keep += [w, v, s]
        d.n_wells = len(w)
        d.well_xyz, d.well_v0, d.well_sigma = _as_dp(w), _as_dp(v), _as_dp(s)
    for side, (xy, lv0, ls, period) in enumerate(leads):
        d.lead_period[side] = float(period)
        if xy is not None and len(xy):
            xy, lv0, ls = _f64(xy).reshape(-1, 2), _f64(lv0), _f64(ls)
            keep += [xy, lv0, ls]
            d.lead_n_wells[side] = len(xy)
            d.lead_well_xy[side] = _as_dp(xy)
            d.lead_well_v0[side] = _as_dp(lv0)
            d.lead_well_sigma[side] = _as_dp(ls)
    d.vg_half[:] = [int(vg_half[0]), int(vg_half[1])]
    if slice_vg is not None:
        sv = _c128(slice_vg)
        keep.append(sv)
        d.slice_vg = sv.ctypes.data
    for side in (0, 1):
        if lead_vg[side] is not None:
            lv = _c128(lead_vg[side])
            keep.append(lv)
            d.lead_vg[side] = lv.ctypes.data
    d.precision = int(precision)
    d.refine_iters = int(refine_iters)
    has_shift = False
    if well_shift_rate is not None:
        r = _f64(well_shift_rate).reshape(-1, 2)
        keep.append(r)
        d.well_shift_rate = _as_dp(r)
        has_shift = True
    if lead_shift_rate is not None:
        lr = np.asarray(lead_shift_rate, dtype=np.float64).reshape(2, 2)
        for side in (0, 1):
            d.lead_shift_rate[side][0] = float(lr[side, 0])
            d.lead_shift_rate[side][1] = float(lr[side, 1])
        has_shift = has_shift or bool(np.any(lr))
    return d, keep, has_shift


def _instance_geometry(inst, refine_iters=0):
    """Keyword arguments of _build_desc for a problem description object
    (attributes as in synthetic.Instance)."""
    leads = [(L.wells_xy, L.v0, L.sigma, L.period) for L in (inst.lead_left, inst.lead_right)]
    lead_vg = inst.lead_vg if inst.lead_vg is not None else (None, None)
    return dict(a1=inst.a1, a2=inst.a2, z_edges=inst.z_edges, ecut=inst.ecut,
                ng_exact=inst.ng_exact, wells_xyz=inst.wells_xyz, v0=inst.v0, sigma=inst.sigma,
                leads=leads, slice_vg=inst.slice_vg, lead_vg=lead_vg, vg_half=inst.vg_half,
                refine_iters=refine_iters,
                well_shift_rate=getattr(inst, "gap_rate_wells", None),
                lead_shift_rate=getattr(inst, "gap_rate_leads", None))


def selftest_tensor_core():
    """(relative error of one TF32 tile product, of the three-product split)
    from the library's tcgen05 self-test on the current device."""
    a = np.zeros(1)
    b = np.zeros(1)
    _check_status(_lib.pw_selftest_tensor_core(_as_dp(a), _as_dp(b)), "pw_selftest_tensor_core")
    return float(a[0]), float(b[0])


def selftest_slice_product(n, ncol):
    """(results differing from the exact leading-slice product, relative error
    of the full slice sum) from the library's exact-slice product self-test
    (the residual's tensor-core path) for a basis of n and ncol columns."""
    bad = ctypes.c_longlong(-1)
    rel = np.zeros(1)
    _check_status(_lib.pw_selftest_slice_product(int(n), int(ncol), ctypes.byref(bad), _as_dp(rel)),
                  "pw_selftest_slice_product")
    return int(bad.value), float(rel[0])


def selftest_f16_split():
    """Relative error of one tile product in the FP16 split (sweep variant
    bit 2) from the library's self-test on the current device."""
    a = np.zeros(1)
    _check_status(_lib.pw_selftest_f16_split(_as_dp(a)), "pw_selftest_f16_split")
    return float(a[0])


def reduce_transmission(T, nopen=None, weight=None, out=None, stream=None):
    """(sum_i w_i T_i, Tbar of Eq. T1_d, mesh points counted) in FP64 on the
    device (pw_reduce_transmission); T, nopen, weight and out are device
    tensors (out: 3 float64 values, allocated when None)."""
    import torch
    if out is None:
        out = torch.zeros(3, dtype=torch.float64, device=T.device)
    _check_status(_lib.pw_reduce_transmission(int(T.numel()), _ptr(T), _ptr(nopen), _ptr(weight), _ptr(out),
                                              stream), "pw_reduce_transmission")
    return out


def selftest_schur(A, select=False):
    """(T, Z, count) of the device Schur form of the complex matrix A."""
    A = np.asfortranarray(np.asarray(A, dtype=np.complex128))
    N = A.shape[0]
    T = np.zeros((N, N), dtype=np.complex128, order="F")
    Z = np.zeros((N, N), dtype=np.complex128, order="F")
    cnt = ctypes.c_int(0)
    _check_status(_lib.pw_selftest_schur(N, A.ctypes.data, T.ctypes.data, Z.ctypes.data, int(bool(select)),
                                         ctypes.byref(cnt)), "pw_selftest_schur")
    return T, Z, cnt.value


def measure_peaks():
    """Measured TFLOP/s of the current device: {'fp64_fma', 'fp64_mma', 'fp32_fma'}."""
    out = np.zeros(3)
    _check_status(_lib.pw_measure_peaks(_as_dp(out)), "pw_measure_peaks")
    return {"fp64_fma": float(out[0]), "fp64_mma": float(out[1]), "fp32_fma": float(out[2])}


def eig_wave(n):
    """Slice Hamiltonians of order n the FP64 eigensolver works on at once on
    the current device (resident CTAs x SMs)."""
    out = ctypes.c_int(0)
    _check_status(_lib.pw_eig_wave(int(n), ctypes.byref(out)), "pw_eig_wave")
    return out.value


def _check_status(st, where):
    if st != 0:
        raise PwError(st, where)


class Context:
    """An owned pw_ctx: one junction problem on the current CUDA device."""

    def __init__(self, *, precision=FP64, stream=None, **geometry):
        d, keep, has_shift = _build_desc(precision=precision, **geometry)
        self.has_shift = has_shift
        h = _vp()
        st = _lib.pw_setup(ctypes.byref(d), stream, ctypes.byref(h))
        if st != 0:
            raise PwError(st, "pw_setup")
        self._h = h
        self.precision = int(precision)

    @classmethod
    def from_instance(cls, inst, precision=FP64, refine_iters=0, stream=None):
        """Marshal a problem description object (attributes as in
        synthetic.Instance) into pw_setup."""
        return cls(precision=precision, stream=stream, **_instance_geometry(inst, refine_iters))

    def close(self):
        if getattr(self, "_h", None):
            _lib.pw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    @property
    def ng(self) -> int:
        return _lib.pw_ng(self._h)

    @property
    def n_slices(self) -> int:
        return _lib.pw_n_slices(self._h)

    def gvectors(self) -> np.ndarray:
        out = np.zeros(2 * self.ng, dtype=np.int32)
        self._check(_lib.pw_get_gvectors(self._h, out.ctypes.data_as(_ip)), "pw_get_gvectors")
        return out.reshape(-1, 2)

    def table_half(self):
        half = np.zeros(2, dtype=np.int32)
        self._check(_lib.pw_potential_tables(self._h, None, half.ctypes.data_as(_ip)),
                    "pw_potential_tables")
        return int(half[0]), int(half[1])

    def potential_tables(self, out):
        self._check(_lib.pw_potential_tables(self._h, _ptr(out), None), "pw_potential_tables")

    def slice_modes(self, kpar, En_out=None, U_out=None):
        k = _f64(kpar)
        self._check(_lib.pw_slice_modes(self._h, _as_dp(k), _ptr(En_out), _ptr(U_out)),
                    "pw_slice_modes")

    def overlaps(self, kpar, O_out):
        k = _f64(kpar)
        self._check(_lib.pw_overlaps(self._h, _as_dp(k), _ptr(O_out)), "pw_overlaps")

    def slice_smatrix(self, E, kpar, iface, S_out):
        E = _f64(E).reshape(-1)
        k = _f64(kpar).reshape(-1, 2)
        self._check(_lib.pw_slice_smatrix(self._h, len(E), _as_dp(E), _as_dp(k), int(iface),
                                          _ptr(S_out)), "pw_slice_smatrix")

    def compose(self, npts, Sa, Sb, Sab):
        self._check(_lib.pw_compose(self._h, int(npts), _ptr(Sa), _ptr(Sb), _ptr(Sab)),
                    "pw_compose")

    def slice_mixed(self, E, kpar, iface, T_out):
        """Mixed elements (I11, I12, S21, S22) of one interface (Eq. recurrence2)."""
        E = _f64(E).reshape(-1)
        k = _f64(kpar).reshape(-1, 2)
        self._check(_lib.pw_slice_mixed(self._h, len(E), _as_dp(E), _as_dp(k), int(iface),
                                        _ptr(T_out)), "pw_slice_mixed")

    def compose_mixed(self, npts, Ta, Tb, Tab):
        """One step of Eq. recurrence2 for npts pairs of mixed elements."""
        self._check(_lib.pw_compose_mixed(self._h, int(npts), _ptr(Ta), _ptr(Tb), _ptr(Tab)),
                    "pw_compose_mixed")

    def transmission_doubling(self, E, kpar, T_out, cond_max=1e4, allow_threshold=False):
        """T by layer doubling (Eq. recurrence2 while the 1-norm of I11 stays
        <= cond_max, then Eq. recurrence) into T_out (device float64[npts]);
        returns the mixed levels done per point (numpy int array)."""
        E = _f64(E).reshape(-1)
        k = _f64(kpar).reshape(-1, 2)
        levels = np.zeros(len(E), dtype=np.int32)
        st = _lib.pw_transmission_doubling(self._h, len(E), _as_dp(E), _as_dp(k), float(cond_max),
                                           _ptr(T_out), levels.ctypes.data_as(_ip))
        if not (st == PW_ETHRESH and allow_threshold):
            self._check(st, "pw_transmission_doubling")
        return levels

    def transmission(self, E, kpar, T_out, t_out=None, nopen_out=None, err_out=None,
                     allow_threshold=False):
        """T(E, k_par) into T_out (device, float64[npts]).  Returns the status
        code (PW_OK, or PW_ETHRESH when allow_threshold is set)."""
        E = _f64(E).reshape(-1)
        k = _f64(kpar).reshape(-1, 2)
        st = _lib.pw_transmission(self._h, len(E), _as_dp(E), _as_dp(k), _ptr(T_out),
                                  _ptr(t_out), _ptr(nopen_out), _ptr(err_out))
        if st == PW_ETHRESH and allow_threshold:
            return st
        self._check(st, "pw_transmission")
        return st

    def grad(self, E, kpar, weight=None, n_wells=None, gap=False):
        """(sum_i w_i T_i, d/dV0 of that sum for every device well) by the
        adjoint in FP64 (pw_grad); with gap=True also d/dtheta of the sum for
        the geometry motion given at setup (a third element)."""
        E = _f64(E).reshape(-1)
        k = _f64(kpar).reshape(-1, 2)
        w = None if weight is None else _f64(weight).reshape(-1)
        sumT = np.zeros(1)
        nw = int(n_wells) if n_wells is not None else 0
        dV0 = np.zeros(max(nw, 1))
        dgap = np.zeros(1)
        st = _lib.pw_grad(self._h, len(E), _as_dp(E), _as_dp(k), _as_dp(w) if w is not None else None,
                          _as_dp(sumT), _as_dp(dV0) if nw else None, _as_dp(dgap) if gap else None)
        self._check(st, "pw_grad")
        if gap:
            return float(sumT[0]), dV0[:nw], float(dgap[0])
        return float(sumT[0]), dV0[:nw]

    def set_sweep_variant(self, variant):
        """Sweep launch variant (pw_set_sweep_variant): bit 0 = 512-thread SIMT
        tiles; mixed form only: bit 1 = GEMM phases on the tcgen05 tensor
        cores, bit 2 = FP16-split [W|Y] of point pairs, bit 3 = LAPACK pivots
        and 128-row triangular blocks, bit 4 = slice-product residual, bit 5 =
        double-float eigenmodes and overlaps, bit 6 = the batch as two point
        groups on two streams."""
        self._check(_lib.pw_set_sweep_variant(self._h, int(variant)), "pw_set_sweep_variant")

    def set_fp64_fallback(self, pivot_ratio_max=1e6, err_max=1e-8):
        """When the mixed form solves a point again in FP64
        (pw_set_fp64_fallback): an LU diagonal spread above pivot_ratio_max,
        an estimated error above err_max, or a zero FP32 pivot."""
        self._check(_lib.pw_set_fp64_fallback(self._h, float(pivot_ratio_max), float(err_max)),
                    "pw_set_fp64_fallback")

    def fp64_fallback(self):
        """(points solved again in FP64, largest LU diagonal spread) of the
        last transmission call."""
        pts = ctypes.c_int(0)
        ratio = ctypes.c_double(0.0)
        self._check(_lib.pw_get_fp64_fallback(self._h, ctypes.byref(pts), ctypes.byref(ratio)),
                    "pw_get_fp64_fallback")
        return pts.value, ratio.value

    def set_profiling(self, on=True, stride=1):
        """Stage and per-kernel launch timing; with `stride` k every k-th
        launch of each kernel kind is bracketed by CUDA events."""
        self._check(_lib.pw_set_profiling(self._h, max(1, int(stride)) if on else 0), "pw_set_profiling")

    def set_projectors(self, params, D, quad_nodes=16):
        """Gaussian separable projectors (pw_set_projectors): params (m, 6) =
        tau_x, tau_y, tau_z, sigma, z_lo, z_hi; D (m, m) complex."""
        P = _f64(params).reshape(-1, 6)
        Dm = np.ascontiguousarray(np.asarray(D, dtype=np.complex128).reshape(len(P), len(P)))
        self._check(_lib.pw_set_projectors(self._h, len(P), _as_dp(P), Dm.ctypes.data if len(P) else None,
                                           int(quad_nodes)), "pw_set_projectors")

    def transmission_nonlocal(self, E, kpar, T_out, C_out=None, allow_threshold=False):
        """T with the projector terms into T_out (device float64); C_out (device
        complex128, npts x m x N_G) or None."""
        E = _f64(E).reshape(-1)
        k = _f64(kpar).reshape(-1, 2)
        st = _lib.pw_transmission_nonlocal(self._h, len(E), _as_dp(E), _as_dp(k), _ptr(T_out), _ptr(C_out))
        if st == PW_ETHRESH and allow_threshold:
            return st
        self._check(st, "pw_transmission_nonlocal")
        return st

    def set_periodic_electrode(self, side, tables, dz, a3_perp=(0.0, 0.0)):
        """A periodic electrode (pw_set_periodic_electrode): side 0 left, 1
        right; tables (M, 2Dm+1, 2Dn+1) complex in the context's table layout."""
        tab = np.ascontiguousarray(np.asarray(tables, dtype=np.complex128))
        dzs = _f64(dz).reshape(-1)
        a3 = _f64(a3_perp).reshape(2)
        self._check(_lib.pw_set_periodic_electrode(self._h, int(side), len(dzs), tab.ctypes.data, _as_dp(dzs),
                                                   _as_dp(a3)), "pw_set_periodic_electrode")

    def transmission_periodic(self, E, kpar, T_out):
        """T between the periodic electrodes into T_out (device float64)."""
        E = _f64(E).reshape(-1)
        k = _f64(kpar).reshape(-1, 2)
        st = _lib.pw_transmission_periodic(self._h, len(E), _as_dp(E), _as_dp(k), _ptr(T_out))
        self._check(st, "pw_transmission_periodic")

    def set_grad_checkpoint(self, interval=0):
        """Segment length of pw_grad's checkpointed recomputation (0: ceil(sqrt(N+1)))."""
        self._check(_lib.pw_set_grad_checkpoint(self._h, int(interval)), "pw_set_grad_checkpoint")

    def workspace_bytes(self):
        """Device bytes the context's per-call workspaces hold now."""
        out = np.zeros(1)
        self._check(_lib.pw_workspace_bytes(self._h, _as_dp(out)), "pw_workspace_bytes")
        return float(out[0])

    def get_kernel_profile(self, reset=True):
        """{kernel kind: (sampled ms, sampled launches, all launches)} since the
        last reset, for every kind that launched."""
        nk = _lib.pw_kernel_kinds()
        out = np.zeros(3 * nk)
        self._check(_lib.pw_get_kernel_profile(self._h, _as_dp(out), int(bool(reset))),
                    "pw_get_kernel_profile")
        return {_lib.pw_kernel_kind_name(k).decode(): (out[3 * k], int(out[3 * k + 1]), int(out[3 * k + 2]))
                for k in range(nk) if out[3 * k + 2] > 0}

    def get_profile(self, reset=True):
        """{'sweep_ms', 'sweep_launches', 'modes_ms', 'modes_stages', 'overlap_ms',
        'overlap_stages', 'refine_ms', 'refine_stages', 'wy_ms', 'wy_launches'}
        accumulated since the last reset."""
        out = np.zeros(10)
        self._check(_lib.pw_get_profile(self._h, _as_dp(out), int(bool(reset))), "pw_get_profile")
        keys = ["sweep_ms", "sweep_launches", "modes_ms", "modes_stages", "overlap_ms",
                "overlap_stages", "refine_ms", "refine_stages", "wy_ms", "wy_launches"]
        # refine_stages counts refinement passes
        return dict(zip(keys, out.tolist()))

    def _check(self, st, where):
        """Raise PwError for a failing status, with the library's record of
        the first failing CUDA call of this context when it has one."""
        if st != 0:
            buf = ctypes.create_string_buffer(160)
            if getattr(self, "_h", None):
                _lib.pw_get_error_detail(self._h, buf, 160)
            raise PwError(st, f"{where} [{buf.value.decode()}]" if buf.value else where)


class Batch:
    """An owned pw_batch: independent problems of uneven basis size and slice
    count, one (E, k_par) point each (pw_setup_batch)."""

    def __init__(self, geometries, precision=FP64, refine_iters=0, stream=None):
        descs = (SetupDesc * len(geometries))()
        keep = []
        for i, g in enumerate(geometries):
            d, k, _ = _build_desc(**dict(g, precision=precision, refine_iters=refine_iters))
            descs[i] = d
            keep.append(k)
        h = _vp()
        st = _lib.pw_setup_batch(len(geometries), descs, stream, ctypes.byref(h))
        if st != 0:
            raise PwError(st, "pw_setup_batch")
        self._h = h
        self.n = len(geometries)

    @classmethod
    def from_instances(cls, insts, precision=FP64, refine_iters=0, stream=None):
        return cls([_instance_geometry(x) for x in insts], precision, refine_iters, stream)

    def set_options(self, use_graph=True, variant=-1):
        _check_status(_lib.pw_batch_set_options(self._h, int(bool(use_graph)), int(variant)),
                       "pw_batch_set_options")

    def transmission(self, E, kpar, T_out, nopen_out=None, err_out=None, allow_threshold=False):
        """T of instance i at (E[i], kpar[i]) into T_out[i] (device float64)."""
        E = _f64(E).reshape(-1)
        k = _f64(kpar).reshape(-1, 2)
        if len(E) != self.n or len(k) != self.n:
            raise ValueError("one (E, k_par) point per instance")
        st = _lib.pw_transmission_batch(self._h, _as_dp(E), _as_dp(k), _ptr(T_out), _ptr(nopen_out),
                                        _ptr(err_out))
        if st == PW_ETHRESH and allow_threshold:
            return st
        _check_status(st, "pw_transmission_batch")
        return st

    def stats(self):
        """Stage times of the last call and the tile variant chosen per N_G."""
        out = np.zeros(8)
        ng = np.zeros(64, dtype=np.int32)
        var = np.zeros(64, dtype=np.int32)
        cnt = np.zeros(1, dtype=np.int32)
        _check_status(_lib.pw_batch_get_stats(self._h, _as_dp(out), ng.ctypes.data_as(_ip),
                                               var.ctypes.data_as(_ip), 64,
                                               cnt.ctypes.data_as(_ip)), "pw_batch_get_stats")
        keys = ["modes_ms", "overlap_ms", "sweep_ms", "refine_ms", "tune_ms", "chunks",
                "graph_launches", "sweep_launches"]
        res = dict(zip(keys, out.tolist()))
        k = int(min(cnt[0], 64))
        res["variant"] = {int(ng[i]): int(var[i]) for i in range(k)}
        return res

    def close(self):
        if getattr(self, "_h", None):
            _lib.pw_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


__all__ = ["Context", "Batch", "PwError", "FP64", "MIXED_FP32", "EXPORTS", "LIB_PATH", "lib",
           "compose_noalloc", "selftest_tensor_core"]
