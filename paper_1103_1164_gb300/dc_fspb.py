"""Python binding of the C-ABI library libdc_fspb.so (include/dc_fspb.h).

Argument marshalling only: every step of the dose computation runs in the
library's CUDA kernels.  Each ``dc_fspb_*`` function here has the name and the
meaning of the C entry point it calls.  Arrays may be NumPy arrays (host
memory) or contiguous float32 torch CUDA tensors (device memory; the
DC_DEVICE_PTRS flag is then set for the call).  There is no CPU fallback: if
the library is not built, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DC_OK, DC_EINVAL, DC_ENOMEM, DC_ECUDA, DC_ETIMEOUT, DC_EUNSUPPORTED = range(6)
DC_DEVICE_PTRS = 1
DC_BATCH_DENSITY = 2
DC_F32, DC_BF16 = 0, 1
DC_LATERAL_ISO, DC_LATERAL_AXIS, DC_LATERAL_MLP = 0, 1, 2
DC_PRECISION_FP32, DC_PRECISION_BF16 = 0, 1
MLP_PARAMS = 7491
DC_SPMM_STATIC_MAX_BEAMLETS, DC_SPMM_STATIC_MAX_PARTIALS = 8192, 4194304

_lib = None


class DcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "DC_OK", 1: "DC_EINVAL", 2: "DC_ENOMEM", 3: "DC_ECUDA", 4: "DC_ETIMEOUT",
           5: "DC_EUNSUPPORTED"}


class dc_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_float), ("dy", C.c_float), ("dz", C.c_float),
                ("ox", C.c_float), ("oy", C.c_float), ("oz", C.c_float)]


class dc_gamma_stats(C.Structure):
    _fields_ = [("gamma_max", C.c_double), ("gamma_avg50", C.c_double), ("pass50_pct", C.c_double),
                ("n50", C.c_int64), ("dose_max", C.c_float)]


class dc_leaf_sequence(C.Structure):
    _fields_ = [("n_leaves", C.c_int32), ("n_cp", C.c_int32), ("edges", C.c_void_p), ("mu", C.c_void_p),
                ("left", C.c_void_p), ("right", C.c_void_p), ("jaw_x1", C.c_float), ("jaw_x2", C.c_float),
                ("jaw_y1", C.c_float), ("jaw_y2", C.c_float), ("transmission", C.c_float)]


class dc_beam(C.Structure):
    _fields_ = [("gantry_deg", C.c_float), ("couch_deg", C.c_float), ("coll_deg", C.c_float),
                ("sad", C.c_float), ("iso", C.c_float * 3), ("field_x", C.c_float),
                ("field_y", C.c_float)]


class dc_kernel_coeffs(C.Structure):
    _fields_ = [("A", C.c_void_p), ("a_nt", C.c_int32), ("a_ntheta", C.c_int32),
                ("a_dt", C.c_float), ("a_dtheta", C.c_float),
                ("water", C.c_void_p), ("w_n", C.c_int32), ("w_dt", C.c_float),
                ("dens", C.c_void_p), ("f_n", C.c_int32), ("f_rho0", C.c_float), ("f_drho", C.c_float),
                ("roi_radius", C.c_float), ("smooth_sigma", C.c_float), ("rho_surface", C.c_float),
                ("density_correction", C.c_int32), ("lateral_mode", C.c_int32),
                ("reserved", C.c_int32 * 2)]


EXPORTS = ["dc_last_error", "dc_status_str", "dc_fspb_create", "dc_fspb_destroy",
           "dc_fspb_n_beamlets", "dc_fspb_n_voxels", "dc_fspb_list_entries", "dc_fspb_dose", "dc_fspb_dose_batch",
           "dc_fspb_pair_count", "dc_fspb_dose_matrix", "dc_fspb_dose_and_matrix", "dc_fspb_get_smoothed",
           "dc_fspb_get_beamlets", "dc_fspb_get_tables", "dc_fspb_set_density",
           "dc_fspb_launch_count", "dc_fspb_autotune", "dc_fspb_spmm_prepare", "dc_fspb_spmm_info",
           "dc_fspb_spmm", "dc_fspb_spmm_noalloc", "dc_fspb_device_status", "dc_fspb_set_surrogate",
           "dc_fspb_set_lateral_mode", "dc_fspb_set_precision", "dc_fspb_set_tables", "dc_fspb_dose_vjp", "dc_fspb_lateral_fallbacks", "dc_fspb_stencils",
           "dc_mlp_create", "dc_mlp_destroy", "dc_mlp_get_params", "dc_mlp_get_state", "dc_mlp_set_state", "dc_mlp_set_precision", "dc_mlp_gradient", "dc_mlp_train",
           "dc_mlp_predict", "dc_fspb_batch_create", "dc_fspb_batch_destroy", "dc_fspb_batch_buffers",
           "dc_fspb_batch_run", "dc_fspb_batch_dose", "dc_fspb_batch_synchronize", "dc_fspb_batch_kernels",
           "dc_fspb_batch_autotune", "dc_fspb_batch_set_variant", "dc_gamma_index", "dc_fluence_from_leaves"]


def library_path() -> str:
    """The library this binding loads: the bounds-checked build when
    DC_FSPB_CHECKED=1 is set in the environment (read at the first load)."""
    return _build.LIB_CHECKED if os.environ.get("DC_FSPB_CHECKED") == "1" else _build.LIB


def load():
    """Loads the built library (raises if it is missing: no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run paper_1103_1164_gb300.build.build() "
                           "(nvcc for sm_103a) first")
    L = C.CDLL(path)
    vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
    L.dc_last_error.restype = C.c_char_p
    L.dc_status_str.restype = C.c_char_p
    L.dc_status_str.argtypes = [C.c_int]
    L.dc_fspb_create.argtypes = [vp, C.POINTER(dc_grid), C.POINTER(dc_beam), i32, C.c_float,
                                 C.c_float, C.POINTER(dc_kernel_coeffs), u32, vp, C.POINTER(vp)]
    L.dc_fspb_destroy.argtypes = [vp]
    L.dc_fspb_n_beamlets.argtypes = [vp, C.POINTER(i32)]
    L.dc_fspb_n_voxels.argtypes = [vp, C.POINTER(i64)]
    L.dc_fspb_dose.argtypes = [vp, vp, vp, u32]
    L.dc_fspb_dose_batch.argtypes = [vp, vp, i32, vp, u32]
    L.dc_fspb_pair_count.argtypes = [vp, C.POINTER(i64)]
    L.dc_fspb_dose_matrix.argtypes = [vp, i32, vp, vp, vp, u32]
    L.dc_fspb_dose_and_matrix.argtypes = [vp, vp, vp, i32, vp, vp, vp, u32]
    L.dc_fspb_get_smoothed.argtypes = [vp, vp, u32]
    L.dc_fspb_get_beamlets.argtypes = [vp, vp]
    L.dc_fspb_get_tables.argtypes = [vp, i32, vp, vp, vp, i32, C.POINTER(i32)]
    L.dc_fspb_set_density.argtypes = [vp, vp, u32]
    L.dc_fspb_launch_count.argtypes = [C.POINTER(C.c_uint64)]
    L.dc_fspb_autotune.argtypes = [vp, vp, u32, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                   C.POINTER(C.c_float)]
    L.dc_fspb_spmm_prepare.argtypes = [vp]
    L.dc_fspb_spmm_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    L.dc_fspb_spmm.argtypes = [vp, vp, i32, vp, u32]
    L.dc_fspb_spmm_noalloc.argtypes = [vp, vp, i32, vp]
    L.dc_fspb_device_status.argtypes = [vp]
    L.dc_fspb_set_surrogate.argtypes = [vp, vp, C.c_float, C.c_float]
    L.dc_fspb_set_lateral_mode.argtypes = [vp, i32]
    L.dc_fspb_set_precision.argtypes = [vp, i32]
    L.dc_fspb_set_tables.argtypes = [vp, vp, vp]
    L.dc_fspb_list_entries.argtypes = [vp, C.POINTER(i64)]
    L.dc_mlp_get_state.argtypes = [vp, vp, vp, vp, C.POINTER(i64)]
    L.dc_mlp_set_state.argtypes = [vp, vp, vp, vp, i64]
    L.dc_mlp_set_precision.argtypes = [vp, i32]
    L.dc_fspb_dose_vjp.argtypes = [vp, vp, vp, vp, vp, vp, u32]
    L.dc_fspb_lateral_fallbacks.argtypes = [vp, C.POINTER(i64)]
    L.dc_fspb_stencils.argtypes = [vp, vp, vp, i32, vp, vp, u32]
    L.dc_mlp_create.argtypes = [vp, vp, C.POINTER(vp)]
    L.dc_mlp_destroy.argtypes = [vp]
    L.dc_mlp_get_params.argtypes = [vp, vp]
    L.dc_mlp_gradient.argtypes = [vp, vp, vp, i32, vp, C.POINTER(C.c_float), u32]
    L.dc_mlp_train.argtypes = [vp, vp, vp, i32, i32, i32, C.c_float, C.POINTER(C.c_float), u32]
    L.dc_mlp_predict.argtypes = [vp, vp, i32, vp, u32, vp]
    L.dc_fspb_batch_create.argtypes = [vp, i32, vp, C.POINTER(vp)]
    L.dc_fspb_batch_destroy.argtypes = [vp]
    L.dc_fspb_batch_buffers.argtypes = [vp, i32, C.POINTER(vp), C.POINTER(vp)]
    L.dc_fspb_batch_run.argtypes = [vp, u32]
    L.dc_fspb_batch_dose.argtypes = [vp, vp, vp, u32]
    L.dc_fspb_batch_synchronize.argtypes = [vp]
    L.dc_fspb_batch_kernels.argtypes = [vp, u32, C.POINTER(i32)]
    L.dc_fspb_batch_autotune.argtypes = [vp, C.POINTER(i32), C.POINTER(C.c_float)]
    L.dc_fspb_batch_set_variant.argtypes = [vp, i32]
    L.dc_gamma_index.argtypes = [vp, vp, C.POINTER(dc_grid), C.c_float, C.c_float, C.c_float, vp,
                                 C.POINTER(dc_gamma_stats), vp, u32]
    L.dc_fluence_from_leaves.argtypes = [vp, C.POINTER(dc_leaf_sequence), vp, u32]
    for name in EXPORTS:
        if name not in ("dc_last_error", "dc_status_str"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status):
    if status != DC_OK:
        raise DcError(status, load().dc_last_error().decode())


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype=np.float32):
    """(pointer, device flag) of a host NumPy array or a CUDA torch tensor.

    dtype is the element type the C entry point reads (None: any, for value
    arrays whose type travels as a separate argument)."""
    if _is_torch(a):
        if not a.is_cuda or not a.is_contiguous():
            raise ValueError("torch tensors must be contiguous CUDA tensors")
        if dtype is not None and str(a.dtype) != "torch." + np.dtype(dtype).name:
            raise ValueError(f"expected a {np.dtype(dtype).name} tensor, got {a.dtype}")
        return C.c_void_p(a.data_ptr()), DC_DEVICE_PTRS
    if not (isinstance(a, np.ndarray) and a.flags.c_contiguous and a.dtype == dtype):
        raise ValueError(f"host arrays must be C-contiguous {np.dtype(dtype).name} NumPy arrays")
    return a.ctypes.data_as(C.c_void_p), 0


def _same_kind(*flags):
    if len(set(flags)) != 1:
        raise ValueError("all array arguments of one call must be host arrays or all CUDA tensors")
    return flags[0]


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class Plan:
    """Owns a dc_plan*; freed by dc_fspb_destroy (or when garbage-collected)."""

    def __init__(self, handle, n_beamlets, n_voxels, grid_shape, keep=(), n_beams=0):
        self.handle = handle
        self.n_beams = n_beams
        self.n_beamlets = n_beamlets
        self.n_voxels = n_voxels
        self.shape = grid_shape
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.dc_fspb_destroy(self.handle)
            self.handle = None


def make_coeffs(comm, lateral_mode=DC_LATERAL_ISO):
    """dc_kernel_coeffs from a synth.Commissioning (arrays kept alive by the caller)."""
    A = np.ascontiguousarray(comm.A, np.float32)
    W = np.ascontiguousarray(comm.water, np.float32)
    D = np.ascontiguousarray(comm.dens, np.float32)
    c = dc_kernel_coeffs(A.ctypes.data, A.shape[1], A.shape[0], comm.a_dt, comm.a_dtheta,
                         W.ctypes.data, W.shape[1], comm.w_dt, D.ctypes.data, D.shape[1],
                         comm.f_rho0, comm.f_drho, comm.roi_radius, comm.smooth_sigma,
                         comm.rho_surface, int(comm.density_correction), int(lateral_mode),
                         (C.c_int32 * 2)(0, 0))
    return c, (A, W, D)


def dc_fspb_create(ct_density, grid, beams, beamlet_x, beamlet_y, comm, stream=None,
                   lateral_mode=DC_LATERAL_ISO) -> Plan:
    """Builds a plan (ct_density: [nz, ny, nx] float32, host array or CUDA tensor)."""
    L = load()
    p_rho, flag = _ptr(ct_density)
    g = dc_grid(grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, grid.ox, grid.oy, grid.oz)
    arr = (dc_beam * len(beams))()
    for q, b in enumerate(beams):
        arr[q] = dc_beam(b.gantry_deg, b.couch_deg, b.coll_deg, b.sad, (C.c_float * 3)(*b.iso),
                         b.field_x, b.field_y)
    coeffs, keep = make_coeffs(comm, lateral_mode)
    h = C.c_void_p()
    s = _current_stream() if stream is None else stream
    _check(L.dc_fspb_create(p_rho, C.byref(g), arr, len(beams), beamlet_x, beamlet_y,
                            C.byref(coeffs), flag, C.c_void_p(s), C.byref(h)))
    nb, nv = C.c_int32(), C.c_int64()
    _check(L.dc_fspb_n_beamlets(h, C.byref(nb)))
    _check(L.dc_fspb_n_voxels(h, C.byref(nv)))
    return Plan(h, nb.value, nv.value, (grid.nz, grid.ny, grid.nx), n_beams=len(beams))


def dc_fspb_create_from(plan_inputs, stream=None, device_density=None,
                        lateral_mode=DC_LATERAL_ISO) -> Plan:
    """dc_fspb_create from a synth.Plan."""
    rho = plan_inputs.rho if device_density is None else device_density
    return dc_fspb_create(np.ascontiguousarray(rho, np.float32) if device_density is None else rho,
                          plan_inputs.grid, plan_inputs.beams, plan_inputs.beamlet_x,
                          plan_inputs.beamlet_y, plan_inputs.comm, stream, lateral_mode)


def dc_fspb_set_density(plan: Plan, ct_density):
    """Recomputes steps 1-6 of the plan for a new density on the same grid."""
    p, flag = _ptr(ct_density)
    _check(load().dc_fspb_set_density(plan.handle, p, flag))


def dc_fspb_autotune(plan: Plan, fluence):
    """Picks the plan's beam's-eye-view cell size by timing; returns (tile, slab, ms)."""
    p, flag = _ptr(fluence)
    t, s, ms = C.c_float(), C.c_float(), C.c_float()
    _check(load().dc_fspb_autotune(plan.handle, p, flag, C.byref(t), C.byref(s), C.byref(ms)))
    return t.value, s.value, ms.value


def dc_fspb_spmm_prepare(plan: Plan):
    """Builds the plan's block-sparse BF16 dose-deposition matrix for dc_fspb_spmm."""
    _check(load().dc_fspb_spmm_prepare(plan.handle))


def dc_fspb_spmm_info(plan: Plan):
    """(tiles of 128 x 16, row-blocks of 128 voxels) of the prepared matrix."""
    c, r = C.c_int64(), C.c_int64()
    _check(load().dc_fspb_spmm_info(plan.handle, C.byref(c), C.byref(r)))
    return c.value, r.value


def _spmm_shapes(plan: Plan, F, Y):
    """k of F [B, k], after checking F and Y [V, k] against the plan (before any launch)."""
    if len(F.shape) != 2 or int(F.shape[0]) != plan.n_beamlets:
        raise ValueError(f"F must be [n_beamlets={plan.n_beamlets}, k], got {tuple(F.shape)}")
    k = int(F.shape[1])
    if tuple(int(s) for s in Y.shape) != (plan.n_voxels, k):
        raise ValueError(f"Y must be [n_voxels={plan.n_voxels}, k={k}], got {tuple(Y.shape)}")
    return k


def dc_fspb_spmm(plan: Plan, F, Y=None):
    """Y [V, k] = M F for F [B, k] (k <= 64) on the tensor cores."""
    if Y is None:
        Y = np.empty((plan.n_voxels, F.shape[1] if len(F.shape) == 2 else 0), np.float32)
    k = _spmm_shapes(plan, F, Y)
    pf, f1 = _ptr(F)
    py, f2 = _ptr(Y)
    _check(load().dc_fspb_spmm(plan.handle, pf, k, py, _same_kind(f1, f2)))
    return Y


def dc_fspb_spmm_noalloc(plan: Plan, F, Y):
    """dc_fspb_spmm for device tensors F [B, k], Y [V, k] with static scratch (no device allocation)."""
    _spmm_shapes(plan, F, Y)
    pf, f1 = _ptr(F)
    py, f2 = _ptr(Y)
    if not (f1 & f2 & DC_DEVICE_PTRS):
        raise ValueError("dc_fspb_spmm_noalloc takes device tensors")
    _check(load().dc_fspb_spmm_noalloc(plan.handle, pf, int(F.shape[1]), py))
    return Y


def dc_fspb_device_status(plan: Plan):
    _check(load().dc_fspb_device_status(plan.handle))


def dc_fspb_set_surrogate(plan: Plan, params, rho_lo=0.05, rho_hi=2.0):
    """Loads the surrogate network's 7491 parameters (host float32) and its training density range."""
    p = np.ascontiguousarray(params, np.float32)
    assert p.size == MLP_PARAMS
    _check(load().dc_fspb_set_surrogate(plan.handle, p.ctypes.data_as(C.c_void_p), rho_lo, rho_hi))


def dc_fspb_set_lateral_mode(plan: Plan, mode: int):
    _check(load().dc_fspb_set_lateral_mode(plan.handle, int(mode)))


def dc_fspb_list_entries(plan: Plan) -> int:
    """(voxel, beam) entries of the plan's voxel lists (the lateral-factor passes' work)."""
    n = C.c_int64()
    _check(load().dc_fspb_list_entries(plan.handle, C.byref(n)))
    return n.value


def dc_fspb_set_tables(plan: Plan, water, dens):
    """New water tables [4, w_n] and density functions [6, f_n] (host float32) for the plan."""
    w = np.ascontiguousarray(water, np.float32)
    d = np.ascontiguousarray(dens, np.float32)
    _check(load().dc_fspb_set_tables(plan.handle, w.ctypes.data_as(C.c_void_p), d.ctypes.data_as(C.c_void_p)))


def dc_fspb_dose_vjp(plan: Plan, fluence, weights, w_n: int, f_n: int, out=None):
    """Gradients of sum_v weights[v] D(v) with respect to the tables:
    (g_water [4, w_n], g_dens [4, f_n], g_corr [2]).  Host arrays, or CUDA
    tensors for all (out = the three device tensors then)."""
    if len(fluence.shape) != 1 or int(fluence.shape[0]) != plan.n_beamlets:
        raise ValueError("fluence must have n_beamlets entries")
    if int(np.prod(weights.shape)) != plan.n_voxels:
        raise ValueError("weights must have n_voxels entries")
    if out is None:
        out = (np.empty((4, w_n), np.float32), np.empty((4, f_n), np.float32), np.empty(2, np.float32))
    pf, f1 = _ptr(fluence)
    pw, f2 = _ptr(weights)
    ptrs, flags = [], [f1, f2]
    for a, n in zip(out, (4 * w_n, 4 * f_n, 2)):
        if int(np.prod(a.shape)) != n:
            raise ValueError("gradient buffers must hold 4 w_n, 4 f_n and 2 entries")
        p, f = _ptr(a)
        ptrs.append(p)
        flags.append(f)
    _check(load().dc_fspb_dose_vjp(plan.handle, pf, pw, *ptrs, _same_kind(*flags)))
    return out


def dc_fspb_set_precision(plan: Plan, precision: int):
    """Arithmetic of the direct dose: DC_PRECISION_FP32 or DC_PRECISION_BF16."""
    _check(load().dc_fspb_set_precision(plan.handle, int(precision)))


def dc_fspb_lateral_fallbacks(plan: Plan) -> int:
    n = C.c_int64()
    _check(load().dc_fspb_lateral_fallbacks(plan.handle, C.byref(n)))
    return n.value


def dc_fspb_stencils(plan: Plan, voxels, beams):
    """(X [n, 48] nearest-voxel taps, T [n, 3] axis-stencil densities) for (voxel, beam) pairs."""
    v = np.ascontiguousarray(voxels, np.int32)
    b = np.ascontiguousarray(beams, np.int32)
    n = v.size
    X = np.empty((n, 48), np.float32)
    T = np.empty((n, 3), np.float32)
    _check(load().dc_fspb_stencils(plan.handle, v.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p), n,
                                   X.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p), 0))
    return X, T


class Mlp:
    """Trainer of the surrogate network (dc_mlp_*) on the GPU: FP32, or BF16
    tensor-core products with FP32 master parameters (precision)."""

    def __init__(self, params, stream=None, precision=DC_PRECISION_FP32):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == MLP_PARAMS
        h = C.c_void_p()
        s = _current_stream() if stream is None else stream
        _check(load().dc_mlp_create(p.ctypes.data_as(C.c_void_p), C.c_void_p(s), C.byref(h)))
        self.handle = h
        if precision != DC_PRECISION_FP32:
            _check(load().dc_mlp_set_precision(self.handle, int(precision)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.dc_mlp_destroy(self.handle)
            self.handle = None

    def params(self):
        out = np.empty(MLP_PARAMS, np.float32)
        _check(load().dc_mlp_get_params(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out

    def state(self):
        """(theta, m1, m2, step): everything training continues from."""
        th, m1, m2 = (np.empty(MLP_PARAMS, np.float32) for _ in range(3))
        st = C.c_int64()
        vp = C.c_void_p
        _check(load().dc_mlp_get_state(self.handle, th.ctypes.data_as(vp), m1.ctypes.data_as(vp),
                                       m2.ctypes.data_as(vp), C.byref(st)))
        return th, m1, m2, st.value

    def set_state(self, theta, m1, m2, step):
        th, a, b = (np.ascontiguousarray(x, np.float32) for x in (theta, m1, m2))
        assert th.size == a.size == b.size == MLP_PARAMS
        vp = C.c_void_p
        _check(load().dc_mlp_set_state(self.handle, th.ctypes.data_as(vp), a.ctypes.data_as(vp),
                                       b.ctypes.data_as(vp), int(step)))

    def gradient(self, X, T):
        X = np.ascontiguousarray(X, np.float32)
        T = np.ascontiguousarray(T, np.float32)
        g = np.empty(MLP_PARAMS, np.float32)
        loss = C.c_float()
        _check(load().dc_mlp_gradient(self.handle, X.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p),
                                      X.shape[0], g.ctypes.data_as(C.c_void_p), C.byref(loss), 0))
        return loss.value, g

    def train(self, X, T, batch=4096, epochs=1, lr=1e-3):
        """Minibatch Adam over X, T in the given order; returns the final loss on all of X."""
        X = np.ascontiguousarray(X, np.float32)
        T = np.ascontiguousarray(T, np.float32)
        loss = C.c_float()
        _check(load().dc_mlp_train(self.handle, X.ctypes.data_as(C.c_void_p), T.ctypes.data_as(C.c_void_p),
                                   X.shape[0], batch, epochs, lr, C.byref(loss), 0))
        return loss.value


def dc_mlp_predict(params, X, stream=None):
    """BF16 tensor-core inference of the network (the dose path's arithmetic): [n, 48] -> [n, 3]."""
    p = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    Y = np.empty((X.shape[0], 3), np.float32)
    s = _current_stream() if stream is None else stream
    _check(load().dc_mlp_predict(p.ctypes.data_as(C.c_void_p), X.ctypes.data_as(C.c_void_p), X.shape[0],
                                 Y.ctypes.data_as(C.c_void_p), 0, C.c_void_p(s)))
    return Y


def dc_fspb_launch_count() -> int:
    n = C.c_uint64()
    _check(load().dc_fspb_launch_count(C.byref(n)))
    return n.value


def dc_fspb_destroy(plan: Plan):
    if plan.handle:
        _check(load().dc_fspb_destroy(plan.handle))
        plan.handle = None


def dc_fspb_dose(plan: Plan, fluence, dose=None):
    """Eq. (1) into `dose` ([V] float32; allocated on the host if None)."""
    if dose is None:
        dose = np.empty(plan.shape, np.float32)
    pf, f1 = _ptr(fluence)
    pd, f2 = _ptr(dose)
    if fluence.shape[-1] != plan.n_beamlets or int(np.prod(dose.shape)) != plan.n_voxels:
        raise ValueError("fluence must have B entries and dose V entries")
    _check(load().dc_fspb_dose(plan.handle, pf, pd, _same_kind(f1, f2)))
    return dose


def dc_fspb_dose_batch(plan: Plan, fluence, dose=None):
    """Eq. (1) for k fluence vectors: fluence [k, B] -> dose [k, V]."""
    k = fluence.shape[0]
    if dose is None:
        dose = np.empty((k,) + tuple(plan.shape), np.float32)
    pf, f1 = _ptr(fluence)
    pd, f2 = _ptr(dose)
    _check(load().dc_fspb_dose_batch(plan.handle, pf, k, pd, _same_kind(f1, f2)))
    return dose


def dc_fspb_pair_count(plan: Plan) -> int:
    n = C.c_int64()
    _check(load().dc_fspb_pair_count(plan.handle, C.byref(n)))
    return n.value


def dc_fspb_dose_matrix(plan: Plan, value_dtype=DC_F32, rowptr=None, cols=None, vals=None):
    """CSR (rowptr int64 [V+1], cols int32 [nnz], vals float32 or bf16 bits) of M[v, i] = D_i(r_v)."""
    nnz = dc_fspb_pair_count(plan)
    if rowptr is None:
        rowptr = np.empty(plan.n_voxels + 1, np.int64)
        cols = np.empty(max(nnz, 1), np.int32)
        vals = np.empty(max(nnz, 1), np.float32 if value_dtype == DC_F32 else np.uint16)
    pr, f1 = _ptr(rowptr, np.int64)
    pc, f2 = _ptr(cols, np.int32)
    pv, f3 = _ptr(vals, vals.dtype if not _is_torch(vals) else None)
    _check(load().dc_fspb_dose_matrix(plan.handle, value_dtype, pr, pc, pv, _same_kind(f1, f2, f3)))
    return rowptr, cols[:nnz] if not _is_torch(cols) else cols, vals[:nnz] if not _is_torch(vals) else vals


def dc_fspb_dose_and_matrix(plan: Plan, fluence, dose=None, value_dtype=DC_F32, rowptr=None, cols=None,
                            vals=None):
    """Dose for `fluence` and the CSR matrix from one pass; returns (dose, rowptr, cols, vals)."""
    nnz = dc_fspb_pair_count(plan)
    if rowptr is None:
        rowptr = np.empty(plan.n_voxels + 1, np.int64)
        cols = np.empty(max(nnz, 1), np.int32)
        vals = np.empty(max(nnz, 1), np.float32 if value_dtype == DC_F32 else np.uint16)
    if dose is None:
        dose = np.empty(plan.shape, np.float32)
    pf, f0 = _ptr(fluence)
    pd, f4 = _ptr(dose)
    pr, f1 = _ptr(rowptr, np.int64)
    pc, f2 = _ptr(cols, np.int32)
    pv, f3 = _ptr(vals, vals.dtype if not _is_torch(vals) else None)
    _check(load().dc_fspb_dose_and_matrix(plan.handle, pf, pd, value_dtype, pr, pc, pv,
                                          _same_kind(f0, f1, f2, f3, f4)))
    trim = lambda a: a[:nnz] if not _is_torch(a) else a
    return dose, rowptr, trim(cols), trim(vals)


def dc_fspb_get_smoothed(plan: Plan):
    out = np.empty(plan.shape, np.float32)
    p, _ = _ptr(out)
    _check(load().dc_fspb_get_smoothed(plan.handle, p, 0))
    return out


def dc_fspb_get_beamlets(plan: Plan):
    rec = np.empty((plan.n_beamlets, 16), np.float32)
    p, _ = _ptr(rec)
    _check(load().dc_fspb_get_beamlets(plan.handle, p))
    return rec


def dc_fspb_get_tables(plan: Plan, i: int, kmax: int = 1 << 16):
    T, W1, W2 = (np.zeros(kmax, np.float32) for _ in range(3))
    K = C.c_int32()
    _check(load().dc_fspb_get_tables(plan.handle, int(i), _ptr(T)[0], _ptr(W1)[0], _ptr(W2)[0],
                                     kmax, C.byref(K)))
    k = min(K.value, kmax)
    return T[:k], W1[:k], W2[:k]


class Batch:
    """Owns a dc_batch*; holds its plans so they outlive it."""

    def __init__(self, handle, plans):
        self.handle = handle
        self.plans = list(plans)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.dc_fspb_batch_destroy(self.handle)
            self.handle = None


def dc_fspb_batch_create(plans, stream=None) -> Batch:
    """One persistent, graph-replayed launch for the doses of several plans."""
    arr = (C.c_void_p * len(plans))(*[p.handle.value if isinstance(p.handle, C.c_void_p) else p.handle
                                      for p in plans])
    h = C.c_void_p()
    s = _current_stream() if stream is None else stream
    _check(load().dc_fspb_batch_create(arr, len(plans), C.c_void_p(s), C.byref(h)))
    return Batch(h, plans)


def dc_fspb_batch_buffers(batch: Batch, i: int):
    """(fluence, dose) device addresses of plan i's batch buffers."""
    f, d = C.c_void_p(), C.c_void_p()
    _check(load().dc_fspb_batch_buffers(batch.handle, int(i), C.byref(f), C.byref(d)))
    return f.value, d.value


def dc_fspb_batch_run(batch: Batch, density=False):
    _check(load().dc_fspb_batch_run(batch.handle, DC_BATCH_DENSITY if density else 0))


def dc_fspb_batch_synchronize(batch: Batch):
    _check(load().dc_fspb_batch_synchronize(batch.handle))


def dc_fspb_batch_kernels(batch: Batch, density=False) -> int:
    n = C.c_int32()
    _check(load().dc_fspb_batch_kernels(batch.handle, DC_BATCH_DENSITY if density else 0, C.byref(n)))
    return n.value


def dc_fspb_batch_autotune(batch: Batch):
    """Picks the batch's form of the pair work by timing (0, 1: the persistent
    kernel for 4 or 5 CTAs per SM; 2: the plans' own launches); returns (variant, ms)."""
    v, ms = C.c_int32(), C.c_float()
    _check(load().dc_fspb_batch_autotune(batch.handle, C.byref(v), C.byref(ms)))
    return v.value, ms.value


def dc_fspb_batch_set_variant(batch: Batch, variant: int):
    """Sets the batch's form of the pair work (0, 1 or 2) without timing."""
    _check(load().dc_fspb_batch_set_variant(batch.handle, int(variant)))


def dc_fspb_batch_dose(batch: Batch, fluences, doses=None, density=False):
    """dose_i of every plan for fluences[i] (host arrays, or CUDA tensors with doses given)."""
    n = len(batch.plans)
    assert len(fluences) == n
    if doses is None:
        doses = [np.empty(p.n_voxels, np.float32) for p in batch.plans]
    fp, dp, flags = [], [], []
    for f, d in zip(fluences, doses):
        a, fa = _ptr(f)
        b, fb = _ptr(d)
        fp.append(a.value)
        dp.append(b.value)
        flags += [fa, fb]
    flag = _same_kind(*flags) | (DC_BATCH_DENSITY if density else 0)
    _check(load().dc_fspb_batch_dose(batch.handle, (C.c_void_p * n)(*fp), (C.c_void_p * n)(*dp), flag))
    return doses


def dc_gamma_index(ref, ev, grid, pct=3.0, dta=0.3, search=None, gamma=None, stream=None):
    """3-D gamma index of the dose ev against the reference dose ref on `grid`
    (pct % of max ref, dta cm, search radius cm, default 5 dta).  Host arrays
    or CUDA tensors [nz, ny, nx]; returns (gamma, statistics dict)."""
    search = 5.0 * dta if search is None else search
    g = dc_grid(grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, grid.ox, grid.oy, grid.oz)
    if gamma is None:
        if _is_torch(ref):
            import torch
            gamma = torch.empty_like(ref)
        else:
            gamma = np.empty(np.shape(ref), np.float32)
    pr, f1 = _ptr(ref)
    pe, f2 = _ptr(ev)
    pg, f3 = _ptr(gamma)
    st = dc_gamma_stats()
    sp = stream if stream is not None else (_current_stream() if f1 else 0)
    _check(load().dc_gamma_index(pr, pe, C.byref(g), pct, dta, search, pg, C.byref(st), C.c_void_p(sp),
                                 _same_kind(f1, f2, f3)))
    return gamma, dict(gamma_max=st.gamma_max, gamma_avg50=st.gamma_avg50, pass50_pct=st.pass50_pct,
                       n50=int(st.n50), dose_max=st.dose_max)


def dc_fluence_from_leaves(plan: Plan, seqs, out=None):
    """The plan's beamlet fluence [B] from one leaf sequence per beam
    (synth.LeafSequence-like objects: edges, mu, left, right, jaws,
    transmission).  out: a host array or a CUDA tensor of B float32 (default:
    a new host array)."""
    if len(seqs) != plan.n_beams:
        raise ValueError("one leaf sequence per beam")
    keep, arr = [], (dc_leaf_sequence * len(seqs))()
    for k, s in enumerate(seqs):
        ed, mu, le, ri = (np.ascontiguousarray(a, np.float32) for a in (s.edges, s.mu, s.left, s.right))
        nl, ncp = ed.size - 1, mu.size
        if le.size != nl * ncp or ri.size != nl * ncp:
            raise ValueError("left/right must be [n_cp][n_leaves]")
        keep += [ed, mu, le, ri]
        x1, x2, y1, y2 = (float(v) for v in s.jaws)
        arr[k] = dc_leaf_sequence(nl, ncp, ed.ctypes.data, mu.ctypes.data, le.ctypes.data, ri.ctypes.data,
                                  x1, x2, y1, y2, float(s.transmission))
    if out is None:
        out = np.empty(plan.n_beamlets, np.float32)
    p, flag = _ptr(out)
    _check(load().dc_fluence_from_leaves(plan.handle, arr, p, flag))
    return out
