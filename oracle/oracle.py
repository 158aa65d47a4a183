"""Python front end of the FP64 CPU oracle (oracle.c) for DC-FSPB.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this module; the product path never does.
It shares no code with the CUDA path: inputs come from the seeded generators in
``paper_1103_1164_gb300.synth`` as plain arrays, are widened to float64, and are
handed to the C oracle, which restates Algorithm A1 and eqs. (1)-(4) of the
paper in double precision.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c and fluence.c with gcc (-O2, OpenMP, IEEE double: no fast-math)."""
    srcs = [os.path.join(_HERE, n) for n in ("oracle.c", "fluence.c")]
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in srcs)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-D_DEFAULT_SOURCE", "-o", tmp, *srcs, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OInputs(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("n_beams", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double),
                ("rho", C.c_void_p), ("beams", C.c_void_p),
                ("bx", C.c_double), ("by", C.c_double),
                ("A", C.c_void_p), ("a_nt", C.c_int32), ("a_nth", C.c_int32),
                ("a_dt", C.c_double), ("a_dth", C.c_double),
                ("water", C.c_void_p), ("w_n", C.c_int32), ("f_n", C.c_int32),
                ("w_dt", C.c_double),
                ("dens", C.c_void_p), ("f_rho0", C.c_double), ("f_drho", C.c_double),
                ("roi", C.c_double), ("sigma", C.c_double), ("rho_surf", C.c_double),
                ("density_correction", C.c_int32), ("lateral_mode", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        vp, i32, i64, d = C.c_void_p, C.c_int, C.c_int64, C.c_double
        L.or_plan_create.restype = vp
        L.or_plan_create.argtypes = [C.POINTER(OInputs), i32]
        L.or_plan_destroy.argtypes = [vp]
        L.or_plan_n_beamlets.argtypes = [vp]
        L.or_plan_step.argtypes = [vp]
        L.or_plan_step.restype = d
        L.or_plan_smoothed.argtypes = [vp, vp]
        L.or_plan_beamlet.argtypes = [vp, i32, vp]
        L.or_plan_table.argtypes = [vp, i32, vp, vp, vp, i32]
        L.or_plan_dose.argtypes = [vp, vp, vp, vp, i32]
        L.or_plan_dose_voxels.argtypes = [vp, vp, vp, i64, vp, vp, i32]
        L.or_plan_pair.argtypes = [vp, i64, i32, vp]
        L.or_plan_matrix_count.argtypes = [vp, vp, i64, vp, i32]
        L.or_plan_pairs_voxels.argtypes = [vp, vp, i64, vp, i32]
        L.or_plan_axis_stencil.argtypes = [vp, i64, i32, vp, vp, vp]
        L.or_plan_matrix_fill.argtypes = [vp, vp, i64, vp, vp, vp, vp, i32]
        L.or_trace_ray.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i32]
        L.or_smooth.argtypes = [vp, i32, i32, i32, d, d, d, d, vp, i32]
        L.or_p.restype = d
        L.or_p.argtypes = [d, d, d]
        L.or_lut1.restype = d
        L.or_lut1.argtypes = [vp, i32, d, d, d]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())


def p_profile(x, u, x0) -> float:
    """Eq. (4) in the oracle's form (scalar)."""
    return lib().or_p(float(x), float(u), float(x0))


def smooth(rho, grid, sigma, threads=None) -> np.ndarray:
    r = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.empty_like(r)
    lib().or_smooth(_p(r), grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, float(sigma),
                    _p(out), threads or default_threads())
    return out


class OraclePlan:
    """FP64 oracle of one plan: ``dose()``, ``matrix()``, per-beamlet tables and pairs."""

    def __init__(self, plan, threads=None, density_correction=None, lateral_mode=0):
        g, cm = plan.grid, plan.comm
        self.plan = plan
        self.threads = threads or default_threads()
        self._keep = []

        def d64(a):
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            self._keep.append(a)
            return a

        beams = np.zeros((len(plan.beams), 10))
        for b, bm in enumerate(plan.beams):
            beams[b, :9] = [bm.gantry_deg, bm.couch_deg, bm.coll_deg, bm.sad, *bm.iso,
                            bm.field_x, bm.field_y]
        dc = cm.density_correction if density_correction is None else density_correction
        ins = OInputs(g.nx, g.ny, g.nz, len(plan.beams), g.dx, g.dy, g.dz, g.ox, g.oy, g.oz,
                      _p(d64(plan.rho)).value, _p(d64(beams)).value,
                      plan.beamlet_x, plan.beamlet_y,
                      _p(d64(cm.A)).value, cm.A.shape[1], cm.A.shape[0], cm.a_dt, cm.a_dtheta,
                      _p(d64(cm.water)).value, cm.water.shape[1], cm.dens.shape[1], cm.w_dt,
                      _p(d64(cm.dens)).value, cm.f_rho0, cm.f_drho,
                      cm.roi_radius, cm.smooth_sigma, cm.rho_surface, int(dc), int(lateral_mode))
        self.grid = g
        self.V = g.n_voxels
        self._h = lib().or_plan_create(C.byref(ins), self.threads)
        self._keep = []
        self.B = lib().or_plan_n_beamlets(self._h)
        self.d = lib().or_plan_step(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_plan_destroy(h)
            self._h = None

    # -- per-plan and per-beamlet state ---------------------------------
    def smoothed(self) -> np.ndarray:
        out = np.empty(self.grid.shape, np.float64)
        lib().or_plan_smoothed(self._h, _p(out))
        return out

    def beamlet(self, i):
        rec = np.empty(17)
        lib().or_plan_beamlet(self._h, int(i), _p(rec))
        return dict(n=rec[0:3].copy(), ex=rec[3:6].copy(), ey=rec[6:9].copy(), theta=rec[9],
                    hit=int(rec[10]), L_in=rec[11], L_out=rec[12], K=int(rec[13]),
                    src=rec[14:17].copy())

    def table(self, i):
        K = self.beamlet(i)["K"]
        T, W1, W2 = (np.zeros(max(K, 1)) for _ in range(3))
        lib().or_plan_table(self._h, int(i), _p(T), _p(W1), _p(W2), K)
        return T[:K], W1[:K], W2[:K]

    def trace_ray(self, src, direction, kmax=100000):
        s = np.ascontiguousarray(src, np.float64)
        n = np.ascontiguousarray(direction, np.float64)
        n = n / np.linalg.norm(n)
        lin, lout = C.c_double(), C.c_double()
        T, W1, W2 = (np.zeros(kmax) for _ in range(3))
        K = lib().or_trace_ray(self._h, _p(s), _p(n), C.byref(lin), C.byref(lout),
                               _p(T), _p(W1), _p(W2), kmax)
        return dict(hit=K > 0, L_in=lin.value, L_out=lout.value, T=T[:K], W1=W1[:K], W2=W2[:K])

    # -- eq. (1) ------------------------------------------------------------
    def dose(self, fluence=None, with_amb=False):
        f = np.ascontiguousarray(self.plan.fluence if fluence is None else fluence, np.float64)
        assert f.shape == (self.B,)
        dose = np.empty(self.V)
        amb = np.empty(self.V) if with_amb else None
        lib().or_plan_dose(self._h, _p(f), _p(dose), _p(amb) if with_amb else None, self.threads)
        dose = dose.reshape(self.grid.shape)
        return (dose, amb.reshape(self.grid.shape)) if with_amb else dose

    def dose_voxels(self, voxels, fluence=None, with_amb=False):
        f = np.ascontiguousarray(self.plan.fluence if fluence is None else fluence, np.float64)
        v = np.ascontiguousarray(voxels, np.int64)
        dose = np.empty(v.size)
        amb = np.empty(v.size)
        lib().or_plan_dose_voxels(self._h, _p(f), _p(v), v.size, _p(dose), _p(amb), self.threads)
        return (dose, amb) if with_amb else dose

    def pairs_voxels(self, voxels):
        """Number of (voxel, beamlet) pairs eq. (1) sums at each listed voxel."""
        v = np.ascontiguousarray(voxels, np.int64)
        out = np.empty(v.size, np.int64)
        lib().or_plan_pairs_voxels(self._h, _p(v), v.size, _p(out), self.threads)
        return out

    def axis_stencil(self, v, beam):
        """(48 trilinear taps, 48 nearest-voxel taps, (rho_omega, rho_x, rho_y)) of voxel v, beam b."""
        taps, near, eff = np.empty(48), np.empty(48), np.empty(3)
        lib().or_plan_axis_stencil(self._h, int(v), int(beam), _p(taps), _p(near), _p(eff))
        return taps, near, eff

    def pair(self, v, i):
        out = np.zeros(9)
        lib().or_plan_pair(self._h, int(v), int(i), _p(out))
        return dict(D=out[0], inside=bool(out[1]), amb=bool(out[2]), x=out[3], y=out[4],
                    t=out[5], teq=out[6], L=out[7], q2=out[8])

    def matrix(self, voxels=None):
        """CSR of candidate entries (rowptr, cols, vals, flags), rows = all voxels
        or the listed ones; flags bit0 = inside ROI and depth range, bit1 =
        decision within rounding margin."""
        v = None if voxels is None else np.ascontiguousarray(voxels, np.int64)
        n = self.V if v is None else v.size
        pv = None if v is None else _p(v)
        counts = np.empty(n, np.int64)
        lib().or_plan_matrix_count(self._h, pv, n, _p(counts), self.threads)
        rowptr = np.zeros(n + 1, np.int64)
        np.cumsum(counts, out=rowptr[1:])
        nnz = int(rowptr[-1])
        cols = np.empty(max(nnz, 1), np.int32)
        vals = np.empty(max(nnz, 1), np.float64)
        flags = np.empty(max(nnz, 1), np.uint8)
        lib().or_plan_matrix_fill(self._h, pv, n, _p(rowptr), _p(cols), _p(vals), _p(flags),
                                  self.threads)
        return rowptr, cols[:nnz], vals[:nnz], flags[:nnz]
