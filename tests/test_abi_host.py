"""Host-side checks of the C ABI (no GPU needed, no kernel launched).

The library must load, export every entry point include/dc_fspb.h declares,
and reject malformed arguments with DC_EINVAL before touching the device.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1103_1164_gb300 import build, dc_fspb, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dc_fspb.load()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dc_\w+)\s*\(", text))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "dc_fspb_create" in names and "dc_fspb_dose" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(dc_fspb.EXPORTS) | set(names)


def test_status_strings(lib):
    assert lib.dc_status_str(0) == b"DC_OK"
    assert lib.dc_status_str(1) == b"DC_EINVAL"
    assert lib.dc_status_str(4) == b"DC_ETIMEOUT"


def _create(plan, **over):
    g = plan.grid
    grid = dc_fspb.dc_grid(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.ox, g.oy, g.oz)
    for k, v in over.get("grid", {}).items():
        setattr(grid, k, v)
    beams = (dc_fspb.dc_beam * len(plan.beams))()
    for q, b in enumerate(plan.beams):
        beams[q] = dc_fspb.dc_beam(b.gantry_deg, b.couch_deg, b.coll_deg, b.sad, (C.c_float * 3)(*b.iso),
                                   b.field_x, b.field_y)
    for k, v in over.get("beam", {}).items():
        setattr(beams[0], k, v)
    coeffs, keep = dc_fspb.make_coeffs(plan.comm)
    for k, v in over.get("coeffs", {}).items():
        setattr(coeffs, k, v)
    rho = over.get("rho", plan.rho)
    out = C.c_void_p(123)
    s = dc_fspb.load().dc_fspb_create(rho.ctypes.data_as(C.c_void_p), C.byref(grid), beams,
                                      over.get("n_beams", len(plan.beams)),
                                      over.get("bx", plan.beamlet_x), plan.beamlet_y,
                                      C.byref(coeffs), 0, None, C.byref(out))
    return s, out


@pytest.mark.parametrize("over", [
    dict(grid=dict(nx=0)),
    dict(grid=dict(dx=-0.1)),
    dict(n_beams=0),
    dict(bx=0.0),
    dict(beam=dict(field_x=1.3)),          # not a multiple of the beamlet
    dict(beam=dict(sad=2.0)),              # source inside the grid
    dict(coeffs=dict(a_nt=1)),
    dict(coeffs=dict(w_dt=0.0)),
    dict(coeffs=dict(roi_radius=-1.0)),
    dict(rho="nan"),
    dict(rho="negative"),
])
def test_create_rejects_bad_arguments(lib, over):
    p = synth.small_plan(0)
    if over.get("rho") == "nan":
        r = p.rho.copy(); r[1, 2, 3] = np.nan; over = dict(rho=r)
    elif over.get("rho") == "negative":
        r = p.rho.copy(); r[0, 0, 0] = -0.5; over = dict(rho=r)
    s, out = _create(p, **over)
    assert s == dc_fspb.DC_EINVAL
    assert out.value is None
    assert len(lib.dc_last_error()) > 0


def test_null_arguments(lib):
    assert lib.dc_fspb_dose(None, None, None, 0) == dc_fspb.DC_EINVAL
    assert lib.dc_fspb_n_beamlets(None, None) == dc_fspb.DC_EINVAL
    assert lib.dc_fspb_destroy(None) == dc_fspb.DC_OK


def test_spmm_wrappers_reject_bad_shapes_before_any_call():
    # a plan object with no library handle: the checks must fire before the
    # binding reaches the C entry point
    plan = dc_fspb.Plan(None, 10, 100, (4, 5, 5))
    good_F, good_Y = np.zeros((10, 4), np.float32), np.zeros((100, 4), np.float32)
    for F, Y in [(np.zeros((9, 4), np.float32), good_Y),          # F rows != n_beamlets
                 (np.zeros(10, np.float32), good_Y),              # F not 2-D
                 (good_F, np.zeros((100, 3), np.float32)),         # Y columns != k
                 (good_F, np.zeros((99, 4), np.float32))]:         # Y rows != n_voxels
        with pytest.raises(ValueError):
            dc_fspb.dc_fspb_spmm(plan, F, Y)
        with pytest.raises(ValueError):
            dc_fspb.dc_fspb_spmm_noalloc(plan, F, Y)
    with pytest.raises(ValueError):                                  # host arrays must be float32
        dc_fspb.dc_fspb_spmm(plan, good_F.astype(np.float64), good_Y)
