"""Pins of the oracle's axis-stencil lateral correction (lateral_mode = 1).

The 48 taps are checked against scipy's trilinear map_coordinates, the
Gaussian-weighted averages against closed forms on linear density fields
(trilinear interpolation is exact there and symmetric weights return the
centre value), and the whole dose against the paper's rho / rho_hat form in
homogeneous media, where both must coincide.
"""
import math

import numpy as np
from scipy import ndimage

from paper_1103_1164_gb300 import synth


def _axes(beam):
    import bruteforce_np as BF
    return BF.beam_axes(beam)


def test_taps_match_library_trilinear(oracle_mod):
    p = synth.small_plan(41, n=(14, 12, 10), vox=0.3, n_beams=2, couch=True)
    op = oracle_mod.OraclePlan(p, lateral_mode=1)
    g = p.grid
    rng = np.random.default_rng(0)
    for v in rng.integers(0, op.V, 25):
        for b, beam in enumerate(p.beams):
            taps, near, eff = op.axis_stencil(v, b)
            i, j, k = v % g.nx, (v // g.nx) % g.ny, v // (g.nx * g.ny)
            r = np.array([g.ox + i * g.dx, g.oy + j * g.dy, g.oz + k * g.dz])
            want = []
            for ax in _axes(beam)[:2] + (_axes(beam)[2],):
                s = (np.arange(-8, 8) + 0.5) * op.d
                pts = r[None, :] + s[:, None] * ax[None, :]
                idx = (pts - np.array([g.ox, g.oy, g.oz])) / np.array([g.dx, g.dy, g.dz])
                idx = np.clip(idx, 0, np.array([g.nx, g.ny, g.nz]) - 1)
                want.append(ndimage.map_coordinates(p.rho.astype(float), idx[:, ::-1].T, order=1, mode="nearest"))
            want = np.concatenate(want)
            assert np.abs(taps - want).max() < 1e-12
            sig = p.comm.smooth_sigma
            w = np.exp(-((np.arange(-8, 8) + 0.5) * op.d) ** 2 / (2 * sig * sig))
            avg = [(w * want[16 * a:16 * a + 16]).sum() / w.sum() for a in range(3)]
            assert np.allclose(eff, [np.mean(avg), avg[0], avg[1]], rtol=0, atol=1e-12)


def test_linear_density_field_gives_centre_value(oracle_mod):
    g = synth.centred_grid(24, 24, 24, 0.25)
    x, y, z = g.centres()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    rho = (1.0 + 0.05 * X - 0.03 * Y + 0.02 * Z).astype(np.float32)
    cm = synth.make_commissioning(roi_radius=1.0)
    plan = synth.Plan("lin", g, rho, [synth.Beam(37.0, 100.0, (0, 0, 0), 2.0, 2.0, 11.0, 23.0)], 0.5, 0.5,
                      cm, np.ones(16, np.float32))
    op = oracle_mod.OraclePlan(plan, lateral_mode=1)
    # interior voxels: every tap (|s| <= 0.94 cm) stays inside the grid
    for (i, j, k) in [(12, 12, 12), (8, 15, 10), (15, 9, 14)]:
        v = (k * g.ny + j) * g.nx + i
        taps, near, eff = op.axis_stencil(v, 0)
        centre = float(rho[k, j, i])
        # taps are exact samples of the linear field (float32 storage rounding only)
        assert np.allclose(eff, centre, rtol=0, atol=2e-6)


def test_homogeneous_media_axis_equals_paper_form(oracle_mod):
    for val in (1.0, 0.6, 1.7):
        p = synth.small_plan(43, phantom="water", n_beams=2)
        p.rho = np.full_like(p.rho, val)
        a = oracle_mod.OraclePlan(p, lateral_mode=0).dose()
        b = oracle_mod.OraclePlan(p, lateral_mode=1).dose()
        assert a.max() > 0
        assert np.abs(a - b).max() < 1e-12 * a.max()
    q = synth.small_plan(44, phantom="random", n_beams=2)
    a = oracle_mod.OraclePlan(q, lateral_mode=0).dose()
    b = oracle_mod.OraclePlan(q, lateral_mode=1).dose()
    assert np.abs(a - b).max() > 1e-4 * a.max()   # the two forms differ in heterogeneous media
