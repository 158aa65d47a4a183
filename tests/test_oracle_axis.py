"""Pins of the oracle's axis-stencil lateral correction (lateral_mode = 1).

The 48 taps are checked against scipy's trilinear map_coordinates, the
Gaussian-weighted averages against closed forms on linear density fields
(trilinear interpolation is exact there and symmetric weights return the
centre value), and the whole dose against the paper's rho / rho_hat form in
homogeneous media, where both must coincide.
"""
import math

import numpy as np
import pytest
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


# --------------------------------------------------------------------------
# Whole axis-form dose against the independent brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed,kw", [(60, {}), (61, dict(couch=True, n_beams=3)),
                                     (62, dict(couch=True, beamlet=0.2, beamlet_y=0.5, field=2.0)),
                                     (63, dict(phantom="slab", n_beams=3, n=(11, 13, 9), vox=0.4))])
def test_axis_oracle_matches_independent_brute_force(oracle_mod, seed, kw):
    import bruteforce_np as BF
    p = synth.small_plan(seed, **kw)
    got = oracle_mod.OraclePlan(p, lateral_mode=1).dose()
    want = BF.dose(p, lateral_mode=1)
    iso = BF.dose(p, lateral_mode=0)
    assert want.max() > 0.1
    assert np.abs(got - want).max() < 1e-11 * want.max()
    assert np.abs(want - iso).max() > 1e-4 * want.max()   # heterogeneous: the forms differ


# --------------------------------------------------------------------------
# Closed forms for densities that vary along one beam axis only
# --------------------------------------------------------------------------

def _one_axis_plan(profile_axis, gantry, n=24, vox=0.25, seed=5, comm=None, field=0.5, roi=2.5):
    """Density varying along one grid axis only (values in [0.2, 1.8]); one beam."""
    g = synth.centred_grid(n, n, n, vox)
    prof = np.random.default_rng(seed).uniform(0.2, 1.8, n)
    shape = [1, 1, 1]
    shape[{"x": 2, "y": 1, "z": 0}[profile_axis]] = n
    rho = np.broadcast_to(prof.reshape(shape), g.shape).astype(np.float32).copy()
    cm = comm if comm is not None else synth.make_commissioning(roi_radius=roi)
    beam = synth.Beam(gantry, 100.0, (0.0, 0.0, 0.0), field, field)
    plan = synth.Plan("axis1d", g, rho, [beam], 0.5, 0.5, cm, np.ones(1, np.float32))
    return plan, prof.astype(np.float32).astype(float)


def _gauss_avg_1d(coord, prof_coords, prof, d, sigma):
    """Gaussian-weighted average of the linearly interpolated 1-D profile
    (end values held) at the 16 taps coord + (j - 7.5) d."""
    s = (np.arange(16) - 7.5) * d
    w = np.exp(-s * s / (2 * sigma * sigma))
    return float((w * np.interp(coord + s, prof_coords, prof)).sum() / w.sum())


@pytest.mark.parametrize("profile_axis,gantry,moving", [("x", 0.0, 1), ("z", 0.0, 2), ("y", 90.0, 1)])
def test_one_axis_density_moves_one_average(oracle_mod, profile_axis, gantry, moving):
    # At gantry 0 the beam's axes are e_x' = +x, e_y' = +z, e_z' = +y; at 90
    # e_x' = +y.  A density that varies only along the grid axis that is e_x'
    # (or e_y') leaves the other two axis averages at the voxel's own density
    # (their taps stay on the voxel's line of constant density) and moves
    # only that axis's average, which is the 1-D interpolated profile averaged
    # with the Gaussian weights.
    plan, prof = _one_axis_plan(profile_axis, gantry)
    op = oracle_mod.OraclePlan(plan, lateral_mode=1)
    g = plan.grid
    ax = {"x": 0, "y": 1, "z": 2}[profile_axis]
    coords = g.centres()[ax]
    rng = np.random.default_rng(9)
    for _ in range(40):
        i, j, k = (int(q) for q in rng.integers(0, g.nx, 3))
        v = (k * g.ny + j) * g.nx + i
        own = prof[(i, j, k)[ax]]
        avg = _gauss_avg_1d(coords[(i, j, k)[ax]], coords, prof, op.d, plan.comm.smooth_sigma)
        _, _, eff = op.axis_stencil(v, 0)
        want = [own, own, own]
        want[moving] = avg
        want[0] = (avg + 2 * own) / 3.0
        assert np.allclose(eff, want, rtol=0, atol=1e-12), (eff, want)


@pytest.mark.parametrize("profile_axis", ["x", "z"])
def test_axis_dose_profiles_take_their_own_axis_average(oracle_mod, profile_axis):
    # One beamlet on the beam axis (gantry 0: it runs along +y, its lateral
    # axes are e_x'' = +x and e_y'' = +z).  With f_u1 = f_omega = 1, b = 0 and
    # omega_1^w = 0, eq. (3) is omega_2 p(x; u_2x) p(y; u_2y) and every factor
    # but the two profiles is the same for all voxels of one depth plane.  For
    # a density varying along x only, u_2x = f_u2(e_x' average) u_2^w and
    # u_2y = f_u2(rho(r)) u_2^w (the e_y' taps stay at the voxel's density);
    # for a density varying along z only, the roles swap.  The dose in a
    # depth plane, divided by its value at a reference voxel, must equal the
    # ratio of the printed eq. (4) profiles with those widths.
    import bruteforce_np as BF
    base = synth.make_commissioning(roi_radius=2.5)
    dens = base.dens.copy()
    dens[0] = 1.0          # f_u1
    dens[2] = 1.0          # f_omega1
    dens[3] = 1.0          # f_omega2
    dens[4] = 0.0          # b_1
    dens[5] = 0.0          # b_2
    water = base.water.copy()
    water[2] = 0.0         # omega_1^w
    water[3] = 1.0         # omega_2^w
    cm = synth.Commissioning(base.A, base.a_dt, base.a_dtheta, water, base.w_dt, dens, base.f_rho0,
                             base.f_drho, roi_radius=2.5, smooth_sigma=base.smooth_sigma)
    plan, prof = _one_axis_plan(profile_axis, 0.0, comm=cm)
    op = oracle_mod.OraclePlan(plan, lateral_mode=1)
    g = plan.grid
    xs, ys, zs = g.centres()
    rho_dom = cm.f_rho0 + cm.f_drho * np.arange(dens.shape[1])
    fu2 = lambda r: float(np.interp(r, rho_dom, dens[1].astype(float)))
    tw = cm.w_dt * np.arange(water.shape[1])
    x0 = y0 = 0.25
    checked = 0
    for j in (6, 12, 18):                       # depth planes (y index)
        ref = None
        for i in range(4, 20, 3):
            for k in range(4, 20, 3):
                v = (k * g.ny + j) * g.nx + i
                pr = op.pair(v, 0)
                if not pr["inside"] or pr["amb"]:
                    continue
                u2w = float(np.interp(pr["t"], tw, water[1].astype(float)))
                if profile_axis == "x":
                    own = prof[i]
                    avg = _gauss_avg_1d(xs[i], xs, prof, op.d, cm.smooth_sigma)
                    u2x, u2y = fu2(avg) * u2w, fu2(own) * u2w
                else:
                    own = prof[k]
                    avg = _gauss_avg_1d(zs[k], zs, prof, op.d, cm.smooth_sigma)
                    u2x, u2y = fu2(own) * u2w, fu2(avg) * u2w
                shape = float(BF.p_paper(pr["x"], u2x, x0)) * float(BF.p_paper(pr["y"], u2y, y0))
                if ref is None:
                    ref = pr["D"] / shape
                    continue
                assert abs(pr["D"] - ref * shape) < 1e-11 * abs(ref), (i, j, k)
                checked += 1
    assert checked > 40
