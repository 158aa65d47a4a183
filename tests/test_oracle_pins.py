"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

No test here compares the oracle with itself: each checks it against a closed
form, an invariant of eqs. (1)-(4), a library routine, or an independent
brute-force restatement (tests/bruteforce_np.py) that computes every step by a
different route.  The paper prints no worked numeric example, so no stored
value comes from it.
"""
import math

import numpy as np
import pytest
from scipy import integrate, ndimage

import bruteforce_np as BF
from paper_1103_1164_gb300 import synth


# --------------------------------------------------------------------------
# Eq. (4): the penumbra profile p(x, u, x0)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("u,x0", [(0.3, 0.25), (2.0, 0.1), (7.5, 0.25), (0.5, 1.0)])
def test_p_integrates_to_beamlet_width(oracle_mod, u, x0):
    # p is a unit box of half-width x0 convolved with the Laplace density
    # (u/2) exp(-u|x|), so its integral is 2 x0 for every u.
    f = lambda x: oracle_mod.p_profile(x, u, x0)
    lim = x0 + 60.0 / u
    val = sum(integrate.quad(f, a, b, epsabs=1e-13, epsrel=1e-13, limit=200)[0]
              for a, b in ((-lim, -x0), (-x0, x0), (x0, lim)))
    assert abs(val - 2 * x0) < 1e-9


@pytest.mark.parametrize("u,x0", [(0.3, 0.25), (4.0, 0.1), (8.0, 0.5)])
def test_p_partition_of_unity_and_continuity(oracle_mod, u, x0):
    # Shifted boxes of width 2 x0 tile the line, so their Laplace-blurred
    # profiles sum to one everywhere.
    for x in np.linspace(-0.7, 0.9, 17):
        s = sum(oracle_mod.p_profile(x - 2 * k * x0, u, x0) for k in range(-4000, 4001))
        assert abs(s - 1.0) < 1e-9
    # continuity at |x| = x0 (the two branches of eq. (4) meet)
    for sgn in (-1, 1):
        a = oracle_mod.p_profile(sgn * x0 * (1 - 1e-12), u, x0)
        b = oracle_mod.p_profile(sgn * x0 * (1 + 1e-12), u, x0)
        assert abs(a - b) < 1e-9


def test_p_matches_printed_form_and_box_limit(oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(2000):
        x, u, x0 = rng.uniform(-6, 6), rng.uniform(0.05, 9), rng.uniform(0.05, 0.6)
        assert abs(oracle_mod.p_profile(x, u, x0) - float(BF.p_paper(x, u, x0))) < 1e-12
    # u -> infinity: the box indicator of [-x0, x0]
    assert abs(oracle_mod.p_profile(0.1, 1e4, 0.25) - 1.0) < 1e-12
    assert oracle_mod.p_profile(0.3, 1e4, 0.25) < 1e-12


# --------------------------------------------------------------------------
# Table lookups (Algorithm A1 steps 9-10)
# --------------------------------------------------------------------------

def test_lut_is_clamped_linear_interpolation(oracle_mod):
    import ctypes as C
    rng = np.random.default_rng(1)
    f = np.ascontiguousarray(rng.uniform(-1, 1, 37))
    x0, h = 0.3, 0.125
    xs = x0 + h * np.arange(37)
    for x in rng.uniform(-1, 6, 500):
        got = oracle_mod.lib().or_lut1(f.ctypes.data_as(C.c_void_p), 37, x0, h, float(x))
        assert abs(got - np.interp(x, xs, f)) < 1e-13


# --------------------------------------------------------------------------
# Step 1: smoothed density
# --------------------------------------------------------------------------

def test_smoothing_matches_library_gaussian_filter(oracle_mod):
    g = synth.centred_grid(14, 11, 9, 0.25, 0.3, 0.4)
    rng = np.random.default_rng(2)
    rho = rng.uniform(0.0, 2.0, g.shape)
    sigma = 0.5
    got = oracle_mod.smooth(rho, g, sigma)
    radius = [int(math.ceil(3 * sigma / d)) for d in (g.dz, g.dy, g.dx)]
    ref = ndimage.gaussian_filter(rho, sigma=[sigma / g.dz, sigma / g.dy, sigma / g.dx],
                                  mode="nearest", radius=radius)
    assert np.abs(got - ref).max() < 1e-13
    # constant density is a fixed point; sigma = 0 is the identity
    assert np.abs(oracle_mod.smooth(np.full(g.shape, 0.7), g, sigma) - 0.7).max() < 1e-14
    assert np.array_equal(oracle_mod.smooth(rho, g, 0.0), rho)


# --------------------------------------------------------------------------
# Steps 4-6: entry/exit and radiological-depth / omega_corr tables
# --------------------------------------------------------------------------

def test_slab_radiological_depth_is_exact_piecewise_linear(oracle_mod):
    p = synth.config1()
    op = oracle_mod.OraclePlan(p)
    tr = op.trace_ray([0.1, -100.0, 0.1], [0.0, 1.0, 0.0])
    # entry face of the 16 cm phantom is at y = -8, exit at y = +8
    assert abs(tr["L_in"] - 92.0) < 1e-12 and abs(tr["L_out"] - 108.0) < 1e-12
    d = op.d
    assert d == 0.125
    t = d * np.arange(len(tr["T"]))
    exact = np.where(t < 5, t, np.where(t < 10, 5 + 0.25 * (t - 5), 6.25 + (t - 10)))
    exact = np.where(t <= 16, exact, 12.25)   # nothing beyond the grid
    assert np.abs(tr["T"] - exact).max() < 1e-12
    # omega_2^corr: b_2(1) = 0 in water, b_2(0.25) in the slab (library interp of the table)
    cm = p.comm
    rho_dom = cm.f_rho0 + cm.f_drho * np.arange(cm.dens.shape[1])
    b2s = np.interp(0.25, rho_dom, cm.dens[5].astype(float))
    b2w = np.interp(1.0, rho_dom, cm.dens[5].astype(float))
    seg_slab = np.clip(np.minimum(t, 10) - 5, 0, None)
    seg_water = np.minimum(t, 5) + np.clip(np.minimum(t, 16) - 10, 0, None)
    assert np.abs(tr["W2"] - (b2s * seg_slab + b2w * seg_water)).max() < 1e-12


def test_oblique_ray_matches_riemann_sum(oracle_mod):
    p = synth.small_plan(5, n=(16, 14, 12), vox=0.4)
    op = oracle_mod.OraclePlan(p)
    g = p.grid
    src = np.array([-40.0, -70.0, 17.0])
    n = np.array([0.45, 0.8, -0.2])
    n /= np.linalg.norm(n)
    tr = op.trace_ray(src, n)
    assert tr["hit"]
    # midpoint Riemann sum with step h: error <= h * (number of voxel crossings) * max rho
    h = 2e-6
    L = d = op.d
    K = len(tr["T"])
    a = tr["L_in"] + h * (np.arange(int((K - 1) * d / h)) + 0.5)
    pos = src[None, :] + a[:, None] * n[None, :]
    idx = np.floor((pos - np.array([g.ox, g.oy, g.oz]) + 0.5 * np.array([g.dx, g.dy, g.dz]))
                   / np.array([g.dx, g.dy, g.dz])).astype(int)
    inside = np.all((idx >= 0) & (idx < np.array([g.nx, g.ny, g.nz])), 1)
    rho = np.zeros(a.size)
    rho[inside] = p.rho[idx[inside, 2], idx[inside, 1], idx[inside, 0]]
    cum = np.concatenate([[0.0], np.cumsum(rho) * h])
    ks = np.arange(K)
    riemann = cum[np.minimum((ks * d / h).round().astype(int), a.size)]
    bound = h * (g.nx + g.ny + g.nz) * 2.0 + 1e-9
    assert np.abs(tr["T"] - riemann).max() < bound
    # the voxel-box brute force gives the same exact samples
    bf = BF.tables(p, g, p.rho, src, n, d)
    assert abs(bf["L_in"] - tr["L_in"]) < 1e-12 and abs(bf["L_out"] - tr["L_out"]) < 1e-12
    assert np.abs(bf["T"] - tr["T"]).max() < 1e-11
    assert np.abs(bf["W1"] - tr["W1"]).max() < 1e-11
    assert np.abs(bf["W2"] - tr["W2"]).max() < 1e-11


# --------------------------------------------------------------------------
# Steps 2-3: beam and beamlet geometry
# --------------------------------------------------------------------------

def test_beam_geometry_closed_forms(oracle_mod):
    p = synth.config1()
    p.beams = [synth.Beam(90.0, 100.0, (0.0, 0.0, 0.0), 10.0, 10.0)]
    p.fluence = np.ones(p.n_beamlets, np.float32)
    op = oracle_mod.OraclePlan(p)
    # gantry 90: source on +x, beam travels -x
    b = op.beamlet(0)
    assert np.allclose(b["src"], [100.0, 0.0, 0.0], atol=1e-12)
    for i in range(op.B):
        b = op.beamlet(i)
        m, n = i % 20, i // 20
        a, c = -5 + (m + 0.5) * 0.5, -5 + (n + 0.5) * 0.5
        target = np.array([0.0, 0.0, 0.0]) + a * np.array([0.0, 1.0, 0.0]) + c * np.array([0, 0, 1.0])
        want = (target - b["src"]) / np.linalg.norm(target - b["src"])
        assert np.allclose(b["n"], want, atol=1e-14)
        assert abs(b["theta"] - math.atan(math.hypot(a, c) / 100.0)) < 1e-14
        F = np.stack([b["ex"], b["ey"], b["n"]])
        assert np.allclose(F @ F.T, np.eye(3), atol=1e-14)
        assert np.allclose(np.cross(b["ex"], b["n"]), b["ey"], atol=1e-14) and b["ey"][2] > 0


# --------------------------------------------------------------------------
# Eq. (2): inverse square and the lateral kernel on the beamlet axis
# --------------------------------------------------------------------------

def _flat_commissioning(roi=1.0, A=0.8, u1=3.0, u2=0.5, w2=0.12):
    cm = synth.make_commissioning(roi_radius=roi)
    cm.A = np.full_like(cm.A, A)
    cm.water = np.stack([np.full(cm.water.shape[1], v, np.float32) for v in (u1, u2, 1 - w2, w2)])
    return cm


def test_inverse_square_on_beamlet_axis(oracle_mod):
    g = synth.centred_grid(9, 21, 9, 0.5)
    cm = _flat_commissioning()
    cm.density_correction = 0
    plan = synth.Plan("axis", g, np.ones(g.shape, np.float32),
                      [synth.Beam(0.0, 100.0, (0.0, 0.0, 0.0), 0.5, 0.5)], 0.5, 0.5, cm,
                      np.ones(1, np.float32))
    op = oracle_mod.OraclePlan(plan)
    dose = op.dose()
    x0 = 0.25
    # the tables hold float32 values
    w1, w2, A = float(np.float32(1 - 0.12)), float(np.float32(0.12)), float(np.float32(0.8))
    F0 = (w1 * (1 - math.exp(-3.0 * x0)) ** 2 + w2 * (1 - math.exp(-0.5 * x0)) ** 2)
    for j in range(21):
        L = 100.0 + (-5.0 + 0.5 * j)
        assert abs(dose[4, j, 4] - F0 * A * (100.0 / L) ** 2) < 1e-13
    # off axis by one voxel in x: x = 0.5 * SAD/L, p from the printed form
    for j in (0, 10, 20):
        L = 100.0 + (-5.0 + 0.5 * j)
        xs = 0.5 * 100.0 / L
        F = (w1 * float(BF.p_paper(xs, 3.0, x0)) * (1 - math.exp(-3.0 * x0))
             + w2 * float(BF.p_paper(xs, 0.5, x0)) * (1 - math.exp(-0.5 * x0)))
        assert abs(dose[4, j, 5] - F * A * (100.0 / L) ** 2) < 1e-13


def test_broad_uniform_field_is_flat(oracle_mod):
    # Partition of unity across beamlets: deep inside a broad uniform field the
    # lateral kernel sums to omega_1 + omega_2 = 1.  Beamlets are made parallel
    # (SAD = 1000 m) and the kernels short (u >= 4/cm) against the ROI (5 cm)
    # and the field half-width (5 cm); every beamlet axis meets the phantom.
    g = synth.centred_grid(23, 5, 23, 0.5)
    cm = _flat_commissioning(roi=5.0, u1=8.0, u2=4.0)
    cm.density_correction = 0
    plan = synth.Plan("flat", g, np.ones(g.shape, np.float32),
                      [synth.Beam(0.0, 1.0e5, (0.0, 0.0, 0.0), 10.0, 10.0)], 0.5, 0.5, cm,
                      np.zeros(0, np.float32))
    plan.fluence = np.ones(plan.n_beamlets, np.float32)
    dose = oracle_mod.OraclePlan(plan).dose()
    y = g.centres()[1]
    isq = (1.0e5 / (1.0e5 + y)) ** 2          # eq. (2)'s inverse square along depth
    assert np.abs(dose[9:14, :, 9:14] / (float(np.float32(0.8)) * isq[None, :, None]) - 1.0).max() < 1e-7


# --------------------------------------------------------------------------
# Eq. (1) and whole-plan invariants
# --------------------------------------------------------------------------

def test_dose_is_linear_in_fluence_and_additive_over_beams(oracle_mod):
    p = synth.small_plan(11, n_beams=3)
    op = oracle_mod.OraclePlan(p)
    rng = np.random.default_rng(3)
    f, h = rng.uniform(0, 1, op.B), rng.uniform(0, 1, op.B)
    a, b = 0.7, 2.3
    lhs = op.dose(a * f + b * h)
    rhs = a * op.dose(f) + b * op.dose(h)
    assert np.abs(lhs - rhs).max() < 1e-12 * max(1.0, np.abs(lhs).max())
    # the plan's dose is the sum of the single-beam plans' doses
    total = np.zeros_like(lhs)
    off = 0
    for bm, nb in zip(p.beams, p.beamlets_per_beam):
        q = synth.Plan("one", p.grid, p.rho, [bm], p.beamlet_x, p.beamlet_y, p.comm,
                       np.asarray(f[off:off + nb], np.float32))
        total += oracle_mod.OraclePlan(q).dose(f[off:off + nb])
        off += nb
    assert np.abs(total - op.dose(f)).max() < 1e-12


def test_homogeneous_water_correction_collapses_to_fspb(oracle_mod):
    # In water rho = rho_hat = 1, f(1) = 1 and b(1) = 0: skipping step 11 must
    # not change the dose (Section 2.1: DC-FSPB degenerates to FSPB).
    p = synth.small_plan(21, phantom="water")
    with_dc = oracle_mod.OraclePlan(p, density_correction=1).dose()
    without = oracle_mod.OraclePlan(p, density_correction=0).dose()
    assert np.abs(with_dc - without).max() < 2e-6 * with_dc.max()
    # and in a heterogeneous phantom it does change it
    q = synth.small_plan(22, phantom="slab")
    a = oracle_mod.OraclePlan(q, density_correction=1).dose()
    b = oracle_mod.OraclePlan(q, density_correction=0).dose()
    assert np.abs(a - b).max() > 1e-3 * a.max()


def test_mirror_symmetry(oracle_mod):
    g = synth.centred_grid(16, 20, 10, 0.25)
    rng = np.random.default_rng(4)
    half = rng.uniform(0.2, 1.8, (g.nz, g.ny, g.nx // 2)).astype(np.float32)
    rho = np.concatenate([half, half[:, :, ::-1]], 2)
    cm = synth.make_commissioning(roi_radius=1.5, smooth_sigma=0.4)
    beam = synth.Beam(0.0, 100.0, (0.0, 0.0, 0.0), 3.0, 2.0)
    plan = synth.Plan("mirror", g, rho, [beam], 0.5, 0.5, cm, np.zeros(0, np.float32))
    fl = rng.uniform(0, 1, (4, 3))
    fl = np.concatenate([fl, fl[:, ::-1]], 1).ravel()   # symmetric in the beamlet column m
    plan.fluence = fl.astype(np.float32)
    dose = oracle_mod.OraclePlan(plan).dose()
    assert dose.max() > 0
    assert np.abs(dose - dose[:, :, ::-1]).max() < 1e-12 * dose.max()


@pytest.mark.parametrize("seed,kw", [(0, {}), (1, dict(couch=True)), (2, dict(density_correction=0)),
                                     (3, dict(beamlet=0.4, beamlet_y=0.6)),
                                     (4, dict(phantom="slab", n_beams=3))])
def test_oracle_matches_independent_brute_force(oracle_mod, seed, kw):
    p = synth.small_plan(seed, **kw)
    got = oracle_mod.OraclePlan(p).dose()
    want = BF.dose(p)
    assert want.max() > 0.1
    assert np.abs(got - want).max() < 1e-11 * want.max()


def test_matrix_rows_reproduce_dose(oracle_mod):
    p = synth.small_plan(7, n_beams=2)
    op = oracle_mod.OraclePlan(p)
    rowptr, cols, vals, flags = op.matrix()
    f = p.fluence.astype(float)
    inside = (flags & 1).astype(bool)
    contrib = np.where(inside, vals * f[cols], 0.0)
    dm = np.add.reduceat(np.concatenate([contrib, [0.0]]), rowptr[:-1]) * (np.diff(rowptr) > 0)
    assert np.abs(dm.reshape(p.grid.shape) - op.dose()).max() < 1e-12
    for v in range(0, op.V, 97):   # columns ascend within each row
        c = cols[rowptr[v]:rowptr[v + 1]]
        assert np.all(np.diff(c) > 0)
