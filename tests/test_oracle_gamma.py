"""Pins of the FP64 gamma-index oracle (oracle/gamma.py) against closed forms,
invariants and an independent nearest-neighbour search."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import gamma as og

SP = (0.25, 0.25, 0.25)


def test_identical_distributions_give_zero():
    rng = np.random.default_rng(1)
    d = rng.uniform(0, 2, (8, 9, 10))
    assert np.all(og.gamma_index(d, d, SP) == 0.0)


@pytest.mark.parametrize("s", [0.01, 0.03, 0.06, 0.5])
def test_uniform_dose_offset(s):
    # constant fields: every candidate has the same dose difference, so the
    # voxel itself is best: gamma = |s| c / (3 % of c), capped at R / dta = 5
    ref = np.full((6, 7, 8), 2.0)
    g = og.gamma_index(ref, ref * (1 + s), SP)
    assert np.allclose(g, min(5.0, s / 0.03), rtol=1e-12)


def test_translated_gradient_closed_form():
    # D_ref = g x on x in [0, 10] cm with g = dD / dta (dD = 3 % of 10 g);
    # D_eval = D_ref shifted by two voxels.  Along x the squared gamma is
    # (o dx / dta)^2 + (g (o - 2) dx / dD)^2 = (dx/dta)^2 (o^2 + (o - 2)^2),
    # least at o = 1: gamma = sqrt(2) dx / dta for voxels whose neighbours at
    # o = 0..2 exist.
    nx = 41
    x = 0.25 * np.arange(nx)
    gslope = 1.0
    ref = np.broadcast_to(gslope * x, (3, 3, nx)).copy()
    ev = np.broadcast_to(gslope * (x - 0.5), (3, 3, nx)).copy()
    g = og.gamma_index(ref, ev, SP)
    want = np.sqrt(2.0) * 0.25 / 0.3
    assert np.allclose(g[:, :, 2:nx - 2], want, rtol=1e-12)


def test_scale_invariance():
    rng = np.random.default_rng(2)
    ref = rng.uniform(0, 1, (6, 6, 6))
    ev = ref + rng.normal(0, 0.02, ref.shape)
    assert np.allclose(og.gamma_index(ref, ev, SP), og.gamma_index(7.5 * ref, 7.5 * ev, SP), rtol=1e-12)


def test_against_4d_nearest_neighbour():
    # gamma is the distance to the nearest evaluated point in the space
    # (x / dta, y / dta, z / dta, D / dD), capped at R / dta (points outside
    # the search sphere are farther than the cap in that space)
    rng = np.random.default_rng(3)
    shape = (7, 8, 9)
    z, y, x = np.meshgrid(*(0.25 * np.arange(n) for n in shape), indexing="ij")
    ref = np.exp(-((x - 1.0) ** 2 + (y - 0.8) ** 2) / 0.5) + 0.05 * z
    ev = 1.04 * np.roll(ref, 1, axis=2) + rng.normal(0, 0.01, shape)
    dta, pct, R = 0.3, 3.0, 0.9
    dD = pct / 100 * ref.max()
    pts = np.stack([x.ravel() / dta, y.ravel() / dta, z.ravel() / dta, ev.ravel() / dD], 1)
    q = np.stack([x.ravel() / dta, y.ravel() / dta, z.ravel() / dta, ref.ravel() / dD], 1)
    dist, _ = cKDTree(pts).query(q)
    want = np.minimum(dist, R / dta).reshape(shape)
    got = og.gamma_index(ref, ev, SP, pct=pct, dta=dta, radius=R)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-12)


def test_stats_definitions():
    ref = np.zeros((1, 1, 10))
    ref[0, 0, :] = np.arange(10)                        # max 9: voxels >= 4.5 are 5..9
    g = np.array([[[0.1, 0.2, 0.3, 0.4, 0.5, 0.5, 1.5, 0.7, 2.0, 0.9]]])
    gmax, gavg, p50, n50 = og.gamma_stats(g, ref)
    assert gmax == 2.0 and n50 == 5
    assert gavg == pytest.approx((0.5 + 1.5 + 0.7 + 2.0 + 0.9) / 5)
    assert p50 == pytest.approx(60.0)


def test_gamma_at_matches_full_grid():
    rng = np.random.default_rng(4)
    ref = rng.uniform(0, 1, (5, 6, 7))
    ev = ref + rng.normal(0, 0.05, ref.shape)
    full = og.gamma_index(ref, ev, (0.2, 0.25, 0.3), pct=2.0, dta=0.25, radius=0.8)
    vox = rng.choice(ref.size, 40, replace=False)
    got = og.gamma_at(ref, ev, (0.2, 0.25, 0.3), vox, pct=2.0, dta=0.25, radius=0.8)
    assert np.allclose(got, full.ravel()[vox], rtol=1e-13)
