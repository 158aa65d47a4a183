"""Pins of the FP64 fluence-from-leaf-sequence oracle (Section 2.3 reading:
fluence = meterset-weighted open area of each beamlet / its area).

Closed forms (static fields, jaws, transmission, a uniform sliding sweep),
invariances (splitting a control-point interval, reversing the bank roles of a
static field), and a brute-force Riemann sum in (x, y, meterset).
"""
import numpy as np
import pytest

from paper_1103_1164_gb300 import synth
from oracle import fluence as ofl


def _seq(edges, mu, left, right, jaws, tau=0.0):
    return synth.LeafSequence(np.asarray(edges, np.float64), np.asarray(mu, np.float64),
                              np.asarray(left, np.float64), np.asarray(right, np.float64),
                              tuple(jaws), tau)


def test_open_area_closed_forms():
    # static rectangle inside the strip, outside it, straddling it
    assert ofl.open_area(0.2, 0.7, 0.2, 0.7, 0.0, 3.0, 0.0, 1.0) == pytest.approx(1.5)
    assert ofl.open_area(2.0, 3.0, 2.0, 3.0, 0.0, 3.0, 0.0, 1.0) == 0.0
    assert ofl.open_area(-1.0, 0.5, -1.0, 0.5, 0.0, 2.0, 0.0, 1.0) == pytest.approx(1.0)
    # r = 2 mu over mu in [0, 1], l = 0, strip [0, 1]: int min(2 mu, 1) = 0.75
    assert ofl.open_area(0.0, 0.0, 0.0, 2.0, 0.0, 1.0, 0.0, 1.0) == pytest.approx(0.75)
    # l = mu - 0.5, r = mu + 0.5, strip [0, 1], mu in [0, 1]: open part of the
    # strip is [max(0, mu - .5), min(1, mu + .5)]: length 0.5 + mu then 1.5 - mu
    assert ofl.open_area(-0.5, 0.5, 0.5, 1.5, 0.0, 1.0, 0.0, 1.0) == pytest.approx(0.75)
    # zero-meterset interval
    assert ofl.open_area(0.0, 1.0, 0.0, 1.0, 2.0, 2.0, 0.0, 1.0) == 0.0


def test_static_open_field_and_jaws():
    fx, fy, bx, by = 2.0, 1.5, 0.2, 0.5
    edges = synth.leaf_edges(fy, 0.5)
    nl = len(edges) - 1
    open_ = np.full((2, nl), 10.0)
    s = _seq(edges, [0.0, 50.0], -open_, open_, (-1.0, 1.0, -0.75, 0.75))
    f = ofl.leaf_fluence(s, fx, fy, bx, by).reshape(3, 10)
    assert np.allclose(f, 50.0)
    # jaws: x1 at -0.7 blocks beamlet 0 of every row and half of beamlet 1;
    # y2 at 0.5 blocks half of the top row
    s = _seq(edges, [0.0, 50.0], -open_, open_, (-0.7, 1.0, -0.75, 0.5))
    f = ofl.leaf_fluence(s, fx, fy, bx, by).reshape(3, 10)
    want = np.full((3, 10), 50.0)
    want[:, 0] = 0.0
    want[:, 1] = 25.0
    want[2] *= 0.5
    assert np.allclose(f, want)


def test_closed_leaves_give_transmission_only():
    fx, fy = 1.0, 1.0
    edges = synth.leaf_edges(fy, 0.5)
    nl = len(edges) - 1
    z = np.zeros((2, nl))
    s = _seq(edges, [0.0, 100.0], z, z, (-0.5, 0.5, -0.5, 0.5), tau=0.02)
    f = ofl.leaf_fluence(s, fx, fy, 0.2, 0.5)
    assert np.allclose(f, 2.0)


def test_leaf_pair_straddling_beamlet_rows():
    # 0.5 cm leaves shifted by 0.25 cm against the 0.5 cm beamlet rows: only
    # one leaf pair open (x in [-0.3, 0.5]); the two rows it half covers get
    # half the open fraction
    fx, fy, bx, by = 1.0, 1.0, 0.2, 0.5
    edges = synth.leaf_edges(fy, 0.5, offset=0.25)
    nl = len(edges) - 1
    j = int(np.searchsorted(edges, 0.0)) - 1      # pair covering y in [-0.25, 0.25]
    L = np.zeros((2, nl)); R = np.zeros((2, nl))
    L[:, j], R[:, j] = -0.3, 0.5
    s = _seq(edges, [0.0, 10.0], L, R, (-0.5, 0.5, -0.5, 0.5))
    f = ofl.leaf_fluence(s, fx, fy, bx, by).reshape(2, 5)
    xs = -0.5 + bx * np.arange(5)
    open_frac = np.clip(np.minimum(xs + bx, 0.5) - np.maximum(xs, -0.3), 0, None) / bx
    assert np.allclose(f[0], 10.0 * 0.5 * open_frac)
    assert np.allclose(f[1], 10.0 * 0.5 * open_frac)


@pytest.mark.parametrize("n_cp", [2, 7])
def test_uniform_sliding_sweep_closed_form(n_cp):
    # both tips at constant speed from x_s to x_e with gap g, total meterset T:
    # a point in [x_s + g, x_e] is open for g T / (x_e - x_s)
    xs, xe, g, T = -2.0, 2.0, 0.4, 80.0
    fx, fy = 3.0, 1.0
    edges = synth.leaf_edges(fy, 0.5)
    nl = len(edges) - 1
    mu = np.linspace(0.0, T, n_cp)
    l = xs + (xe - g - xs) * mu / T
    L = np.repeat(l[:, None], nl, 1)
    s = _seq(edges, mu, L, L + g, (-1.5, 1.5, -0.5, 0.5))
    f = ofl.leaf_fluence(s, fx, fy, 0.2, 0.5)
    assert np.allclose(f, g * T / (xe - g - xs))


def test_splitting_an_interval_changes_nothing():
    rng = np.random.default_rng(3)
    s = synth.sliding_window(rng, 3.0, 2.0, n_cp=9, transmission=0.015)
    f0 = ofl.leaf_fluence(s, 3.0, 2.0, 0.2, 0.5)
    # insert the midpoint of every interval (positions interpolated linearly)
    mu = np.asarray(s.mu, np.float64)
    L, R = np.asarray(s.left, np.float64), np.asarray(s.right, np.float64)
    mu2 = np.empty(2 * len(mu) - 1); mu2[0::2] = mu; mu2[1::2] = 0.5 * (mu[:-1] + mu[1:])
    L2 = np.empty((len(mu2), L.shape[1])); L2[0::2] = L; L2[1::2] = 0.5 * (L[:-1] + L[1:])
    R2 = np.empty_like(L2); R2[0::2] = R; R2[1::2] = 0.5 * (R[:-1] + R[1:])
    s2 = _seq(s.edges, mu2, L2, R2, s.jaws, s.transmission)
    assert np.allclose(ofl.leaf_fluence(s2, 3.0, 2.0, 0.2, 0.5), f0, rtol=1e-12, atol=1e-9)


def _riemann(s, fx, fy, bx, by, n=240):
    """Midpoint rule in (x, y, meterset) of the open indicator, per beamlet.
    The y cells are 0.025 cm, so leaf edges and jaws on that lattice fall on
    cell boundaries and the y integral is exact; x and meterset carry the
    discretisation error."""
    M, N = int(round(fx / bx)), int(round(fy / by))
    edges = np.asarray(s.edges, np.float64)
    mu = np.asarray(s.mu, np.float64)
    L, R = np.asarray(s.left, np.float64), np.asarray(s.right, np.float64)
    x1, x2, y1, y2 = s.jaws
    out = np.zeros(M * N)
    for nn in range(N):
        ys = -0.5 * fy + nn * by + by * (np.arange(20) + 0.5) / 20
        for m in range(M):
            xs = -0.5 * fx + m * bx + bx * (np.arange(n) + 0.5) / n
            tot = 0.0
            for c in range(len(mu) - 1):
                dm = mu[c + 1] - mu[c]
                if dm <= 0:
                    continue
                u = (np.arange(n) + 0.5) / n
                for y in ys:
                    if not (y1 <= y <= y2) or y < edges[0] or y >= edges[-1]:
                        continue
                    j = int(np.searchsorted(edges, y, side="right")) - 1
                    l = L[c, j] + (L[c + 1, j] - L[c, j]) * u
                    r = R[c, j] + (R[c + 1, j] - R[c, j]) * u
                    inj = (xs[None, :] >= x1) & (xs[None, :] <= x2)
                    op = (xs[None, :] > l[:, None]) & (xs[None, :] < r[:, None])
                    val = ((1 - s.transmission) * op + s.transmission) * inj
                    tot += val.mean() * dm * (by / 20) * bx
            out[nn * M + m] = tot / (bx * by)
    return out


@pytest.mark.parametrize("kind", ["sliding", "shoot"])
def test_oracle_matches_brute_force(kind):
    rng = np.random.default_rng(11 if kind == "sliding" else 12)
    fx, fy = 1.0, 1.0
    make = synth.sliding_window if kind == "sliding" else synth.step_and_shoot
    kw = dict(n_cp=5) if kind == "sliding" else dict(n_seg=3)
    s = make(rng, fx, fy, transmission=0.02, jaw_margin=-0.05, offset=0.1, **kw)
    f = ofl.leaf_fluence(s, fx, fy, 0.2, 0.5)
    b = _riemann(s, fx, fy, 0.2, 0.5)
    mu_total = float(s.mu[-1])
    assert np.abs(f - b).max() < 1e-3 * mu_total, np.abs(f - b).max()
