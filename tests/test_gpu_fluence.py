"""Beamlet fluence from MLC leaf sequences on the GPU (dc_fluence_from_leaves)
against the FP64 oracle, and the leaf-sequence -> fluence -> dose chain.

Bar: |f_gpu - f_oracle| <= 2e-5 of the sequence's total meterset per beamlet
(FP32 sums of up to a few hundred interval terms against FP64).
"""
import numpy as np
import pytest

from paper_1103_1164_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1103_1164_gb300 import build, dc_fspb
    build.build()
    dc_fspb.load()
    return dc_fspb


@pytest.fixture(scope="module")
def ofl():
    from oracle import fluence
    return fluence


def _plan(fields, bx=0.2, by=0.5):
    g = synth.centred_grid(16, 14, 12, 0.4, 0.4, 0.25)
    beams = [synth.Beam(40.0 * k, 100.0, (0.0, 0.0, 0.0), fx, fy) for k, (fx, fy) in enumerate(fields)]
    comm = synth.make_commissioning(synth.COEFF_SEED, roi_radius=1.5)
    p = synth.Plan("leaf", g, np.ones(g.shape, np.float32), beams, bx, by, comm, np.zeros(0, np.float32))
    return p


def _close(got, want, seqs, plan_inputs):
    off = 0
    for s, n in zip(seqs, plan_inputs.beamlets_per_beam):
        tol = 2e-5 * float(np.max(s.mu))
        err = np.abs(np.asarray(got[off:off + n], np.float64) - want[off:off + n])
        assert err.max() <= tol + 1e-30, (err.max(), tol)
        off += n


@pytest.mark.parametrize("kind,kw", [
    ("sliding", dict(n_cp=64, transmission=0.015)),
    ("sliding", dict(n_cp=7, offset=0.25, jaw_margin=-0.3)),
    ("shoot", dict(n_seg=6, transmission=0.02, offset=0.1)),
    ("shoot", dict(n_seg=1, width=1.0, jaw_margin=0.2)),
])
def test_fluence_matches_oracle(dc, ofl, kind, kw):
    # three beams with ragged fields (rows and columns not multiples of a warp)
    p = _plan([(3.0, 2.5), (4.6, 1.5), (1.0, 3.5)])
    plan = dc.dc_fspb_create_from(p)
    seqs = synth.plan_sequences(p, 5 if kind == "sliding" else 6, kind, **kw)
    got = dc.dc_fluence_from_leaves(plan, seqs)
    want = ofl.plan_fluence(p, seqs)
    assert want.max() > 0
    _close(got, want, seqs, p)


def test_device_output_equals_host_output(dc):
    import torch
    p = _plan([(3.0, 2.5), (2.0, 2.0)])
    plan = dc.dc_fspb_create_from(p)
    seqs = synth.plan_sequences(p, 9, "sliding", n_cp=33)
    host = dc.dc_fluence_from_leaves(plan, seqs)
    dev = torch.full((plan.n_beamlets,), float("nan"), device="cuda")
    dc.dc_fluence_from_leaves(plan, seqs, dev)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)


def test_degenerate_sequences(dc, ofl):
    p = _plan([(2.0, 2.0)])
    plan = dc.dc_fspb_create_from(p)
    base = synth.plan_sequences(p, 3, "sliding", n_cp=9)[0]
    nl = base.n_leaves
    # one control point: no meterset, no fluence
    one = synth.LeafSequence(base.edges, base.mu[:1], base.left[:1], base.right[:1], base.jaws, 0.02)
    assert np.all(dc.dc_fluence_from_leaves(plan, [one]) == 0.0)
    # all leaves closed, 2 % transmission: 2 % of the meterset where the jaws are open
    z = np.zeros((2, nl), np.float32)
    closed = synth.LeafSequence(base.edges, np.array([0.0, 50.0], np.float32), z, z, (-0.5, 1.0, -1.0, 1.0), 0.02)
    got = dc.dc_fluence_from_leaves(plan, [closed])
    want = ofl.plan_fluence(p, [closed])
    assert np.abs(got - want).max() <= 1e-5 * 50.0 and np.isclose(want.max(), 1.0)
    # jaws shut: nothing
    shut = synth.LeafSequence(base.edges, base.mu, base.left, base.right, (0.3, 0.3, -1.0, 1.0), 0.0)
    assert np.all(dc.dc_fluence_from_leaves(plan, [shut]) == 0.0)
    # a leaf bank narrower than the field: rows outside it get nothing
    edges = np.array([-0.5, 0.0, 0.5], np.float32)
    o = np.full((2, 2), 5.0, np.float32)
    narrow = synth.LeafSequence(edges, np.array([0.0, 10.0], np.float32), -o, o, (-1.0, 1.0, -1.0, 1.0), 0.0)
    got = dc.dc_fluence_from_leaves(plan, [narrow]).reshape(4, 10)
    assert np.all(got[[0, 3]] == 0.0) and np.allclose(got[[1, 2]], 10.0)


def test_rejects_bad_sequences(dc):
    p = _plan([(2.0, 2.0)])
    plan = dc.dc_fspb_create_from(p)
    s = synth.plan_sequences(p, 4, "sliding", n_cp=5)[0]
    bad_lr = synth.LeafSequence(s.edges, s.mu, s.right + 1.0, s.right, s.jaws, 0.0)
    bad_mu = synth.LeafSequence(s.edges, s.mu[::-1].copy(), s.left, s.right, s.jaws, 0.0)
    bad_edges = synth.LeafSequence(s.edges[::-1].copy(), s.mu, s.left, s.right, s.jaws, 0.0)
    bad_tau = synth.LeafSequence(s.edges, s.mu, s.left, s.right, s.jaws, 1.5)
    nan = s.left.copy(); nan[2, 1] = np.nan
    bad_nan = synth.LeafSequence(s.edges, s.mu, nan, s.right, s.jaws, 0.0)
    bad_jaws = synth.LeafSequence(s.edges, s.mu, s.left, s.right, (1.0, -1.0, -1.0, 1.0), 0.0)
    for b in (bad_lr, bad_mu, bad_edges, bad_tau, bad_nan, bad_jaws):
        with pytest.raises(dc.DcError):
            dc.dc_fluence_from_leaves(plan, [b])
    with pytest.raises(ValueError):
        dc.dc_fluence_from_leaves(plan, [s, s])


def test_table1_case_leaf_sequences_to_dose(dc, ofl, oracle_mod):
    # the nasal-cavity case (8 non-coplanar beams, 3,382 beamlets of
    # 0.2 x 0.5 cm) delivered by sliding-window sequences of 96 control points:
    # the fluence of every beamlet against the oracle, then the dose from the
    # library's fluence against the oracle's dose from the oracle's fluence on
    # seeded voxels
    p = synth.table1_case("H3")
    seqs = synth.plan_sequences(p, 1102, "sliding", n_cp=96, transmission=0.015)
    plan = dc.dc_fspb_create_from(p)
    f = dc.dc_fluence_from_leaves(plan, seqs)
    fo = ofl.plan_fluence(p, seqs)
    _close(f, fo, seqs, p)
    d = np.asarray(dc.dc_fspb_dose(plan, f)).reshape(-1)
    op = oracle_mod.OraclePlan(p)
    rng = np.random.default_rng(77)
    hot = np.flatnonzero(d > 0.1 * d.max())
    vox = np.unique(np.concatenate([rng.integers(0, op.V, 800), rng.choice(hot, 800)]))
    want, amb = op.dose_voxels(vox, fluence=fo, with_amb=True)
    dmax = float(d.max())
    assert np.all(np.abs(d[vox] - want) <= 5e-3 * dmax + amb)
