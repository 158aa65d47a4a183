"""The reduced-precision form of the direct dose (DC_PRECISION_BF16) and the
surrogate + BF16 form of the multi-plan batch.

Bars: against the FP64 oracle, the surrogate bar (1 % of the maximum dose per
voxel, plus the dose of pairs whose ROI or depth decision lies within
rounding); a plan's share of a batch equals its own single-plan launch in the
same precision to 1e-6 of its maximum (same per-pair arithmetic, same sums).
"""
import numpy as np
import pytest

from paper_1103_1164_gb300 import synth
from parity_util import assert_dose_close

pytestmark = pytest.mark.gpu

SURROGATE_TOL = 1e-2


@pytest.fixture(scope="module")
def dc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1103_1164_gb300 import build, dc_fspb
    build.build()
    dc_fspb.load()
    return dc_fspb


@pytest.mark.parametrize("seed,kw", [(70, {}), (71, dict(couch=True, n_beams=3)),
                                     (72, dict(n=(22, 20, 16), vox=0.25, roi=2.0, field=3.0, beamlet=0.25)),
                                     (73, dict(beamlet=0.2, beamlet_y=0.5, field=2.0, n_beams=3))])
def test_bf16_dose_matches_oracle(dc, oracle_mod, seed, kw):
    p = synth.small_plan(seed, **kw)
    plan = dc.dc_fspb_create_from(p)
    f32 = dc.dc_fspb_dose(plan, p.fluence)
    dc.dc_fspb_set_precision(plan, dc.DC_PRECISION_BF16)
    bf = dc.dc_fspb_dose(plan, p.fluence)
    want, amb = oracle_mod.OraclePlan(p).dose(with_amb=True)
    assert_dose_close(bf, want, amb, tol=SURROGATE_TOL, label=f"bf16 small{seed}")
    assert np.abs(bf - f32).max() > 0          # the reduced-precision kernel ran
    dc.dc_fspb_set_precision(plan, dc.DC_PRECISION_FP32)
    assert np.array_equal(dc.dc_fspb_dose(plan, p.fluence), f32)


def test_bf16_slab64_and_rejects_unknown(dc, oracle_mod):
    p = synth.config1()
    plan = dc.dc_fspb_create_from(p)
    dc.dc_fspb_set_precision(plan, dc.DC_PRECISION_BF16)
    got = dc.dc_fspb_dose(plan, p.fluence)
    want, amb = oracle_mod.OraclePlan(p).dose(with_amb=True)
    assert_dose_close(got, want, amb, tol=SURROGATE_TOL, label="bf16 slab64")
    with pytest.raises(dc.DcError) as ei:
        dc.dc_fspb_set_precision(plan, 7)
    assert ei.value.status == dc.DC_EINVAL


def test_mixed_precision_batch_equals_single_plans(dc):
    specs = [(synth.small_plan(74, n=(20, 16, 12), vox=0.25, n_beams=3, roi=1.5, field=3.0), dc.DC_LATERAL_ISO,
              dc.DC_PRECISION_BF16),
             (synth.small_plan(75, n=(14, 12, 10), vox=0.35, n_beams=2), dc.DC_LATERAL_AXIS, dc.DC_PRECISION_BF16),
             (synth.small_plan(76, n=(16, 14, 12), vox=0.25, n_beams=2), dc.DC_LATERAL_ISO, dc.DC_PRECISION_FP32),
             (synth.small_plan(77, n=(12, 12, 12), vox=0.25, n_beams=1, couch=True), dc.DC_LATERAL_AXIS,
              dc.DC_PRECISION_FP32)]
    plans = []
    for p, mode, prec in specs:
        pl = dc.dc_fspb_create_from(p, lateral_mode=mode)
        dc.dc_fspb_set_precision(pl, prec)
        plans.append(pl)
    batch = dc.dc_fspb_batch_create(plans)
    got = dc.dc_fspb_batch_dose(batch, [np.ascontiguousarray(s[0].fluence, np.float32) for s in specs])
    for j, ((p, _, _), pl) in enumerate(zip(specs, plans)):
        own = dc.dc_fspb_dose(pl, p.fluence)
        scale = float(np.abs(own).max())
        assert scale > 0
        assert float(np.abs(np.asarray(got[j]).reshape(-1) - own.reshape(-1)).max()) <= 1e-6 * scale, j
    # four groups (per-voxel / per-item factors x FP32 / BF16): four pair launches
    # plus a prefix launch each and the beam sums
    assert dc.dc_fspb_batch_kernels(batch) == 9


def test_surrogate_bf16_head_neck_batch_against_oracle(dc, oracle_mod):
    # the 16-plan head-and-neck batch in the surrogate + BF16 form, as the
    # benchmark runs it: network densities (axis fallback outside the training
    # range) and packed-BF16 exponentials; the largest and the smallest plan
    # against the oracle's axis form on seeded voxels
    from paper_1103_1164_gb300 import surrogate
    X, T = surrogate.generate_samples(n_phantoms=48, per_phantom=4000, seed=77)
    params, loss = surrogate.train(X, T, epochs=8, batch=2048, lr=3e-3, seed=8)
    assert np.isfinite(loss)
    inputs = synth.config5_plans()
    plans = [dc.dc_fspb_create_from(p) for p in inputs]
    for pl in plans:
        dc.dc_fspb_set_surrogate(pl, params, surrogate.RHO_LO, surrogate.RHO_HI)
        dc.dc_fspb_set_lateral_mode(pl, dc.DC_LATERAL_MLP)
        dc.dc_fspb_set_precision(pl, dc.DC_PRECISION_BF16)
    batch = dc.dc_fspb_batch_create(plans)
    got = dc.dc_fspb_batch_dose(batch, [np.ascontiguousarray(p.fluence, np.float32) for p in inputs],
                                density=True)
    sizes = [pl.n_voxels for pl in plans]
    rng = np.random.default_rng(1006)
    for j in (int(np.argmax(sizes)), int(np.argmin(sizes))):
        d = np.asarray(got[j]).reshape(-1)
        hot = np.flatnonzero(d > 0.1 * d.max())
        vox = np.unique(np.concatenate([rng.integers(0, d.size, 400), rng.choice(hot, 400)]))
        want, amb = oracle_mod.OraclePlan(inputs[j], lateral_mode=1).dose_voxels(vox, with_amb=True)
        err = np.abs(d[vox] - want)
        dmax = float(d.max())
        assert np.all(err <= SURROGATE_TOL * dmax + amb), (j, float((err / dmax).max()))


def _bf16_round(x):
    """Round-to-nearest-even to BF16, returned as float64 (library-independent)."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("k,seed,kw", [(2, 80, dict(n_beams=3, couch=True)),
                                       (17, 81, dict(n=(26, 22, 18), vox=0.3, n_beams=3, roi=2.0, field=4.0)),
                                       (64, 82, dict(beamlet=0.2, beamlet_y=0.5, field=2.0, n_beams=2))])
def test_bf16_tensor_core_dose_batch(dc, oracle_mod, k, seed, kw):
    # dc_fspb_dose_batch with k > 1 in the reduced-precision setting: the pair
    # values and fluences rounded to BF16, their products summed on the tensor
    # cores.  Data path: the exact product of the library's BF16 matrix entries
    # (the same FP32 pair values, rounded the same way) and the BF16 fluences,
    # in FP64 here, up to FP32 summation order.  Method: the FP64 oracle's
    # matrix times the unrounded fluences, the BF16 bar of 1 % of each
    # vector's maximum dose (rows with an ambiguous pair left out).
    from scipy import sparse
    p = synth.small_plan(seed, **kw)
    plan = dc.dc_fspb_create_from(p)
    V, B = plan.n_voxels, plan.n_beamlets
    rng = np.random.default_rng(seed)
    F = rng.uniform(0, 1, (k, B)).astype(np.float32)
    rowptr, cols, vals = dc.dc_fspb_dose_matrix(plan, dc.DC_BF16)
    Mb = sparse.csr_matrix(((vals.astype(np.uint32) << 16).view(np.float32).astype(np.float64), cols, rowptr),
                           shape=(V, B))
    f32 = dc.dc_fspb_dose_batch(plan, F).reshape(k, V).astype(np.float64)
    dc.dc_fspb_set_precision(plan, dc.DC_PRECISION_BF16)
    got = dc.dc_fspb_dose_batch(plan, F).reshape(k, V).astype(np.float64)
    dc.dc_fspb_device_status(plan)
    assert np.all(np.isfinite(got))
    exact = np.asarray((Mb @ _bf16_round(F).T).T)
    colmax = np.abs(exact).max(1, keepdims=True) + 1e-30
    assert np.all(np.abs(got - exact) <= 1e-4 * colmax), float((np.abs(got - exact) / colmax).max())
    op = oracle_mod.OraclePlan(p)
    o_ptr, o_cols, o_vals, o_flags = op.matrix()
    Mo = sparse.csr_matrix((o_vals * (o_flags & 1), o_cols, o_ptr), shape=(op.V, op.B))
    want = np.asarray((Mo @ F.astype(np.float64).T).T)
    amb_rows = np.zeros(op.V, bool)
    amb_rows[np.repeat(np.arange(op.V), np.diff(o_ptr))[(o_flags & 2).astype(bool)]] = True
    err = np.abs(got - want) / (np.abs(want).max(1, keepdims=True) + 1e-30)
    assert err[:, ~amb_rows].max() <= 1e-2, float(err[:, ~amb_rows].max())
    assert np.abs(got - f32).max() > 0                     # the tensor-core form ran
    # a single vector keeps the direct form's own reduced-precision kernel
    one = dc.dc_fspb_dose_batch(plan, np.ascontiguousarray(F[:1])).reshape(-1)
    assert np.array_equal(one, dc.dc_fspb_dose(plan, np.ascontiguousarray(F[0])).reshape(-1))
