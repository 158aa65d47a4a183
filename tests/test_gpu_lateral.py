"""Lateral-correction forms on the GPU: axis stencils, samples, the network's
trainer and inference, and the network-corrected dose.

Bars: axis-form dose within 0.5 % of the oracle's maximum (the plain-path
bar); stencil samples equal to the oracle's (nearest taps exact, effective
densities to 1e-5); GPU FP32 gradients within 1e-4 of the oracle's FP64
analytic gradients (themselves pinned by finite differences); BF16 inference
within 2e-2 of the FP64 forward; the network-corrected dose within 1 % of the
plain axis form, closer to it than the paper's form is, and within 1 % of the
FP64 oracle's axis-form dose per voxel.
"""
import numpy as np
import pytest

from paper_1103_1164_gb300 import synth
from parity_util import assert_dose_close

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


@pytest.mark.parametrize("seed,kw", [(51, {}), (52, dict(couch=True, n_beams=3)),
                                     (53, dict(n=(21, 19, 15), vox=0.25, roi=1.2, field=2.5))])
def test_axis_dose_matches_oracle(dc, oracle_mod, seed, kw):
    p = synth.small_plan(seed, **kw)
    plan = dc.dc_fspb_create_from(p, lateral_mode=dc.DC_LATERAL_AXIS)
    got = dc.dc_fspb_dose(plan, p.fluence)
    want, amb = oracle_mod.OraclePlan(p, lateral_mode=1).dose(with_amb=True)
    assert_dose_close(got, want, amb, label=f"axis{seed}")


def test_axis_dose_config1_and_mode_switch(dc, oracle_mod):
    p = synth.config1()
    plan = dc.dc_fspb_create_from(p)
    iso = dc.dc_fspb_dose(plan, p.fluence)
    dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_AXIS)
    axis = dc.dc_fspb_dose(plan, p.fluence)
    want, amb = oracle_mod.OraclePlan(p, lateral_mode=1).dose(with_amb=True)
    assert_dose_close(axis, want, amb, label="axis slab64")
    dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_ISO)
    assert np.array_equal(dc.dc_fspb_dose(plan, p.fluence), iso)


def test_stencil_samples_match_oracle(dc, oracle_mod):
    p = synth.small_plan(54, n=(20, 18, 16), vox=0.3, n_beams=3, couch=True)
    plan = dc.dc_fspb_create_from(p)
    op = oracle_mod.OraclePlan(p, lateral_mode=1)
    rng = np.random.default_rng(3)
    vox = rng.integers(0, op.V, 300).astype(np.int32)
    beam = rng.integers(0, 3, 300).astype(np.int32)
    X, T = dc.dc_fspb_stencils(plan, vox, beam)
    exact = 0
    for s in range(300):
        taps, near, eff = op.axis_stencil(vox[s], beam[s])
        exact += int(np.array_equal(X[s].astype(np.float64), near))
        assert np.abs(T[s] - eff).max() < 1e-5
    assert exact >= 297      # nearest-voxel ties at exact half-voxel positions may round either way


def test_mlp_gradient_matches_oracle(dc):
    from oracle import mlp as omlp
    from paper_1103_1164_gb300 import surrogate
    rng = np.random.default_rng(4)
    th = surrogate.init_params(5) + rng.normal(0, 0.05, omlp.N_PARAMS).astype(np.float32)
    p = synth.small_plan(55, n=(20, 18, 16), vox=0.3, n_beams=3)
    plan = dc.dc_fspb_create_from(p)
    X, T = dc.dc_fspb_stencils(plan, rng.integers(0, plan.n_voxels, 1000).astype(np.int32),
                               rng.integers(0, 3, 1000).astype(np.int32))
    net = dc.Mlp(th)
    loss, g = net.gradient(X, T)
    lo, go = omlp.loss_grad(th.astype(np.float64), X, T)
    assert abs(loss - lo) <= 1e-5 * max(1.0, lo)
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    # one Adam step with lr moves against the gradient
    loss1 = net.train(X, T, batch=1000, epochs=1, lr=1e-3)
    assert loss1 < loss


def test_mlp_bf16_inference_matches_fp64_forward(dc):
    from oracle import mlp as omlp
    from paper_1103_1164_gb300 import surrogate
    th = surrogate.init_params(6)
    X = np.random.default_rng(7).uniform(0.05, 2.0, (333, 48)).astype(np.float32)
    Y = dc.dc_mlp_predict(th, X)
    Yo = omlp.forward(th.astype(np.float64), X)
    assert np.abs(Y - Yo).max() < 2e-2


def test_trained_surrogate_dose(dc, oracle_mod):
    from paper_1103_1164_gb300 import surrogate
    X, T = surrogate.generate_samples(n_phantoms=48, per_phantom=4000, seed=77)
    n_tr = int(0.9 * X.shape[0])
    params, loss = surrogate.train(X[:n_tr], T[:n_tr], epochs=8, batch=2048, lr=3e-3, seed=8)
    assert np.isfinite(loss) and loss < 2e-3
    pred = dc.dc_mlp_predict(params, X[n_tr:])
    held = np.abs(pred - T[n_tr:]).max(1)          # held-out error in density units
    assert np.median(held) < 0.01 and np.percentile(held, 99) < 0.1
    p = synth.config1()
    plan = dc.dc_fspb_create_from(p, lateral_mode=dc.DC_LATERAL_AXIS)
    axis = dc.dc_fspb_dose(plan, p.fluence)
    dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_ISO)
    iso = dc.dc_fspb_dose(plan, p.fluence)
    dc.dc_fspb_set_surrogate(plan, params, surrogate.RHO_LO, surrogate.RHO_HI)
    dc.dc_fspb_set_lateral_mode(plan, dc.DC_LATERAL_MLP)
    net = dc.dc_fspb_dose(plan, p.fluence)
    assert dc.dc_fspb_lateral_fallbacks(plan) == 0       # the slab phantom is inside the training range
    dmax = float(axis.max())
    err_net = float(np.abs(net - axis).max()) / dmax
    err_iso = float(np.abs(iso - axis).max()) / dmax
    assert err_net <= 1e-2, err_net
    assert err_net < err_iso, (err_net, err_iso)
    # the network-corrected dose against the FP64 oracle's axis form, per voxel:
    # the surrogate bar (1 % of the oracle's maximum, plus the dose of pairs
    # whose ROI or depth decision lies within rounding of its boundary)
    want, amb = oracle_mod.OraclePlan(p, lateral_mode=1).dose(with_amb=True)
    assert_dose_close(net, want, amb, tol=1e-2, label="network slab64 vs FP64 oracle")


def test_trainer_checkpoint_resumes_bit_for_bit(dc, tmp_path):
    # a trainer saved after one epoch and resumed in a new trainer takes the
    # same steps as the original (deterministic FP32 training, Adam state and
    # step count restored)
    from paper_1103_1164_gb300 import checkpoint as ck, surrogate
    X, T = surrogate.generate_samples(n_phantoms=4, per_phantom=2000, seed=91)
    a = dc.Mlp(surrogate.init_params(3))
    a.train(X, T, batch=500, epochs=1, lr=2e-3)
    path = str(tmp_path / "trainer.npz")
    ck.save_trainer(path, a, extra={"epochs": 1})
    b = ck.load_trainer(path)
    a.train(X, T, batch=500, epochs=1, lr=2e-3)
    b.train(X, T, batch=500, epochs=1, lr=2e-3)
    sa, sb = a.state(), b.state()
    for x, y in zip(sa[:3], sb[:3]):
        assert np.array_equal(x, y)
    assert sa[3] == sb[3] == 2 * (X.shape[0] // 500)


def test_mlp_bf16_gradient_matches_oracle(dc):
    # the tensor-core BF16 gradient kernel against the FP64 analytic gradient:
    # BF16 operands (8 significant bits) in the products, so the bound is the
    # BF16 one (3 % of the gradient's norm), far below the gradient's own scale
    from oracle import mlp as omlp
    from paper_1103_1164_gb300 import surrogate
    rng = np.random.default_rng(14)
    th = surrogate.init_params(15) + rng.normal(0, 0.05, omlp.N_PARAMS).astype(np.float32)
    p = synth.small_plan(56, n=(20, 18, 16), vox=0.3, n_beams=3)
    plan = dc.dc_fspb_create_from(p)
    X, T = dc.dc_fspb_stencils(plan, rng.integers(0, plan.n_voxels, 1000).astype(np.int32),
                               rng.integers(0, 3, 1000).astype(np.int32))
    net = dc.Mlp(th, precision=dc.DC_PRECISION_BF16)
    loss, g = net.gradient(X, T)
    lo, go = omlp.loss_grad(th.astype(np.float64), X, T)
    assert abs(loss - lo) <= 2e-2 * lo
    assert np.linalg.norm(g - go) <= 3e-2 * np.linalg.norm(go)
    assert np.abs(g - go).max() <= 5e-2 * np.abs(go).max()
    # every parameter block is written (no stale or missing partials)
    for a, b in ((0, 48 * 64), (48 * 64, 48 * 64 + 64), (48 * 64 + 64, 48 * 64 + 64 + 4096),
                 (7491 - 195, 7491 - 3), (7491 - 3, 7491)):
        assert np.linalg.norm(g[a:b] - go[a:b]) <= 5e-2 * np.linalg.norm(go[a:b]) + 1e-9, (a, b)
    # deterministic: the same gradient twice
    _, g2 = net.gradient(X, T)
    assert np.array_equal(g, g2)


def test_bf16_training_matches_fp32_training(dc):
    # the network trained with the BF16 gradient reaches the held-out error of
    # the FP32-trained one (same data, same schedule)
    from paper_1103_1164_gb300 import surrogate
    X, T = surrogate.generate_samples(n_phantoms=48, per_phantom=4000, seed=78)
    n_tr = int(0.9 * X.shape[0])
    perm = np.random.default_rng(9).permutation(n_tr)
    held = {}
    for prec in (dc.DC_PRECISION_FP32, dc.DC_PRECISION_BF16):
        net = dc.Mlp(surrogate.init_params(9), precision=prec)
        loss = net.train(X[perm], T[perm], batch=2048, epochs=8, lr=3e-3)
        assert np.isfinite(loss)
        pred = dc.dc_mlp_predict(net.params(), X[n_tr:])
        held[prec] = float(np.median(np.abs(pred - T[n_tr:]).max(1)))
    assert held[dc.DC_PRECISION_BF16] < 0.01
    assert held[dc.DC_PRECISION_BF16] <= 2.0 * held[dc.DC_PRECISION_FP32] + 1e-3, held
