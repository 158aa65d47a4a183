"""Several plans in one persistent, graph-replayed launch (dc_fspb_batch_*).

Bars:
* against each plan's own dc_fspb_dose: the batch runs the same per-pair
  arithmetic and sums each voxel's pairs and beams in the same order, so the
  bound is 1e-6 of the plan's maximum dose;
* against the FP64 oracle: the single-plan bar (0.5 % of the maximum dose per
  voxel, plus the pairs whose ROI or depth decision lies within rounding).
The full 16-plan head-and-neck batch (grids up to 256 x 256 x 192, 5-9 beams,
0.25 cm beamlets) is checked on seeded voxel samples of its largest and
smallest plans.
"""
import numpy as np
import pytest

from paper_1103_1164_gb300 import synth
from parity_util import assert_dose_close

pytestmark = pytest.mark.gpu

SAME = 1e-6


@pytest.fixture(scope="module")
def dc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1103_1164_gb300 import build, dc_fspb
    build.build()
    dc_fspb.load()
    return dc_fspb


def _uneven(dc):
    """Four small plans: merged and unmerged tables (voxel 0.25 vs 0.35 cm),
    1-4 beams, the paper's and the axis-stencil lateral forms, and one plan
    without the density correction."""
    specs = [(synth.small_plan(40, n=(20, 16, 12), vox=0.25, n_beams=3, roi=1.5, field=3.0), dc.DC_LATERAL_ISO),
             (synth.small_plan(41, n=(14, 12, 10), vox=0.35, n_beams=2), dc.DC_LATERAL_AXIS),
             (synth.small_plan(42, n=(24, 10, 8), vox=0.3, n_beams=4, density_correction=0, field=2.0),
              dc.DC_LATERAL_ISO),
             (synth.small_plan(43, n=(12, 12, 12), vox=0.25, n_beams=1, couch=True), dc.DC_LATERAL_AXIS)]
    inputs = [s[0] for s in specs]
    plans = [dc.dc_fspb_create_from(p, lateral_mode=m) for p, m in specs]
    return inputs, plans


def _groups(inputs, modes, dc):
    """Plan groups of the batch: per-voxel or per-item lateral factors."""
    return len({bool(p.comm.density_correction) and m != dc.DC_LATERAL_ISO for p, m in zip(inputs, modes)})


def _close(a, b, label):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    scale = float(np.abs(b).max())
    assert scale > 0, label
    err = float(np.abs(a - b).max() / scale)
    assert err <= SAME, f"{label}: {err:.3e}"


class _DeviceArray:
    """A float32 device buffer of the library, viewed by torch without a copy."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False),
                                         "version": 3, "strides": None}


def _device_view(ptr, n):
    import torch
    return torch.as_tensor(_DeviceArray(ptr, n), device="cuda")


def test_batch_matches_single_plans_and_oracle(dc, oracle_mod):
    inputs, plans = _uneven(dc)
    single = [dc.dc_fspb_dose(pl, p.fluence) for p, pl in zip(inputs, plans)]
    batch = dc.dc_fspb_batch_create(plans)
    flu = [np.ascontiguousarray(p.fluence, np.float32) for p in inputs]
    for rep in range(2):   # first run captures the graph, the second replays it
        got = dc.dc_fspb_batch_dose(batch, flu)
        for j in range(len(plans)):
            _close(got[j], single[j], f"plan {j} run {rep}")
    # one prefix and one persistent pair kernel per plan group, one beam sum
    modes = [dc.DC_LATERAL_ISO, dc.DC_LATERAL_AXIS, dc.DC_LATERAL_ISO, dc.DC_LATERAL_AXIS]
    assert _groups(inputs, modes, dc) == 2
    assert dc.dc_fspb_batch_kernels(batch) == 1 + 2 * 2
    for j, p in enumerate(inputs):
        want, amb = oracle_mod.OraclePlan(p, lateral_mode=1 if j in (1, 3) else 0).dose(with_amb=True)
        assert_dose_close(got[j], want, amb, label=f"batch plan {j}")
    # with the density-dependent steps in the graph: same doses
    got = dc.dc_fspb_batch_dose(batch, flu, density=True)
    for j in range(len(plans)):
        _close(got[j], single[j], f"plan {j} density run")
    assert dc.dc_fspb_batch_kernels(batch, density=True) > 3 * len(plans)


def test_batch_device_buffers_and_new_fluence(dc):
    import torch
    inputs, plans = _uneven(dc)
    batch = dc.dc_fspb_batch_create(plans)
    rng = np.random.default_rng(5)
    flu = [torch.from_numpy(rng.uniform(0, 1, pl.n_beamlets).astype(np.float32)).cuda() for pl in plans]
    out = [torch.full((pl.n_voxels,), float("nan"), device="cuda") for pl in plans]
    dc.dc_fspb_batch_dose(batch, flu, out)
    for j, pl in enumerate(plans):
        want = dc.dc_fspb_dose(pl, flu[j].cpu().numpy())
        _close(out[j].cpu().numpy(), want, f"plan {j} device buffers")
    # the batch's own buffers, filled in place, then a bare replay
    for j, pl in enumerate(plans):
        fptr, dptr = dc.dc_fspb_batch_buffers(batch, j)
        assert fptr and dptr
        _device_view(fptr, pl.n_beamlets).copy_(flu[j])
    dc.dc_fspb_batch_run(batch)
    dc.dc_fspb_batch_synchronize(batch)
    for j, pl in enumerate(plans):
        _, dptr = dc.dc_fspb_batch_buffers(batch, j)
        _close(_device_view(dptr, pl.n_voxels).cpu().numpy(), out[j].cpu().numpy(), f"plan {j} bare replay")


def test_batch_follows_plan_changes(dc):
    inputs, plans = _uneven(dc)
    batch = dc.dc_fspb_batch_create(plans)
    flu = [np.ascontiguousarray(p.fluence, np.float32) for p in inputs]
    dc.dc_fspb_batch_dose(batch, flu)
    # another lateral form on plan 0 and another binning on plan 1
    dc.dc_fspb_set_lateral_mode(plans[0], dc.DC_LATERAL_AXIS)
    dc.dc_fspb_autotune(plans[1], flu[1])
    got = dc.dc_fspb_batch_dose(batch, flu)
    for j, (p, pl) in enumerate(zip(inputs, plans)):
        _close(got[j], dc.dc_fspb_dose(pl, p.fluence), f"plan {j} after changes")
    # every form of the pair work gives the same doses; the plans' own
    # launches (variant 2) give each plan's dc_fspb_dose bit for bit
    variant, ms = dc.dc_fspb_batch_autotune(batch)
    assert variant in (0, 1, 2) and ms > 0
    again = dc.dc_fspb_batch_dose(batch, flu)
    for j in range(len(plans)):
        _close(again[j], got[j], f"plan {j} after autotune")
    for v in (0, 1, 2):
        dc.dc_fspb_batch_set_variant(batch, v)
        for density in (False, True):
            res = dc.dc_fspb_batch_dose(batch, flu, density=density)
            for j, (p, pl) in enumerate(zip(inputs, plans)):
                own = dc.dc_fspb_dose(pl, p.fluence)
                if v == 2:
                    assert np.array_equal(np.reshape(res[j], -1), np.reshape(own, -1)), \
                        f"plan {j}, per-plan launches, density {density}"
                else:
                    _close(res[j], own, f"plan {j}, variant {v}, density {density}")
    with pytest.raises(dc.DcError) as ei:
        dc.dc_fspb_batch_set_variant(batch, 3)
    assert ei.value.status == dc.DC_EINVAL


def test_batch_rejects_bad_arguments(dc):
    inputs, plans = _uneven(dc)
    with pytest.raises(dc.DcError) as ei:
        dc.dc_fspb_batch_create([plans[0], plans[1], plans[0]])
    assert ei.value.status == dc.DC_EINVAL
    with pytest.raises(dc.DcError) as ei:
        dc.dc_fspb_batch_create([])
    assert ei.value.status == dc.DC_EINVAL
    batch = dc.dc_fspb_batch_create(plans[:2])
    with pytest.raises(dc.DcError):
        dc.dc_fspb_batch_buffers(batch, 2)


def test_head_neck_batch_full_size_sampled(dc, oracle_mod):
    # the 16 uneven head-and-neck plans, in the launch configuration the
    # benchmark times; every plan against its own single-plan launch, the
    # largest and smallest plans against the oracle on seeded voxel samples
    inputs = synth.config5_plans()
    plans = [dc.dc_fspb_create_from(p) for p in inputs]
    batch = dc.dc_fspb_batch_create(plans)
    got = dc.dc_fspb_batch_dose(batch, [np.ascontiguousarray(p.fluence, np.float32) for p in inputs])
    # one lateral form: one persistent pair launch for all 16 plans (one of
    # them has merged tables, the others not)
    assert dc.dc_fspb_batch_kernels(batch) == 3
    for j, (p, pl) in enumerate(zip(inputs, plans)):
        _close(got[j], dc.dc_fspb_dose(pl, p.fluence), f"hn{j}")
    sizes = [pl.n_voxels for pl in plans]
    rng = np.random.default_rng(1005)
    for j in (int(np.argmax(sizes)), int(np.argmin(sizes))):
        op = oracle_mod.OraclePlan(inputs[j])
        d = np.asarray(got[j]).reshape(-1)
        # half the sample where the dose is above 10 % of the maximum
        hot = np.flatnonzero(d > 0.1 * d.max())
        vox = np.unique(np.concatenate([rng.integers(0, op.V, 400), rng.choice(hot, 400)]))
        want, amb = op.dose_voxels(vox, with_amb=True)
        err = np.abs(d[vox] - want)
        dmax = float(d.max())
        assert np.all(err <= 5e-3 * dmax + amb), (j, float((err / dmax).max()))
