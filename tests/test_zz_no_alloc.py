"""dc_fspb_spmm_noalloc: the tensor-core SpMM with static scratch.

The variant must give what dc_fspb_spmm gives (same kernels, same arithmetic;
only where the packed fluences and partial rows live differs) on two calls in
a row, for a single-beam plan (output written directly) and a multi-beam plan
(partials in the static array, reduced in beam order), must leave the
device's free memory unchanged, and must reject problems larger than its fixed
scratch with DC_EINVAL.
"""
import numpy as np
import pytest

from paper_1103_1164_gb300 import synth

pytestmark = pytest.mark.gpu

# bound on |noalloc - spmm| relative to each fluence column's maximum: the
# two paths run the same kernels in the same order
TOL = 1e-6


@pytest.fixture(scope="module")
def dc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1103_1164_gb300 import build, dc_fspb
    build.build()
    dc_fspb.load()
    return dc_fspb


def _two_calls(dc, p, k, seed):
    import torch
    plan = dc.dc_fspb_create_from(p)
    dc.dc_fspb_spmm_prepare(plan)
    rng = np.random.default_rng(seed)
    for call in range(2):
        F = torch.from_numpy(rng.uniform(0, 1, (plan.n_beamlets, k)).astype(np.float32)).cuda()
        Y_ref = torch.full((plan.n_voxels, k), float("nan"), device="cuda")
        Y = torch.full((plan.n_voxels, k), float("nan"), device="cuda")
        dc.dc_fspb_spmm(plan, F, Y_ref)
        dc.dc_fspb_spmm_noalloc(plan, F, Y)
        dc.dc_fspb_device_status(plan)
        a, r = Y.cpu().numpy(), Y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), f"call {call}: output not written in full"
        colmax = np.abs(r).max(0) + 1e-30
        err = float((np.abs(a - r) / colmax).max())
        assert err <= TOL, f"call {call}: {err}"
        assert np.abs(r).max() > 0
    return plan


def test_noalloc_single_beam(dc):
    _two_calls(dc, synth.config1(32), 64, 3)


@pytest.mark.parametrize("k", [5, 16])
def test_noalloc_multi_beam(dc, k):
    p = synth.small_plan(31, n=(26, 22, 18), vox=0.3, n_beams=3, roi=2.0, field=4.0)
    _two_calls(dc, p, k, 100 + k)


def test_noalloc_allocates_no_device_memory(dc):
    # the defining property: after a first call (which looks up the static
    # arrays' addresses), further calls leave the device's free memory as it was
    import torch
    p = synth.small_plan(32, n=(26, 22, 18), vox=0.3, n_beams=3, roi=2.0, field=4.0)
    plan = dc.dc_fspb_create_from(p)
    dc.dc_fspb_spmm_prepare(plan)
    F = torch.rand(plan.n_beamlets, 16, device="cuda")
    Y = torch.zeros(plan.n_voxels, 16, device="cuda")
    dc.dc_fspb_spmm_noalloc(plan, F, Y)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        dc.dc_fspb_spmm_noalloc(plan, F, Y)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    dc.dc_fspb_device_status(plan)
    assert free1 >= free0, (free0, free1)


def test_noalloc_rejects_oversize(dc):
    import torch
    p = synth.config2(0.5)
    plan = dc.dc_fspb_create_from(p)
    dc.dc_fspb_spmm_prepare(plan)
    _, n_rb = dc.dc_fspb_spmm_info(plan)
    n_beams = len(p.beams)
    k = 64
    # every row-block but the last of each beam holds 128 list entries
    assert (n_rb - n_beams) * 128 * k > dc.DC_SPMM_STATIC_MAX_PARTIALS
    F = torch.rand(plan.n_beamlets, k, device="cuda")
    Y = torch.zeros(plan.n_voxels, k, device="cuda")
    with pytest.raises(dc.DcError) as ei:
        dc.dc_fspb_spmm_noalloc(plan, F, Y)
    assert ei.value.status == dc.DC_EINVAL
    assert "static scratch" in str(ei.value)
    # the plan stays usable
    dc.dc_fspb_spmm(plan, F, Y)
    dc.dc_fspb_device_status(plan)
