"""Failure detection on the device, without a GPU fault.

The tensor-core SpMM's waits on its mbarriers are bounded (2 s by the global
timer).  A test hook makes its producer issue no copies, so the consumers'
waits run out with nothing in flight: the call must end, the plan's status
word must report DC_ETIMEOUT, and the next call on the same plan must succeed
with the same result as before (tensor memory freed, no MMA left running).
"""
import os

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


def test_spmm_bounded_wait_runs_out_and_plan_recovers(dc):
    import torch
    p = synth.config1(32)                  # one beam, 256 row-blocks: one wave of CTAs
    plan = dc.dc_fspb_create_from(p)
    dc.dc_fspb_spmm_prepare(plan)
    F = torch.from_numpy(np.random.default_rng(5).uniform(0, 1, (plan.n_beamlets, 16))
                         .astype(np.float32)).cuda()
    Y_ref = torch.empty(plan.n_voxels, 16, device="cuda")
    dc.dc_fspb_spmm(plan, F, Y_ref)
    dc.dc_fspb_device_status(plan)
    Y = torch.empty_like(Y_ref)
    os.environ["DC_FSPB_TEST_SPMM_STALL"] = "1"
    try:
        dc.dc_fspb_spmm(plan, F, Y)
        with pytest.raises(dc.DcError) as ei:
            dc.dc_fspb_device_status(plan)
    finally:
        del os.environ["DC_FSPB_TEST_SPMM_STALL"]
    assert ei.value.status == dc.DC_ETIMEOUT
    # the plan and the context stay usable, and the result is unchanged
    Y2 = torch.full_like(Y_ref, float("nan"))
    dc.dc_fspb_spmm(plan, F, Y2)
    dc.dc_fspb_device_status(plan)
    assert torch.equal(Y2, Y_ref)
