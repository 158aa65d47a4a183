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


def test_allocation_failure_reports_enomem_and_frees_everything(dc):
    # host-side injection: the N-th device allocation fails; plan creation
    # must report DC_ENOMEM and release what it had allocated, for every N
    import torch
    p = synth.small_plan(90, n=(16, 14, 12), vox=0.3, n_beams=2)
    dc.dc_fspb_destroy(dc.dc_fspb_create_from(p))       # the CUDA runtime's first-use allocations
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    for n in range(1, 200):
        os.environ["DC_FSPB_FAIL_ALLOC_AT"] = str(n)
        try:
            plan = dc.dc_fspb_create_from(p)
        except dc.DcError as e:
            assert e.status == dc.DC_ENOMEM, (n, str(e))
            failed += 1
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] >= free0, n
            continue
        finally:
            del os.environ["DC_FSPB_FAIL_ALLOC_AT"]
        dc.dc_fspb_destroy(plan)      # n is past the last allocation: creation succeeds
        break
    assert failed >= 20, failed
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0


_CHECKED_RUN = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from paper_1103_1164_gb300 import dc_fspb as dc, synth
out = {{}}
cases = [(95, dict(n=(13, 11, 9), vox=0.35, n_beams=3, couch=True)),
         (96, dict(n=(17, 9, 7), vox=0.3, n_beams=2, beamlet=0.2, beamlet_y=0.5)),
         (97, dict(n=(10, 12, 14), vox=0.25, n_beams=1, field=3.0)),
         (98, None)]                     # the thorax plan at 3/8 scale: 9 fields, 5,601 beamlets
for seed, kw in cases:
    p = synth.small_plan(seed, **kw) if kw is not None else synth.config2(0.375)
    plan = dc.dc_fspb_create_from(p)
    out[f"dose{{seed}}"] = dc.dc_fspb_dose(plan, p.fluence)
    d, rowptr, cols, vals = dc.dc_fspb_dose_and_matrix(plan, p.fluence)
    out[f"fused{{seed}}"] = d
    out[f"rowptr{{seed}}"] = rowptr
    out[f"cols{{seed}}"] = cols
    out[f"vals{{seed}}"] = vals
    # the SpMM tiles come from their own pair passes (mark, tile fill)
    dc.dc_fspb_spmm_prepare(plan)
    F = np.random.default_rng(seed).uniform(0, 1, (plan.n_beamlets, 4)).astype(np.float32)
    out[f"spmm{{seed}}"] = dc.dc_fspb_spmm(plan, F)
    dc.dc_fspb_device_status(plan)
np.savez({out!r}, **out)
print("run ok")
"""


def test_bounds_checked_build_runs_clean_and_identical(dc, tmp_path):
    # the DC_BOUNDS_CHECK build guards every index of the pair kernels; on
    # tiny ragged grids and a reduced thorax plan it must report no violation
    # and give the normal build's results bit for bit
    import subprocess
    import sys
    from paper_1103_1164_gb300 import build
    build.build(checked=True)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for tag, checked in (("plain", "0"), ("checked", "1")):
        out = str(tmp_path / f"{tag}.npz")
        env = dict(os.environ, DC_FSPB_CHECKED=checked)
        r = subprocess.run([sys.executable, "-c", _CHECKED_RUN.format(root=root, out=out)], env=env,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        res[tag] = dict(np.load(out))
    assert res["plain"].keys() == res["checked"].keys()
    for k in res["plain"]:
        assert np.array_equal(res["plain"][k], res["checked"][k]), k
