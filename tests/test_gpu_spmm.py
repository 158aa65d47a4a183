"""Tensor-core BF16 SpMM (multi-fluence dose, eq. 1 for k fluence vectors).

Two bars:
* data path: against the exact product of the BF16 matrix the library stores
  and the BF16-rounded fluences, evaluated in FP64 here, the only difference is
  FP32 accumulation order, so the bound is tight (1e-5 of the column maximum);
* method: against the FP64 oracle's matrix times the unrounded fluences, the
  BF16 storage bound applies: 1 % of each fluence column's maximum dose.
"""
import numpy as np
import pytest
from scipy import sparse

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


def bf16_round(x):
    """Round-to-nearest-even to BF16, returned as float64 (library-independent)."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _matrix_dense_ops(dc, plan, V, B):
    rowptr, cols, vals = dc.dc_fspb_dose_matrix(plan, dc.DC_BF16)
    m = (vals.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return sparse.csr_matrix((m, cols, rowptr), shape=(V, B))


def _check(dc, oracle_mod, p, k, seed):
    plan = dc.dc_fspb_create_from(p)
    dc.dc_fspb_spmm_prepare(plan)
    chunks, rbs = dc.dc_fspb_spmm_info(plan)
    assert chunks > 0 and rbs > 0
    rng = np.random.default_rng(seed)
    F = rng.uniform(0, 1, (plan.n_beamlets, k)).astype(np.float32)
    Y = dc.dc_fspb_spmm(plan, F)
    assert Y.shape == (plan.n_voxels, k) and np.all(np.isfinite(Y))
    # data path: exact BF16 x BF16 product, FP64 here
    Mb = _matrix_dense_ops(dc, plan, plan.n_voxels, plan.n_beamlets)
    Yx = Mb @ bf16_round(F)
    colmax = np.abs(Yx).max(0) + 1e-30
    assert np.all(np.abs(Y - Yx) <= 1e-5 * colmax + 1e-7), float((np.abs(Y - Yx) / colmax).max())
    # method: FP64 oracle matrix (entries inside ROI and depth range) times F
    op = oracle_mod.OraclePlan(p)
    o_ptr, o_cols, o_vals, o_flags = op.matrix()
    inside = (o_flags & 1).astype(np.float64)
    Mo = sparse.csr_matrix((o_vals * inside, o_cols, o_ptr), shape=(op.V, op.B))
    Yo = Mo @ F.astype(np.float64)
    amb_rows = np.zeros(op.V, bool)
    amb_rows[np.repeat(np.arange(op.V), np.diff(o_ptr))[(o_flags & 2).astype(bool)]] = True
    err = np.abs(Y - Yo) / (np.abs(Yo).max(0) + 1e-30)
    assert err[~amb_rows].max() <= 1e-2, float(err[~amb_rows].max())
    return float(err[~amb_rows].max()), plan, F, Y


def test_spmm_single_beam_config1_64_fluences(dc, oracle_mod):
    worst, plan, F, Y = _check(dc, oracle_mod, synth.config1(), 64, 7)
    # and against the FP32 direct path for the same fluences
    D = dc.dc_fspb_dose_batch(plan, np.ascontiguousarray(F.T)).reshape(64, -1).T
    scale = np.abs(D).max(0)
    assert np.all(np.abs(Y - D) <= 1e-2 * scale)


@pytest.mark.parametrize("k", [1, 5, 16])
def test_spmm_multi_beam(dc, oracle_mod, k):
    p = synth.small_plan(31, n=(26, 22, 18), vox=0.3, n_beams=3, roi=2.0, field=4.0)
    _check(dc, oracle_mod, p, k, 11 + k)


def test_spmm_device_pointers(dc):
    import torch
    p = synth.small_plan(32, n=(24, 20, 16), vox=0.3, n_beams=2, roi=2.0, field=3.0)
    plan = dc.dc_fspb_create_from(p)
    dc.dc_fspb_spmm_prepare(plan)
    F = torch.rand(plan.n_beamlets, 64, device="cuda")
    Y = torch.empty(plan.n_voxels, 64, device="cuda")
    dc.dc_fspb_spmm(plan, F, Y)
    dc.dc_fspb_device_status(plan)
    host = dc.dc_fspb_spmm(plan, F.cpu().numpy())
    assert np.array_equal(Y.cpu().numpy(), host)
