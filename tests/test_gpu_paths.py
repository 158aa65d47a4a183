"""GPU tests of internal paths that the parity cases do not force on their own
(through the C ABI, against the FP64 oracle or the library's other path):

* the single-fluence dose pass records the per-(voxel, beam) pair counts; the
  matrix built from them equals the one built after a separate count pass;
* the Siddon trace splits each ray over the 32 lanes of a warp and falls back
  to one lane for rays with more segments per piece than its buffer holds
  (rays of ~1000 voxel crossings here, FP64 sums: rays > 40 cm);
* dc_fspb_dose_and_matrix fills the matrix and accumulates eq. (1) in one
  pass: both results bit-identical to the separate calls, into device
  buffers, pageable host buffers and page-locked host buffers;
* the SpMM numbers its tile columns in 4 x 4 beamlet patches, including
  beamlet grids whose sides are not multiples of 4, and a one-beam plan zeroes
  the output rows of voxels that are in no beam list.
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


def test_dose_pass_counts_give_the_same_matrix(dc):
    p = synth.config2(0.375)          # 48 x 48 x 36 thorax, 9 fields
    a = dc.dc_fspb_create_from(p)
    b = dc.dc_fspb_create_from(p)
    # a: pattern from the count pass; b: from the counts the dose pass records
    na = dc.dc_fspb_pair_count(a)
    dc.dc_fspb_dose(b, p.fluence)
    nb = dc.dc_fspb_pair_count(b)
    assert na == nb > 0
    ra, ca, va = dc.dc_fspb_dose_matrix(a)
    rb, cb, vb = dc.dc_fspb_dose_matrix(b)
    assert np.array_equal(ra, rb) and np.array_equal(ca, cb) and np.array_equal(va, vb)
    # and again after a new density (the recorded counts must not outlive it)
    rho2 = np.ascontiguousarray(p.rho * np.float32(1.05))
    dc.dc_fspb_set_density(b, rho2)
    dc.dc_fspb_dose(b, p.fluence)
    c = dc.dc_fspb_create_from(p)
    dc.dc_fspb_set_density(c, rho2)
    assert dc.dc_fspb_pair_count(b) == dc.dc_fspb_pair_count(c)
    assert np.array_equal(dc.dc_fspb_dose_matrix(b)[1], dc.dc_fspb_dose_matrix(c)[1])


@pytest.mark.parametrize("value_dtype", [0, 1])
def test_dose_and_matrix_in_one_pass(dc, value_dtype):
    import torch
    p = synth.config2(0.375)
    a = dc.dc_fspb_create_from(p)
    b = dc.dc_fspb_create_from(p)
    # b: fresh plan, the pattern comes from a count pass inside the call
    dose_b, rb, cb, vb = dc.dc_fspb_dose_and_matrix(b, p.fluence, value_dtype=value_dtype)
    dose_a = dc.dc_fspb_dose(a, p.fluence)
    ra, ca, va = dc.dc_fspb_dose_matrix(a, value_dtype)
    assert np.array_equal(dose_a, dose_b)
    assert np.array_equal(ra, rb) and np.array_equal(ca, cb) and np.array_equal(va, vb)
    # device buffers, a second fluence, after a new density
    rho2 = np.ascontiguousarray(p.rho * np.float32(0.97))
    for pl in (a, b):
        dc.dc_fspb_set_density(pl, rho2)
    f2 = np.ascontiguousarray(p.fluence[::-1], np.float32)
    nnz = dc.dc_fspb_pair_count(b)
    vt = torch.float32 if value_dtype == 0 else torch.int16
    d_dev = torch.full(p.grid.shape, float("nan"), device="cuda")
    r_dev = torch.empty(p.grid.n_voxels + 1, dtype=torch.int64, device="cuda")
    c_dev = torch.empty(nnz, dtype=torch.int32, device="cuda")
    v_dev = torch.empty(nnz, dtype=vt, device="cuda")
    dc.dc_fspb_dose_and_matrix(b, torch.from_numpy(f2).cuda(), d_dev, value_dtype, r_dev, c_dev, v_dev)
    torch.cuda.synchronize()
    dose_a = dc.dc_fspb_dose(a, f2)
    ra, ca, va = dc.dc_fspb_dose_matrix(a, value_dtype)
    assert np.array_equal(d_dev.cpu().numpy(), dose_a)
    assert np.array_equal(r_dev.cpu().numpy(), ra) and np.array_equal(c_dev.cpu().numpy(), ca)
    assert np.array_equal(v_dev.cpu().numpy().view(va.dtype), va)
    # page-locked host buffers: the same dose and matrix, and the guard cells
    # past nnz stay untouched
    pin = lambda n, dt: torch.empty(n, dtype=dt, pin_memory=True).numpy()
    d_h = pin(p.grid.n_voxels, torch.float32).reshape(p.grid.shape)
    r_h = pin(p.grid.n_voxels + 1, torch.int64)
    c_h = pin(nnz + 8, torch.int32)
    v_h = pin(nnz + 8, vt)
    c_h[nnz:] = -7
    v_h.view(np.uint8)[:] = 0xAB
    guard_v = v_h[nnz:].copy()
    f2c = np.ascontiguousarray(f2)
    dc.dc_fspb_dose_and_matrix(b, f2c, d_h, value_dtype, r_h, c_h, v_h.view(va.dtype))
    assert np.array_equal(d_h, dose_a)
    assert np.array_equal(r_h, ra) and np.array_equal(c_h[:nnz], ca)
    assert np.array_equal(v_h[:nnz].view(va.dtype), va)
    assert np.all(c_h[nnz:] == -7) and np.array_equal(v_h[nnz:], guard_v)


def test_long_rays_take_the_single_lane_trace(dc, oracle_mod):
    # 960 voxels of 0.1 cm along x, the beam along -x: ~960 crossings per ray
    g = synth.centred_grid(960, 4, 4, 0.1)
    rho = np.ones(g.shape, np.float32)
    rho[:, :, 300:420] = 0.3          # a low-density slab along the path
    comm = synth.make_commissioning(synth.COEFF_SEED, roi_radius=0.3)
    beams = [synth.Beam(90.0, 100.0, (0.0, 0.0, 0.0), 0.4, 0.4)]
    p = synth.Plan("longray", g, rho, beams, 0.2, 0.2, comm, np.zeros(0, np.float32))
    p.fluence = synth.uniform_fluence(p.n_beamlets, 5)
    plan = dc.dc_fspb_create_from(p)
    op = oracle_mod.OraclePlan(p)
    rec = dc.dc_fspb_get_beamlets(plan)
    for i in range(op.B):
        o = op.beamlet(i)
        assert o["hit"] and o["K"] > 1500
        assert abs(rec[i, 11] - o["L_in"]) < 2e-5 * o["L_in"]
        assert abs(rec[i, 12] - o["L_out"]) < 2e-5 * o["L_out"]
        assert abs(int(rec[i, 13]) - o["K"]) <= 1
        T, W1, W2 = dc.dc_fspb_get_tables(plan, i)
        To, W1o, W2o = op.table(i)
        k = min(len(T), len(To))
        scale = max(1.0, float(np.abs(To).max()))
        assert np.abs(T[:k] - To[:k]).max() < 2e-5 * scale
        assert np.abs(W2[:k] - W2o[:k]).max() < 2e-6 * scale
    want, amb = op.dose(with_amb=True)
    assert_dose_close(dc.dc_fspb_dose(plan, p.fluence), want, amb, label="long rays")


def _ragged_plan(n_beams):
    # fields of 7 x 5 and 3 x 6 beamlets of 0.5 cm inside a wider grid: most
    # voxels are in no beam list, and no beamlet grid side is a multiple of 4
    g = synth.centred_grid(40, 36, 24, 0.3)
    rho = synth.slab_phantom(g, (2.0, 5.0), 0.4)
    comm = synth.make_commissioning(synth.COEFF_SEED, roi_radius=1.0)
    beams = [synth.Beam(0.0, 100.0, (0.0, 0.0, 0.0), 3.5, 2.5), synth.Beam(70.0, 100.0, (0.3, 0.0, 0.0), 1.5, 3.0)]
    p = synth.Plan("ragged", g, rho, beams[:n_beams], 0.5, 0.5, comm, np.zeros(0, np.float32))
    p.fluence = synth.uniform_fluence(p.n_beamlets, 9)
    return p


@pytest.mark.parametrize("n_beams", [1, 2])
def test_spmm_ragged_patches_and_unlisted_rows(dc, n_beams):
    import torch
    p = _ragged_plan(n_beams)
    plan = dc.dc_fspb_create_from(p)
    dc.dc_fspb_spmm_prepare(plan)
    k = 24
    rng = np.random.default_rng(11)
    F = rng.uniform(0, 1, (plan.n_beamlets, k)).astype(np.float32)
    Fd = torch.from_numpy(F).cuda()
    for rep in range(2):
        Y = torch.full((plan.n_voxels, k), float("nan"), device="cuda")   # no row may keep this
        dc.dc_fspb_spmm(plan, Fd, Y)
        dc.dc_fspb_device_status(plan)
        y = Y.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(y)), f"call {rep}: rows left unwritten"
    D = dc.dc_fspb_dose_batch(plan, np.ascontiguousarray(F.T))          # FP32 direct, [k, V]
    D = D.reshape(k, -1).T.astype(np.float64)
    colmax = np.abs(D).max(0)
    assert np.all(colmax > 0)
    assert np.all(np.abs(y - D) <= 1e-2 * colmax)      # BF16 storage bar
    assert np.all(y[np.abs(D).max(1) == 0] == 0.0)     # voxels no pair reaches
    assert (np.abs(D).max(1) == 0).mean() > 0.3         # the case has many of them


def test_plan_without_body_gives_empty_results(dc, oracle_mod):
    """Every beamlet axis misses the body (air everywhere): no pair exists, so
    the dose is zero, the matrix has no entry, and the SpMM gives zeros."""
    g = synth.centred_grid(10, 12, 8, 0.5)
    rho = np.full(g.shape, 0.001, np.float32)
    for n_beams in (1, 2):
        beams = [synth.Beam(90.0 * b, 100.0, (0, 0, 0), 3.0, 3.0) for b in range(n_beams)]
        p = synth.Plan("air", g, rho, beams, 0.5, 0.5, synth.make_commissioning(roi_radius=1.0),
                       np.ones(36 * n_beams, np.float32))
        want = oracle_mod.OraclePlan(p).dose()
        assert np.all(want == 0)
        plan = dc.dc_fspb_create_from(p)
        assert dc.dc_fspb_pair_count(plan) == 0
        assert np.all(dc.dc_fspb_dose(plan, p.fluence) == 0)
        rowptr, cols, vals = dc.dc_fspb_dose_matrix(plan)
        assert np.all(rowptr == 0) and cols.size == 0 and vals.size == 0
        dose, rowptr, cols, vals = dc.dc_fspb_dose_and_matrix(plan, p.fluence)
        assert np.all(dose == 0) and np.all(rowptr == 0) and cols.size == 0
        dc.dc_fspb_spmm_prepare(plan)
        F = np.ones((plan.n_beamlets, 4), np.float32)
        Y = dc.dc_fspb_spmm(plan, F)
        assert np.all(Y == 0)
        dc.dc_fspb_destroy(plan)
